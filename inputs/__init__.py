"""Seeded synthetic task-DAG workloads (generators only, no scheduling arithmetic).

The C generators in ``gen.c`` build random layered DAGs (the auto-generated
layered graphs of Sec. 4.4 / Sec. 5.2) and tiled Cholesky / LU / QR DAGs
(Sec. 5.3) with integer nanosecond cost tables.  This module wraps them with
ctypes and returns numpy arrays in the batch layout the library consumes:

    task_base[ndag+1]  int64   first task of DAG d in the concatenated arrays
    edge_base[ndag+1]  int64   first edge of DAG d
    row_ptr[n_total+ndag] int32  DAG d's n_d+1 local edge offsets start at task_base[d]+d
    col_idx[m_total]   int32   local successor ids, ascending within each row
    type[n_total]      uint8
    type_cost[ndag, n_types, 2] int64 (CPU ns, GPU ns)
    task_cost[n_total, 2] int64 or None (per-task costs override type costs)

Both the CUDA path and the oracle are fed from these arrays; neither side
generates its own inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libinspgen.so")
_SRC = os.path.join(_HERE, "gen.c")
_lock = threading.Lock()
_lib = None

BASE_SEED = 20240403

KIND_CHOLESKY, KIND_LU, KIND_QR = 0, 1, 2
KIND_NAMES = {KIND_CHOLESKY: "cholesky", KIND_LU: "lu", KIND_QR: "qr"}

US = 1000  # ns per microsecond

# Per-type (CPU, GPU) base costs in ns.
CHOLESKY_COST = np.array([[200, 150], [400, 60], [400, 60], [800, 40]], dtype=np.int64) * US  # POTRF TRSM SYRK GEMM
LU_COST = np.array([[300, 200], [400, 60], [800, 40]], dtype=np.int64) * US  # GETRF TRSM GEMM
QR_COST = np.array([[500, 300], [800, 120], [800, 200], [1600, 100]], dtype=np.int64) * US  # GEQRT UNMQR TSQRT TSMQR
TILED_COST = {KIND_CHOLESKY: CHOLESKY_COST, KIND_LU: LU_COST, KIND_QR: QR_COST}


class _LayeredParams(ctypes.Structure):
    _fields_ = [
        ("n_min", ctypes.c_int32), ("n_max", ctypes.c_int32),
        ("w_min", ctypes.c_int32), ("w_max", ctypes.c_int32),
        ("p_min", ctypes.c_double), ("p_max", ctypes.c_double),
        ("d_min", ctypes.c_int32), ("d_max", ctypes.c_int32),
        ("n_types", ctypes.c_int32),
        ("cost_median_ns", ctypes.c_double), ("cost_sigma", ctypes.c_double),
        ("speed_min", ctypes.c_double), ("speed_max", ctypes.c_double), ("typing", ctypes.c_int32),
    ]


class _CBatch(ctypes.Structure):
    _fields_ = [
        ("ndag", ctypes.c_int32), ("n_types", ctypes.c_int32),
        ("n_total", ctypes.c_int64), ("m_total", ctypes.c_int64),
        ("task_base", ctypes.POINTER(ctypes.c_int64)),
        ("edge_base", ctypes.POINTER(ctypes.c_int64)),
        ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
        ("col_idx", ctypes.POINTER(ctypes.c_int32)),
        ("type", ctypes.POINTER(ctypes.c_uint8)),
        ("type_cost", ctypes.POINTER(ctypes.c_int64)),
        ("task_cost", ctypes.POINTER(ctypes.c_int64)),
    ]


def build(force: bool = False) -> str:
    """Compile gen.c into libinspgen.so (host C, gcc)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.insg_layered.restype = ctypes.POINTER(_CBatch)
        lib.insg_layered.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.POINTER(_LayeredParams)]
        lib.insg_tiled.restype = ctypes.POINTER(_CBatch)
        lib.insg_tiled.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
        lib.insg_free.argtypes = [ctypes.POINTER(_CBatch)]
        lib.insg_tiled_count.restype = ctypes.c_int64
        lib.insg_tiled_count.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.insg_mixed.restype = ctypes.POINTER(_CBatch)
        lib.insg_mixed.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.POINTER(_LayeredParams), ctypes.POINTER(ctypes.c_int64)]
        lib.insg_mixed_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        lib.insg_dag_seed.restype = ctypes.c_uint64
        lib.insg_dag_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        _lib = lib
    return _lib


@dataclass
class Machine:
    """A modelled heterogeneous machine: workers 0..n_cpu-1 are CPUs, then GPUs."""
    n_cpu: int
    n_gpu: int
    xfer_ns: int

    @property
    def n_workers(self) -> int:
        return self.n_cpu + self.n_gpu


@dataclass
class Dag:
    """One DAG in local numbering with per-task resolved costs."""
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    type: np.ndarray
    c_cpu: np.ndarray
    c_gpu: np.ndarray

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) if self.n >= 0 else 0

    def cost(self) -> np.ndarray:
        return np.stack([self.c_cpu, self.c_gpu], axis=1)


@dataclass
class Batch:
    ndag: int
    n_types: int
    task_base: np.ndarray
    edge_base: np.ndarray
    row_ptr: np.ndarray
    col_idx: np.ndarray
    type: np.ndarray
    type_cost: np.ndarray  # (ndag, n_types, 2)
    task_cost: np.ndarray | None  # (n_total, 2) or None

    @property
    def n_total(self) -> int:
        return int(self.task_base[-1])

    @property
    def m_total(self) -> int:
        return int(self.edge_base[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.task_base)

    def dag(self, d: int) -> Dag:
        tb, te = int(self.task_base[d]), int(self.task_base[d + 1])
        eb, ee = int(self.edge_base[d]), int(self.edge_base[d + 1])
        n = te - tb
        rp = self.row_ptr[tb + d: te + d + 1]
        ci = self.col_idx[eb:ee]
        ty = self.type[tb:te]
        if self.task_cost is not None:
            c = self.task_cost[tb:te]
            c_cpu, c_gpu = c[:, 0].copy(), c[:, 1].copy()
        else:
            tc = self.type_cost[d]
            c_cpu = tc[ty.astype(np.int64), 0].copy()
            c_gpu = tc[ty.astype(np.int64), 1].copy()
        return Dag(n, rp, ci, ty, c_cpu, c_gpu)

    def subset(self, idx) -> "Batch":
        """A batch holding the listed DAGs (in the listed order)."""
        return concat_dags([self.dag(int(i)) for i in idx])


def _from_c(ptr) -> Batch:
    if not ptr:
        raise RuntimeError("generator failed (invalid parameters or out of memory)")
    try:
        b = ptr.contents
        nd, nt = b.ndag, b.n_types
        n, m = b.n_total, b.m_total
        tb = np.ctypeslib.as_array(b.task_base, shape=(nd + 1,)).copy()
        eb = np.ctypeslib.as_array(b.edge_base, shape=(nd + 1,)).copy()
        rp = np.ctypeslib.as_array(b.row_ptr, shape=(n + nd,)).copy() if n + nd > 0 else np.zeros(0, np.int32)
        ci = np.ctypeslib.as_array(b.col_idx, shape=(m,)).copy() if m > 0 else np.zeros(0, np.int32)
        ty = np.ctypeslib.as_array(b.type, shape=(n,)).copy() if n > 0 else np.zeros(0, np.uint8)
        tc = (np.ctypeslib.as_array(b.type_cost, shape=(nd * nt * 2,)).copy().reshape(nd, nt, 2)
              if bool(b.type_cost) and nd > 0 else np.ones((nd, nt, 2), np.int64))
        kc = (np.ctypeslib.as_array(b.task_cost, shape=(n * 2,)).copy().reshape(n, 2)
              if bool(b.task_cost) and n > 0 else None)
    finally:
        _load().insg_free(ptr)
    return Batch(nd, nt, tb, eb, rp, ci, ty, tc, kc)


def layered(ndag: int, cfg: int = 2, first: int = 0, *, n_min=50, n_max=2000, w_min=4, w_max=64,
            p_min=0.1, p_max=0.5, d_min=1, d_max=3, n_types=8, cost_median_ns=100 * US,
            cost_sigma=1.0, speed_min=0.5, speed_max=20.0, typing: str = "random", base_seed=BASE_SEED) -> Batch:
    """Random layered DAGs (defaults: the 4096-DAG layered workload's shape).
    typing "degree": 16 task types by in/out degree bucket instead of random types."""
    ty = {"random": 0, "degree": 1}[typing]
    if ty == 1:
        n_types = 16
    p = _LayeredParams(n_min, n_max, w_min, w_max, p_min, p_max, d_min, d_max, n_types,
                       float(cost_median_ns), float(cost_sigma), float(speed_min), float(speed_max), ty)
    return _from_c(_load().insg_layered(base_seed, cfg, first, ndag, ctypes.byref(p)))


def tiled(kind: int, N: int, ndag: int = 1, cfg: int = 3, first: int = 0, *, perturb: bool = True,
          base_cost: np.ndarray | None = None, base_seed=BASE_SEED) -> Batch:
    """ndag instances of a tiled Cholesky / LU / QR DAG of N x N tiles."""
    bc = np.ascontiguousarray(TILED_COST[kind] if base_cost is None else base_cost, dtype=np.int64)
    ptr = _load().insg_tiled(kind, N, base_seed, cfg, first, ndag,
                             bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1 if perturb else 0)
    return _from_c(ptr)


def mixed(ndag: int, cfg: int = 5, first: int = 0, *, n_lo: int = 100, n_hi: int = 200000,
          base_seed=BASE_SEED) -> Batch:
    """The mixed-size stress workload: task counts log-uniform in [n_lo, n_hi]; even DAG indices
    random layered DAGs (the 4096-DAG workload's shape, 8 types), odd ones tiled Cholesky / LU /
    QR DAGs of the largest tile count within the drawn size, per-task costs (+-20 % on the
    tiled ones)."""
    p = _LayeredParams(0, 0, 4, 64, 0.1, 0.5, 1, 3, 8, float(100 * US), 1.0, 0.5, 20.0, 0)
    bc = np.zeros((3, 4, 2), np.int64)
    for k, tab in TILED_COST.items():
        bc[k, :tab.shape[0]] = tab
    bc = np.ascontiguousarray(bc)
    return _from_c(_load().insg_mixed(base_seed, cfg, first, ndag, n_lo, n_hi, ctypes.byref(p),
                                      bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))


def mixed_sizes(ndag: int, cfg: int = 5, first: int = 0, *, n_lo: int = 100, n_hi: int = 200000,
                base_seed=BASE_SEED) -> np.ndarray:
    """The task counts mixed() draws (tiled DAGs round them down to a whole tile count)."""
    out = np.zeros(max(ndag, 1), np.int64)
    _load().insg_mixed_sizes(base_seed, cfg, first, ndag, n_lo, n_hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out[:ndag]


def layered_1m(n: int = 1_000_000, cfg: int = 6, base_seed=BASE_SEED) -> Batch:
    """The one large layered DAG of the mixed-size stress workload: n tasks in layers of 256,
    edge probability 0.05 to the next U{1,2,3} layers, 8 types, log-normal costs."""
    return layered(1, cfg=cfg, n_min=n, n_max=n, w_min=256, w_max=256, p_min=0.05, p_max=0.05,
                   base_seed=base_seed)


def tiled_count(kind: int, N: int) -> int:
    return int(_load().insg_tiled_count(kind, N))


def concat_dags(dags: list[Dag], n_types: int | None = None) -> Batch:
    """Build a batch from per-DAG arrays; costs are stored per task."""
    nd = len(dags)
    ns = np.array([d.n for d in dags], dtype=np.int64)
    ms = np.array([int(d.row_ptr[-1]) if d.n > 0 else 0 for d in dags], dtype=np.int64)
    tb = np.zeros(nd + 1, np.int64); tb[1:] = np.cumsum(ns)
    eb = np.zeros(nd + 1, np.int64); eb[1:] = np.cumsum(ms)
    rp = np.concatenate([np.asarray(d.row_ptr, np.int32) if d.n > 0 else np.zeros(1, np.int32) for d in dags]) \
        if nd else np.zeros(0, np.int32)
    ci = np.concatenate([np.asarray(d.col_idx, np.int32) for d in dags]) if nd else np.zeros(0, np.int32)
    ty = np.concatenate([np.asarray(d.type, np.uint8) for d in dags]) if nd else np.zeros(0, np.uint8)
    nt = n_types or (int(ty.max()) + 1 if ty.size else 1)
    kc = np.concatenate([np.stack([d.c_cpu, d.c_gpu], 1).astype(np.int64) for d in dags]) \
        if nd else np.zeros((0, 2), np.int64)
    tc = np.ones((nd, nt, 2), np.int64)
    return Batch(nd, nt, tb, eb, rp, ci, ty, tc, kc)


def concat(batches: list[Batch]) -> Batch:
    dags = [b.dag(i) for b in batches for i in range(b.ndag)]
    return concat_dags(dags)


def concat_batches(batches: list[Batch]) -> Batch:
    """Concatenate whole batches (per-DAG local row offsets and successor ids stay as they are);
    costs become per task."""
    nt = max(b.n_types for b in batches)
    tb = [np.zeros(1, np.int64)]
    eb = [np.zeros(1, np.int64)]
    n0 = m0 = 0
    costs = []
    tcs = []
    for b in batches:
        tb.append(b.task_base[1:] + n0)
        eb.append(b.edge_base[1:] + m0)
        n0 += b.n_total
        m0 += b.m_total
        if b.task_cost is not None:
            costs.append(np.asarray(b.task_cost, np.int64))
        else:
            d_of = np.repeat(np.arange(b.ndag), np.diff(b.task_base))
            costs.append(b.type_cost[d_of, b.type.astype(np.int64)])
        tc = np.ones((b.ndag, nt, 2), np.int64)
        tc[:, :b.n_types] = b.type_cost
        tcs.append(tc)
    return Batch(sum(b.ndag for b in batches), nt, np.concatenate(tb), np.concatenate(eb),
                 np.concatenate([b.row_ptr for b in batches]), np.concatenate([b.col_idx for b in batches]),
                 np.concatenate([b.type for b in batches]), np.concatenate(tcs), np.concatenate(costs))


def make_dag(n: int, edges, c_cpu, c_gpu, type=None) -> Dag:
    """A small DAG from an edge list (u, v) with u < v (tests and examples)."""
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
    rp = np.zeros(n + 1, np.int32)
    ci = []
    for u in range(n):
        r = sorted(rows[u])
        ci.extend(r)
        rp[u + 1] = rp[u] + len(r)
    ty = np.zeros(n, np.uint8) if type is None else np.asarray(type, np.uint8)
    return Dag(n, rp, np.asarray(ci, np.int32), ty, np.asarray(c_cpu, np.int64), np.asarray(c_gpu, np.int64))


# ----------------------------------------------------------------- workloads
# Machines of the five workloads (CPU workers, GPU workers, transfer ns).
MACHINE_CHOLESKY8 = Machine(4, 1, 20 * US)
MACHINE_LAYERED = Machine(8, 2, 20 * US)
MACHINE_TILED = Machine(16, 4, 20 * US)
MACHINE_MIXED = Machine(32, 8, 20 * US)


def mixed_workload(ndag: int = 10000, with_large: bool = True) -> Batch:
    """The mixed-size stress batch: `ndag` DAGs of mixed() and, with_large, the 1M-task layered
    DAG after them (all with per-task costs)."""
    parts = [mixed(ndag)]
    if with_large:
        parts.append(layered_1m())
    return concat_batches(parts) if len(parts) > 1 else parts[0]


def cholesky8() -> Batch:
    """Tiled Cholesky of 8x8 tiles (120 tasks), per-type costs, one DAG."""
    return tiled(KIND_CHOLESKY, 8, 1, cfg=1, perturb=False)


def layered4096(ndag: int = 4096, first: int = 0) -> Batch:
    """The 4096 random layered DAGs (or a prefix / window of them)."""
    return layered(ndag, cfg=2, first=first)


def layered4096_degree(ndag: int = 4096, first: int = 0) -> Batch:
    """The same 4096 layered DAG shapes with task types by in/out degree."""
    return layered(ndag, cfg=2, first=first, typing="degree")


def tiled_workload(Ns=(16, 32, 64), instances: int = 256, kinds=(KIND_CHOLESKY, KIND_LU, KIND_QR)) -> Batch:
    """Cholesky / LU / QR at the listed tile counts, `instances` perturbed instances each."""
    parts = []
    cfg_index = 0
    for kind in kinds:
        for N in Ns:
            parts.append(tiled(kind, N, instances, cfg=3, first=cfg_index << 20))
            cfg_index += 1
    return concat(parts) if len(parts) > 1 else parts[0]
