"""CPU ORACLE -- test infrastructure only.

Plain, slow restatement of INSPIRIT's schedule evaluation (arxiv 2404.03226),
used by the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline.
The library never imports it and it imports nothing from the library: the two
share only the seeded input generators in ``inputs``.

The arithmetic lives in ``oracle.c`` (single-threaded C, compiled with gcc);
this module compiles it on demand and wraps it with ctypes.  See the header of
``oracle.c`` for the definitions and readings each function follows.

Parity status: every function here is pinned by CPU tests (closed forms,
brute force on tiny DAGs, hand-traced controller cases, bounds and an
exhaustive optimum); the exact controller decisions on full-size paper-shaped
workloads are "parity unpinned" beyond those pins because the paper prints no
schedule to compare against.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOTTOPO, ENOMEM, EOVERFLOW, ECYCLE = 0, 1, 2, 3, 6, 8
POLICY_INSPIRIT, POLICY_FIFO, POLICY_LEARNED, POLICY_DMDAP_IA, POLICY_DMDAP_BL = 0, 1, 2, 3, 4
MODE_FIFO, MODE_ABILITY, MODE_EFI, MODE_EFI_LOC, MODE_LEARNED, MODE_PRIO = 0, 1, 2, 3, 4, 5
STATE_INC, STATE_DEC = 0, 1
MLP_IN, MLP_H = 16, 64

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i16p = ctypes.POINTER(ctypes.c_int16)


class Policy(ctypes.Structure):
    """Scheduling policy; zero fields take the defaults for P workers (task
    window, s_inc, s_dec, dec_step = P; c = max(1, P/2); k_inc = P tasks per
    unit time)."""
    _fields_ = [("policy", ctypes.c_int32), ("task_window", ctypes.c_int32), ("s_inc", ctypes.c_int32),
                ("s_dec", ctypes.c_int32), ("dec_step", ctypes.c_int32), ("c", ctypes.c_int32),
                ("k_inc_tasks", ctypes.c_int64), ("k_inc_ns", ctypes.c_int64)]


class Ctrl(ctypes.Structure):
    _fields_ = [("peak", ctypes.c_int64), ("prev_n", ctypes.c_int64), ("prev_t", ctypes.c_int64),
                ("count", ctypes.c_int64), ("mode", ctypes.c_int32), ("state", ctypes.c_int32)]


class _Trace(ctypes.Structure):
    _fields_ = [("t", _i64p), ("nready", _i32p), ("mode", _i32p), ("task", _i32p), ("worker", _i32p),
                ("npop", ctypes.c_int32), ("feat_pop", ctypes.c_int32), ("feat_cap", ctypes.c_int32),
                ("n_feat", ctypes.c_int32), ("feat_task", _i32p), ("feat", _i32p),
                ("push_t", _i64p), ("push_task", _i32p), ("push_worker", _i32p), ("push_nready", _i32p),
                ("npush", ctypes.c_int32)]


class _Force(ctypes.Structure):
    _fields_ = [("force_pop", ctypes.c_int32), ("force_task", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_check_dag.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, _i64p, ctypes.c_int64]
        lib.orc_ia.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        lib.orc_renumber.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        lib.orc_ie.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, ctypes.c_int64, _i32p]
        lib.orc_default_unit_time.restype = ctypes.c_int64
        lib.orc_default_unit_time.argtypes = [ctypes.c_int32, _i64p]
        lib.orc_resolve_policy.argtypes = [ctypes.POINTER(Policy), ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(Policy)]
        lib.orc_ctrl_step.argtypes = [ctypes.POINTER(Ctrl), ctypes.POINTER(Policy), ctypes.c_int64, ctypes.c_int64]
        lib.orc_mlp_score.restype = ctypes.c_int64
        lib.orc_mlp_score.argtypes = [_i16p, _i32p]
        lib.orc_mlp_nweights.restype = ctypes.c_int32
        lib.orc_simulate.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, _i64p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, ctypes.POINTER(Policy), ctypes.c_int64, _i32p, _i32p, _i16p,
                                     ctypes.POINTER(_Force), _i32p, _i64p, _i64p, _i64p, ctypes.POINTER(_Trace)]
        lib.orc_validate.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, _i64p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, _i32p, _i64p, _i64p, ctypes.c_int64, _i32p]
        _dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_unit_time_search.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, ctypes.POINTER(ctypes.c_uint8),
                                             ctypes.c_int32, _i64p, _i32p]
        lib.orc_bottom_level.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, _i64p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int64, _i64p]
        lib.orc_mlp_loss_grad.restype = ctypes.c_double
        lib.orc_mlp_loss_grad.argtypes = [ctypes.c_int32] * 3 + [_dp, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _dp]
        lib.orc_adamw.argtypes = [ctypes.c_int32, _dp, _dp, _dp, _dp, ctypes.c_int32] + [ctypes.c_double] * 5
        lib.orc_optimum.restype = ctypes.c_int64
        lib.orc_optimum.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p, _i64p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int64, ctypes.c_int64]
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def check_dag(dag, xfer_ns: int = 0) -> int:
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    return _L().orc_check_dag(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(_i64(dag.c_cpu), _i64p),
                              _p(_i64(dag.c_gpu), _i64p), xfer_ns)


def renumber(dag) -> tuple[int, np.ndarray]:
    """(rc, new_id[old]): the DAG's own ids when they are topological, else Kahn rounds with
    ascending old id within a round; rc ECYCLE for a cycle (see orc_renumber)."""
    out = np.zeros(max(dag.n, 1), np.int32)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx if dag.col_idx.size else np.zeros(1))
    rc = _L().orc_renumber(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(out, _i32p))
    return int(rc), out[:dag.n]


def relabel(dag, new_id):
    """The same DAG with task old -> new_id[old]: rows moved, successors mapped and sorted,
    types and costs moved with their tasks."""
    n = dag.n
    old_of = np.empty(n, np.int64)
    old_of[np.asarray(new_id, np.int64)] = np.arange(n)
    rows = [np.sort(np.asarray(new_id)[dag.col_idx[dag.row_ptr[o]:dag.row_ptr[o + 1]]]) for o in old_of]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows]) if n else []
    ci = np.concatenate(rows).astype(np.int32) if n and rp[-1] else np.zeros(0, np.int32)
    return type(dag)(n, rp, ci, np.asarray(dag.type)[old_of], np.asarray(dag.c_cpu)[old_of],
                     np.asarray(dag.c_gpu)[old_of])


def ia(dag) -> np.ndarray:
    """Inspiring ability: strict descendant count of every task."""
    out = np.zeros(max(dag.n, 1), np.int32)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    rc = _L().orc_ia(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(out, _i32p))
    if rc:
        raise RuntimeError(f"orc_ia failed: {rc}")
    return out[:dag.n]


def ie(dag, unit_time: int | None = None) -> np.ndarray:
    """Inspiring efficiency for unit time T (default: default_unit_time)."""
    T = default_unit_time(dag) if not unit_time else int(unit_time)
    out = np.zeros(max(dag.n, 1), np.int32)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    rc = _L().orc_ie(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(_i64(dag.c_gpu), _i64p), T, _p(out, _i32p))
    if rc:
        raise RuntimeError(f"orc_ie failed: {rc}")
    return out[:dag.n]


def default_unit_time(dag) -> int:
    """4 x the lower median of the DAG's GPU costs (at least 1)."""
    cg = _i64(dag.c_gpu) if dag.n > 0 else np.zeros(1, np.int64)
    return int(_L().orc_default_unit_time(dag.n, _p(cg, _i64p)))


def resolve_policy(policy: Policy, n_workers: int, unit_time: int) -> Policy:
    out = Policy()
    _L().orc_resolve_policy(ctypes.byref(policy), n_workers, unit_time, ctypes.byref(out))
    return out


def ctrl_step(state: Ctrl, policy: Policy, cur: int, now: int) -> Ctrl:
    """Apply one Nready-controller judgement in place; returns the state."""
    _L().orc_ctrl_step(ctypes.byref(state), ctypes.byref(policy), cur, now)
    return state


def mlp_nweights() -> int:
    return int(_L().orc_mlp_nweights())


def mlp_score(weights_k: np.ndarray, feat: np.ndarray) -> int:
    """Score (units of 1/64) of one integer feature vector; weights are int16 grid numerators."""
    w = np.ascontiguousarray(weights_k, dtype=np.int16)
    f = _i32(feat)
    assert w.size == mlp_nweights() and f.size == MLP_IN
    return int(_L().orc_mlp_score(_p(w, _i16p), _p(f, _i32p)))


def simulate(dag, machine, policy: Policy | None = None, unit_time: int | None = None, ia_=None, ie_=None,
             mlp_weights=None, force=None, trace: bool = False, feat_pop: int = -1, feat_cap: int = 0):
    """Run the event simulation; returns a dict with worker/start/end/makespan
    (and the per-pop trace when requested).  ia_/ie_ default to the oracle's
    own attributes for unit_time (default: the DAG's default unit time), and
    unit_time also sets the default ascending slope k_inc = P tasks per
    unit_time ns."""
    pol = policy or Policy()
    T = int(unit_time) if unit_time else default_unit_time(dag)
    a = _i32(ia(dag) if ia_ is None else ia_)
    e = _i32(ie(dag, T) if ie_ is None else ie_)
    n = dag.n
    worker = np.zeros(max(n, 1), np.int32)
    start = np.zeros(max(n, 1), np.int64)
    end = np.zeros(max(n, 1), np.int64)
    mk = np.zeros(1, np.int64)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    cc, cg = _i64(dag.c_cpu), _i64(dag.c_gpu)
    w = None if mlp_weights is None else np.ascontiguousarray(mlp_weights, dtype=np.int16)
    fobj = None
    if force is not None:
        fobj = _Force(int(force[0]), int(force[1]))
    tr = None
    bufs = {}
    if trace or feat_pop >= 0:
        cap = max(n, 1)
        bufs = dict(t=np.zeros(cap, np.int64), nready=np.zeros(cap, np.int32), mode=np.zeros(cap, np.int32),
                    task=np.zeros(cap, np.int32), worker=np.zeros(cap, np.int32),
                    feat_task=np.zeros(max(feat_cap, 1), np.int32), feat=np.zeros(max(feat_cap, 1) * MLP_IN, np.int32),
                    push_t=np.zeros(cap, np.int64), push_task=np.zeros(cap, np.int32),
                    push_worker=np.zeros(cap, np.int32), push_nready=np.zeros(cap, np.int32))
        tr = _Trace(_p(bufs["t"], _i64p), _p(bufs["nready"], _i32p), _p(bufs["mode"], _i32p),
                    _p(bufs["task"], _i32p), _p(bufs["worker"], _i32p), 0, feat_pop, feat_cap, 0,
                    _p(bufs["feat_task"], _i32p), _p(bufs["feat"], _i32p),
                    _p(bufs["push_t"], _i64p) if trace else None, _p(bufs["push_task"], _i32p),
                    _p(bufs["push_worker"], _i32p), _p(bufs["push_nready"], _i32p), 0)
    # k_inc's default is P tasks per T, the unit time the attributes use (Sec. 4.2-4.4 share one
    # unit time window: inspiring efficiency counts releases within it, and the ascending slope
    # is a task count per such window).
    rc = _L().orc_simulate(n, _p(rp, _i32p), _p(ci, _i32p), _p(cc, _i64p), _p(cg, _i64p), machine.n_cpu,
                           machine.n_gpu, machine.xfer_ns, ctypes.byref(pol), T, _p(a, _i32p), _p(e, _i32p),
                           None if w is None else _p(w, _i16p), None if fobj is None else ctypes.byref(fobj),
                           _p(worker, _i32p), _p(start, _i64p), _p(end, _i64p), _p(mk, _i64p),
                           None if tr is None else ctypes.byref(tr))
    out = dict(rc=rc, worker=worker[:n], start=start[:n], end=end[:n], makespan=int(mk[0]), ia=a, ie=e,
               unit_time=T)
    if tr is not None:
        k = tr.npop
        out["trace"] = {key: bufs[key][:k] for key in ("t", "nready", "mode", "task", "worker")}
        out["trace"].update({key: bufs[key][:tr.npush] for key in ("push_t", "push_task", "push_worker",
                                                                     "push_nready")})
        nf = tr.n_feat if feat_pop >= 0 else 0
        out["feat_task"] = bufs["feat_task"][:nf]
        out["feat"] = bufs["feat"][:nf * MLP_IN].reshape(nf, MLP_IN)
    return out


def unit_time_search(dag, k_max: int = 16) -> tuple[int, int]:
    """(T, k): the searched unit time of a DAG and its exponent (see orc_unit_time_search)."""
    T = np.zeros(1, np.int64)
    k = np.zeros(1, np.int32)
    ty = np.ascontiguousarray(dag.type if dag.n > 0 else np.zeros(1), np.uint8)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    rc = _L().orc_unit_time_search(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(_i64(dag.c_gpu) if dag.n else
                                   np.ones(1, np.int64), _i64p), ty.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   k_max, _p(T, _i64p), _p(k, _i32p))
    assert rc == OK
    return int(T[0]), int(k[0])


def bottom_level(dag, machine) -> np.ndarray:
    """Static priority of the DMDAP baseline: HEFT upward rank over mean costs (int64 per task)."""
    bl = np.zeros(max(dag.n, 1), np.int64)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    rc = _L().orc_bottom_level(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(_i64(dag.c_cpu), _i64p),
                               _p(_i64(dag.c_gpu), _i64p), machine.n_cpu, machine.n_gpu, machine.xfer_ns, _p(bl, _i64p))
    assert rc == OK
    return bl[:dag.n]


def validate(dag, machine, worker, start, end, makespan) -> tuple[int, int]:
    """(code, task): code 0 if feasible; see orc_validate for the rule codes."""
    bad = np.zeros(1, np.int32)
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    code = _L().orc_validate(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(_i64(dag.c_cpu), _i64p),
                             _p(_i64(dag.c_gpu), _i64p), machine.n_cpu, machine.n_gpu, machine.xfer_ns,
                             _p(_i32(worker), _i32p), _p(_i64(start), _i64p), _p(_i64(end), _i64p),
                             int(makespan), _p(bad, _i32p))
    return int(code), int(bad[0])


def optimum(dag, machine, upper_bound: int = 0) -> int:
    """Exact minimum makespan by branch and bound (n <= 10 recommended)."""
    rp, ci = _i32(dag.row_ptr), _i32(dag.col_idx)
    return int(_L().orc_optimum(dag.n, _p(rp, _i32p), _p(ci, _i32p), _p(_i64(dag.c_cpu), _i64p),
                                _p(_i64(dag.c_gpu), _i64p), machine.n_cpu, machine.n_gpu, machine.xfer_ns,
                                upper_bound))


def simulate_batch(batch, machine, policy: Policy | None = None, idx=None, unit_time: int | None = None):
    """Simulate DAGs of a batch one after another (single thread)."""
    res = []
    for d in (range(batch.ndag) if idx is None else idx):
        res.append(simulate(batch.dag(int(d)), machine, policy, unit_time))
    return res


def mlp_nweights_dims(inp: int, h1: int, h2: int) -> int:
    return inp * h1 + h1 + h1 * h2 + h2 + h2 + 1


def mlp_loss_grad(w, x, target, dims=(16, 64, 64), mode: int = 1):
    """(loss, grad) of the scorer's training loss in fp64; mode 0 smooth, 1
    quantisation-aware with straight-through estimators (see oracle.c)."""
    _dp = ctypes.POINTER(ctypes.c_double)
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(target, np.float64)
    g = np.zeros_like(w)
    n = t.size
    loss = _L().orc_mlp_loss_grad(dims[0], dims[1], dims[2], w.ctypes.data_as(_dp), mode, n, x.ctypes.data_as(_dp),
                                  t.ctypes.data_as(_dp), g.ctypes.data_as(_dp))
    return float(loss), g


def adamw(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step in place (fp64)."""
    _dp = ctypes.POINTER(ctypes.c_double)
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    _L().orc_adamw(w.size, w.ctypes.data_as(_dp), m.ctypes.data_as(_dp), v.ctypes.data_as(_dp),
                   g.ctypes.data_as(_dp), t, lr, b1, b2, eps, wd)
