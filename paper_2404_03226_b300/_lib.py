"""ctypes binding of libinspirit.so: the C ABI of include/inspirit.h, one Python
function per C entry point with the same name.  Arguments are marshalled
(numpy arrays and torch tensors become raw pointers); nothing is computed here.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

INSP_OK, INSP_EINVAL, INSP_ENOTTOPO, INSP_ENOMEM, INSP_ECUDA, INSP_ETIMEOUT, INSP_EOVERFLOW = range(7)
INSP_ECHECK, INSP_ECYCLE = 7, 8
INSP_SCORE_TIMEOUT = -(1 << 63)  # insp_scorer_eval's score of a row whose tile did not complete (INT64_MIN)
INSP_POLICY_INSPIRIT, INSP_POLICY_FIFO, INSP_POLICY_LEARNED, INSP_POLICY_DMDAP_IA, INSP_POLICY_DMDAP_BL = 0, 1, 2, 3, 4
ERROR_NAMES = {0: "INSP_OK", 1: "INSP_EINVAL", 2: "INSP_ENOTTOPO", 3: "INSP_ENOMEM", 4: "INSP_ECUDA",
               5: "INSP_ETIMEOUT", 6: "INSP_EOVERFLOW", 7: "INSP_ECHECK", 8: "INSP_ECYCLE"}

_vp = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64


class insp_policy(ctypes.Structure):
    _fields_ = [("policy", _i32), ("task_window", _i32), ("s_inc", _i32), ("s_dec", _i32), ("dec_step", _i32),
                ("c", _i32), ("k_inc_tasks", _i64), ("k_inc_ns", _i64)]


class insp_tuning(ctypes.Structure):
    _fields_ = [("groups", _i32), ("attr_overlap", _i32), ("ia_warps", _i32), ("ie_warps", _i32),
                ("ie_ring_mb", _i32), ("sim_warps", _i32), ("sim_queue", _i32), ("group_split", _i32),
                ("ia_block", _i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class insp_trace(ctypes.Structure):
    _fields_ = [("push_time", ctypes.c_void_p), ("push_task", ctypes.c_void_p), ("push_worker", ctypes.c_void_p),
                ("push_nready", ctypes.c_void_p), ("pop_time", ctypes.c_void_p), ("pop_task", ctypes.c_void_p),
                ("pop_worker", ctypes.c_void_p), ("pop_nready", ctypes.c_void_p), ("pop_mode", ctypes.c_void_p)]


class InspError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes)
_PROTOS = {
    "insp_last_error": (ctypes.c_char_p, []),
    "insp_machine_create": (ctypes.c_int, [_i32, _i32, _i64, ctypes.POINTER(insp_policy), ctypes.POINTER(_vp)]),
    "insp_machine_destroy": (None, [_vp]),
    "insp_set_scorer": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "insp_dag_load_csr": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _i32, _vp, _vp, ctypes.POINTER(_vp)]),
    "insp_batch_load_csr": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, ctypes.POINTER(_vp)]),
    "insp_batch_destroy": (None, [_vp]),
    "insp_dag_destroy": (None, [_vp]),
    "insp_attributes": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp]),
    "insp_attributes_batch": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "insp_simulate": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_simulate_batch": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_evaluate_batch": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_evaluate_batch_async": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_simulate_trace": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(insp_trace), _vp]),
    "insp_bottom_level_batch": (ctypes.c_int, [_vp, _vp, _vp]),
    "insp_unit_time_search": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp]),
    "insp_selftest_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]),
    "insp_simulate_per_dag": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_batch_status": (ctypes.c_int, [_vp, _vp]),
    "insp_batch_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "insp_batch_set_policy": (ctypes.c_int, [_vp, ctypes.POINTER(insp_policy)]),
    "insp_batch_structures": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "insp_batch_set_timing": (ctypes.c_int, [_vp, _i32]),
    "insp_batch_timing": (ctypes.c_int, [_vp, _vp, _vp, _i32]),
    "insp_scorer_eval": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "insp_simulate_rollout": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp,
                                             _vp, _vp]),
    "insp_scorer_train_grad": (ctypes.c_int, [_i32, _i32, _i32, _vp, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_scorer_train_grad_tc": (ctypes.c_int, [_i32, _i32, _i32, _vp, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_adamw": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float, _vp]),
    "insp_scorer_quantize": (ctypes.c_int, [_i64, _vp, _vp, _vp]),
    "insp_batch_record": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "insp_batch_replay": (ctypes.c_int, [_vp, _vp]),
    "insp_batch_autotune": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(insp_tuning)]),
    "insp_batch_set_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(insp_tuning)]),
    "insp_batch_get_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(insp_tuning)]),
    "insp_machine_set_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(insp_tuning)]),
    "insp_simulate_noalloc": (ctypes.c_int, [_i32, _vp, _vp, _vp, _i32, _vp, _vp, _i32, _i32, _i64,
                                             ctypes.POINTER(insp_policy), _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}


def so_path() -> str:
    return _build.SO


def lib():
    """Load libinspirit.so (compiling it first if the sources are newer).
    Raises if the CUDA library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libinspirit.so missing at {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def symbols() -> list[str]:
    return list(_PROTOS)


def last_error() -> str:
    return lib().insp_last_error().decode()


def check(rc: int) -> None:
    if rc != INSP_OK:
        raise InspError(rc, last_error())


def ptr(x):
    """Raw pointer of a numpy array, torch tensor or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------ same-name wrappers
def insp_machine_create(n_cpu: int, n_gpu: int, xfer_ns: int, policy: insp_policy | None = None):
    h = _vp()
    check(lib().insp_machine_create(n_cpu, n_gpu, xfer_ns, None if policy is None else ctypes.byref(policy),
                                    ctypes.byref(h)))
    return h


def insp_machine_destroy(m) -> None:
    lib().insp_machine_destroy(m)


def insp_set_scorer(m, bf16_weights) -> None:
    check(lib().insp_set_scorer(m, ptr(bf16_weights), bf16_weights.nbytes if hasattr(bf16_weights, "nbytes")
                                else bf16_weights.numel() * bf16_weights.element_size()))


def insp_dag_load_csr(m, n, row_ptr, col_idx, type, n_types, type_cost, task_cost):
    h = _vp()
    check(lib().insp_dag_load_csr(m, n, ptr(row_ptr), ptr(col_idx), ptr(type), n_types, ptr(type_cost),
                                  ptr(task_cost), ctypes.byref(h)))
    return h


def insp_batch_load_csr(m, ndag, task_base, edge_base, row_ptr, col_idx, type, n_types, type_cost, task_cost):
    h = _vp()
    check(lib().insp_batch_load_csr(m, ndag, ptr(task_base), ptr(edge_base), ptr(row_ptr), ptr(col_idx), ptr(type),
                                    n_types, ptr(type_cost), ptr(task_cost), ctypes.byref(h)))
    return h


def insp_batch_destroy(b) -> None:
    lib().insp_batch_destroy(b)


def insp_dag_destroy(d) -> None:
    lib().insp_dag_destroy(d)


def insp_attributes(d, unit_time_ns: int, ia, ie, stream=None) -> None:
    check(lib().insp_attributes(d, unit_time_ns, ptr(ia), ptr(ie), stream_ptr(stream)))


def insp_attributes_batch(b, unit_time_ns, ia, ie, stream=None) -> None:
    check(lib().insp_attributes_batch(b, ptr(unit_time_ns), ptr(ia), ptr(ie), stream_ptr(stream)))


def insp_simulate(d, ia, ie, worker, start, end, makespan, stream=None) -> None:
    check(lib().insp_simulate(d, ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end), ptr(makespan),
                              stream_ptr(stream)))


def insp_simulate_batch(b, ia, ie, worker, start, end, makespan, stream=None) -> None:
    check(lib().insp_simulate_batch(b, ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end), ptr(makespan),
                                    stream_ptr(stream)))


def insp_evaluate_batch(b, unit_time_ns, ia, ie, worker, start, end, makespan, stream=None) -> None:
    check(lib().insp_evaluate_batch(b, ptr(unit_time_ns), ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end),
                                    ptr(makespan), stream_ptr(stream)))


def insp_evaluate_batch_async(b, unit_time_ns, ia, ie, worker, start, end, makespan, stream=None) -> None:
    check(lib().insp_evaluate_batch_async(b, ptr(unit_time_ns), ptr(ia), ptr(ie), ptr(worker), ptr(start),
                                          ptr(end), ptr(makespan), stream_ptr(stream)))


def insp_simulate_per_dag(b, ia, ie, worker, start, end, makespan, stream=None) -> None:
    check(lib().insp_simulate_per_dag(b, ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end), ptr(makespan),
                                      stream_ptr(stream)))


def insp_batch_status(b, status=None) -> int:
    return int(lib().insp_batch_status(b, ptr(status)))


def insp_batch_info(b) -> tuple[int, int, int]:
    nd, nt, ne = _i32(), _i64(), _i64()
    check(lib().insp_batch_info(b, ctypes.byref(nd), ctypes.byref(nt), ctypes.byref(ne)))
    return nd.value, nt.value, ne.value


def insp_batch_structures(b) -> int:
    k = _i32()
    check(lib().insp_batch_structures(b, ctypes.byref(k)))
    return k.value


def insp_batch_set_policy(b, policy: insp_policy) -> None:
    check(lib().insp_batch_set_policy(b, ctypes.byref(policy)))


def insp_batch_set_timing(b, enable: bool) -> None:
    check(lib().insp_batch_set_timing(b, 1 if enable else 0))


def insp_batch_timing(b, reset: bool = False):
    """(ms[4], launches[4]) per kernel: inspiring ability, inspiring efficiency,
    batched simulation, per-DAG simulation."""
    import numpy as np
    ms = np.zeros(4, np.float64)
    n = np.zeros(4, np.int64)
    check(lib().insp_batch_timing(b, ptr(ms), ptr(n), 1 if reset else 0))
    return ms, n


INSP_NOALLOC_MAX_TASKS = 65536  # include/inspirit.h; a CPU test keeps the two equal

_NOALLOC_DTYPES = dict(row_ptr="int32", col_idx="int32", type="uint8", type_cost="int64", task_cost="int64",
                       ia="int32", ie="int32", worker="int32", start="int64", end="int64", makespan="int64")


def _check_noalloc_tensor(name, x):
    """A raw pointer is taken from each array, so its dtype, layout and device are checked here."""
    if x is None:
        return
    if not hasattr(x, "data_ptr"):
        return  # host arrays are rejected by the library itself (INSP_EINVAL)
    import torch
    want = getattr(torch, _NOALLOC_DTYPES[name])
    if x.dtype != want:
        raise TypeError(f"{name} must be {want}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if x.is_cuda and x.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {x.device}, not on the current device cuda:{torch.cuda.current_device()}")


def insp_simulate_noalloc(n, row_ptr, col_idx, type, n_types, type_cost, task_cost, n_cpu, n_gpu, xfer_ns,
                          policy, ia, ie, worker, start, end, makespan, stream=None) -> None:
    """The single-DAG simulation that allocates no device memory (all arrays
    must be device tensors the caller owns); see include/inspirit.h."""
    for name, x in (("row_ptr", row_ptr), ("col_idx", col_idx), ("type", type), ("type_cost", type_cost),
                    ("task_cost", task_cost), ("ia", ia), ("ie", ie), ("worker", worker), ("start", start),
                    ("end", end), ("makespan", makespan)):
        _check_noalloc_tensor(name, x)
    check(lib().insp_simulate_noalloc(n, ptr(row_ptr), ptr(col_idx), ptr(type), n_types, ptr(type_cost),
                                      ptr(task_cost), n_cpu, n_gpu, xfer_ns,
                                      None if policy is None else ctypes.byref(policy), ptr(ia), ptr(ie),
                                      ptr(worker), ptr(start), ptr(end), ptr(makespan), stream_ptr(stream)))


def _check_tensor(name, x, dtype: str, numel: int):
    """A raw pointer is taken from x: its dtype, layout, length and device are checked first."""
    if x is None or not hasattr(x, "data_ptr"):
        return  # the library rejects NULL and host pointers itself (INSP_EINVAL)
    import torch
    if x.dtype != getattr(torch, dtype):
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if x.numel() < numel:
        raise ValueError(f"{name} holds {x.numel()} elements, {numel} needed")
    if x.is_cuda and x.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {x.device}, not on the current device cuda:{torch.cuda.current_device()}")


def insp_scorer_eval(m, feat, n, score, stream=None) -> None:
    _check_tensor("feat", feat, "int32", 16 * n)
    _check_tensor("score", score, "int64", n)
    check(lib().insp_scorer_eval(m, ptr(feat), n, ptr(score), stream_ptr(stream)))


def insp_simulate_rollout(b, ia, ie, worker, start, end, makespan, force_pop=None, force_task=None, feat_pop=None,
                          feat_cap=0, feat_task=None, feat=None, feat_n=None, stream=None) -> None:
    check(lib().insp_simulate_rollout(b, ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end), ptr(makespan),
                                      ptr(force_pop), ptr(force_task), ptr(feat_pop), feat_cap, ptr(feat_task),
                                      ptr(feat), ptr(feat_n), stream_ptr(stream)))


def insp_scorer_train_grad(inp, h1, h2, w, mode, n, x, target, work, grad, loss, stream=None) -> None:
    check(lib().insp_scorer_train_grad(inp, h1, h2, ptr(w), mode, n, ptr(x), ptr(target), ptr(work), ptr(grad),
                                       ptr(loss), stream_ptr(stream)))


def insp_scorer_train_grad_tc(inp, h1, h2, w, mode, n, x, target, part, grad, loss, stream=None) -> None:
    check(lib().insp_scorer_train_grad_tc(inp, h1, h2, ptr(w), mode, n, ptr(x), ptr(target), ptr(part), ptr(grad),
                                          ptr(loss), stream_ptr(stream)))


def insp_adamw(nw, w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0, stream=None) -> None:
    check(lib().insp_adamw(nw, ptr(w), ptr(m), ptr(v), ptr(g), t, lr, b1, b2, eps, wd, stream_ptr(stream)))


def insp_scorer_quantize(nw, w, out, stream=None) -> None:
    check(lib().insp_scorer_quantize(nw, ptr(w), ptr(out), stream_ptr(stream)))


def insp_batch_record(b, ia, ie, worker, start, end, makespan, stream) -> None:
    check(lib().insp_batch_record(b, ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end), ptr(makespan),
                                  stream_ptr(stream)))


def insp_batch_replay(b, stream) -> None:
    check(lib().insp_batch_replay(b, stream_ptr(stream)))


def insp_batch_autotune(b, stream=None) -> insp_tuning:
    t = insp_tuning()
    check(lib().insp_batch_autotune(b, stream_ptr(stream), ctypes.byref(t)))
    return t


def insp_batch_set_tuning(b, t: insp_tuning) -> None:
    check(lib().insp_batch_set_tuning(b, ctypes.byref(t)))


def insp_batch_get_tuning(b) -> insp_tuning:
    t = insp_tuning()
    check(lib().insp_batch_get_tuning(b, ctypes.byref(t)))
    return t


def insp_machine_set_tuning(m, t: insp_tuning) -> None:
    check(lib().insp_machine_set_tuning(m, ctypes.byref(t)))


TRACE_FIELDS = ("push_time", "push_task", "push_worker", "push_nready", "pop_time", "pop_task", "pop_worker",
                "pop_nready", "pop_mode")


def insp_simulate_trace(b, ia, ie, worker, start, end, makespan, trace: dict, stream=None) -> None:
    """trace: dict of the TRACE_FIELDS names to device tensors."""
    t = insp_trace(*[ptr(trace[k]) for k in TRACE_FIELDS])
    check(lib().insp_simulate_trace(b, ptr(ia), ptr(ie), ptr(worker), ptr(start), ptr(end), ptr(makespan),
                                    ctypes.byref(t), stream_ptr(stream)))


def insp_bottom_level_batch(b, bl, stream=None) -> None:
    check(lib().insp_bottom_level_batch(b, ptr(bl), stream_ptr(stream)))


def insp_unit_time_search(b, k_max: int, unit_time_ns, stream=None) -> None:
    check(lib().insp_unit_time_search(b, int(k_max), ptr(unit_time_ns), stream_ptr(stream)))


def insp_selftest_wait(flag_value: int, wait_value: int, limit: int, stream=None) -> None:
    check(lib().insp_selftest_wait(int(flag_value), int(wait_value), int(limit), stream_ptr(stream)))
