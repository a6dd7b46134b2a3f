"""B300-native evaluation of INSPIRIT's adaptive-priority list scheduling
(arxiv 2404.03226).

The work runs in CUDA kernels for sm_103a behind the C ABI of
``include/inspirit.h`` (libinspirit.so, built in-tree).  ``_lib`` binds that
ABI one function per entry point; the classes below only hold handles and
torch output tensors.  There is no CPU fallback: without the CUDA library or a
GPU the calls raise.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (INSP_POLICY_DMDAP_BL, INSP_POLICY_DMDAP_IA, INSP_POLICY_FIFO,  # noqa: F401
                   INSP_POLICY_INSPIRIT, INSP_POLICY_LEARNED, InspError, insp_policy, insp_tuning)

__all__ = ["Machine", "DagBatch", "InspError", "insp_policy", "insp_tuning", "INSP_POLICY_INSPIRIT",
           "INSP_POLICY_FIFO", "INSP_POLICY_LEARNED", "INSP_POLICY_DMDAP_IA", "INSP_POLICY_DMDAP_BL"]


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Machine:
    """A modelled machine: n_cpu CPU workers, n_gpu GPU workers, a transfer
    cost between memory nodes, and the scheduling policy."""

    def __init__(self, n_cpu: int, n_gpu: int, xfer_ns: int, policy: insp_policy | None = None):
        self.n_cpu, self.n_gpu, self.xfer_ns = n_cpu, n_gpu, xfer_ns
        self.handle = _lib.insp_machine_create(n_cpu, n_gpu, xfer_ns, policy)

    def set_tuning(self, t: dict) -> None:
        """Launch shapes that batches loaded later on this machine start with."""
        _lib.insp_machine_set_tuning(self.handle, insp_tuning(**t))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.insp_machine_destroy(h)
            self.handle = None


@dataclass
class Schedule:
    worker: "object"
    start: "object"
    end: "object"
    makespan: "object"


class DagBatch:
    """DAGs resident in device memory.  `src` provides the batch arrays
    (task_base, edge_base, row_ptr, col_idx, type, n_types, type_cost,
    task_cost) as numpy arrays; see insp_batch_load_csr."""

    def __init__(self, machine: Machine, src):
        self.machine = machine
        self.ndag = int(src.ndag)
        tc = None if src.task_cost is None else _np(src.task_cost, np.int64)
        self.handle = _lib.insp_batch_load_csr(
            machine.handle, self.ndag, _np(src.task_base, np.int64), _np(src.edge_base, np.int64),
            _np(src.row_ptr, np.int32), _np(src.col_idx, np.int32), _np(src.type, np.uint8), int(src.n_types),
            _np(src.type_cost, np.int64), tc)
        self.ndag, self.n_tasks, self.n_edges = _lib.insp_batch_info(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.insp_batch_destroy(h)
            self.handle = None

    # torch tensors on the current CUDA device
    def _out(self, n, dtype):
        import torch
        return torch.empty(max(n, 1), dtype=dtype, device="cuda")[:n]

    def attributes(self, unit_time_ns=None, stream=None):
        """(ia, ie) int32 CUDA tensors; unit_time_ns: None, or int64 array per DAG."""
        import torch
        ia = self._out(self.n_tasks, torch.int32)
        ie = self._out(self.n_tasks, torch.int32)
        ut = None if unit_time_ns is None else _np(unit_time_ns, np.int64)
        _lib.insp_attributes_batch(self.handle, ut, ia, ie, stream or torch.cuda.current_stream())
        return ia, ie

    def simulate(self, ia, ie, stream=None, per_dag: bool = False) -> Schedule:
        import torch
        sch = Schedule(self._out(self.n_tasks, torch.int32), self._out(self.n_tasks, torch.int64),
                       self._out(self.n_tasks, torch.int64), self._out(self.ndag, torch.int64))
        f = _lib.insp_simulate_per_dag if per_dag else _lib.insp_simulate_batch
        f(self.handle, ia, ie, sch.worker, sch.start, sch.end, sch.makespan, stream or torch.cuda.current_stream())
        return sch

    def simulate_trace(self, ia, ie, stream=None):
        """Schedule plus the push/pop trace: (Schedule, dict of device tensors, the
        k-th push / pop of DAG d at task_base[d] + k)."""
        import torch
        sch = Schedule(self._out(self.n_tasks, torch.int32), self._out(self.n_tasks, torch.int64),
                       self._out(self.n_tasks, torch.int64), self._out(self.ndag, torch.int64))
        tr = {k: self._out(self.n_tasks, torch.int64 if k.endswith("_time") else torch.int32)
              for k in _lib.TRACE_FIELDS}
        _lib.insp_simulate_trace(self.handle, ia, ie, sch.worker, sch.start, sch.end, sch.makespan, tr,
                                 stream or torch.cuda.current_stream())
        return sch, tr

    def unit_time_search(self, k_max: int = 16, stream=None):
        """int64 CUDA tensor [ndag]: the searched unit time of every DAG."""
        import torch
        ut = self._out(self.ndag, torch.int64)
        _lib.insp_unit_time_search(self.handle, k_max, ut, stream or torch.cuda.current_stream())
        return ut

    def bottom_level(self, stream=None):
        """int64 CUDA tensor: each task's bottom level (static priority of INSP_POLICY_DMDAP_BL)."""
        import torch
        bl = self._out(self.n_tasks, torch.int64)
        _lib.insp_bottom_level_batch(self.handle, bl, stream or torch.cuda.current_stream())
        return bl

    def evaluate(self, unit_time_ns=None, stream=None):
        """Attributes and schedule in one pipelined call: (ia, ie, Schedule)."""
        import torch
        ia = self._out(self.n_tasks, torch.int32)
        ie = self._out(self.n_tasks, torch.int32)
        sch = Schedule(self._out(self.n_tasks, torch.int32), self._out(self.n_tasks, torch.int64),
                       self._out(self.n_tasks, torch.int64), self._out(self.ndag, torch.int64))
        ut = None if unit_time_ns is None else _np(unit_time_ns, np.int64)
        _lib.insp_evaluate_batch(self.handle, ut, ia, ie, sch.worker, sch.start, sch.end, sch.makespan,
                                 stream or torch.cuda.current_stream())
        return ia, ie, sch

    def autotune(self, stream=None) -> dict:
        """Time the library's candidate launch shapes on this batch and keep the
        fastest per kernel; returns the chosen tuning as a dict."""
        import torch
        return _lib.insp_batch_autotune(self.handle, stream or torch.cuda.current_stream()).as_dict()

    @property
    def tuning(self) -> dict:
        return _lib.insp_batch_get_tuning(self.handle).as_dict()

    @tuning.setter
    def tuning(self, t: dict) -> None:
        _lib.insp_batch_set_tuning(self.handle, insp_tuning(**t))

    def status(self) -> np.ndarray:
        st = np.zeros(max(self.ndag, 1), np.int32)
        _lib.insp_batch_status(self.handle, st)
        return st[:self.ndag]
