"""insp_simulate_noalloc, the entry point for callers that cannot allocate
device memory (for example code inside a framework whose allocator owns the
whole GPU, or a latency-critical loop that cannot absorb cudaMalloc's implicit
synchronisation).  It must give exactly the schedule of the regular entry
points while using only the library's fixed scratch array.

Checked through the C ABI: two calls in a row on DAGs of different sizes (the
second call runs over the scratch the first one left behind) against
insp_dag_load_csr + insp_attributes + insp_simulate; exact equality, the
tolerance of every parity test here.  This file is named to run last.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def _device_inputs(dag):
    import torch
    dev = torch.device("cuda")
    return dict(
        row_ptr=torch.from_numpy(np.ascontiguousarray(dag.row_ptr, np.int32)).to(dev),
        col_idx=torch.from_numpy(np.ascontiguousarray(dag.col_idx, np.int32) if dag.col_idx.size
                                 else np.zeros(1, np.int32)).to(dev),
        type=torch.zeros(max(dag.n, 1), dtype=torch.uint8, device=dev),
        task_cost=torch.from_numpy(np.ascontiguousarray(np.stack([dag.c_cpu, dag.c_gpu], 1), np.int64)).to(dev),
    )


def _regular(dag, machine):
    """Schedule from the existing single-DAG entry points."""
    from paper_2404_03226_b300 import _lib
    import paper_2404_03226_b300 as P
    M = P.Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns)
    h = _lib.insp_dag_load_csr(M.handle, dag.n, dag.row_ptr, dag.col_idx, None, 1, None,
                               np.ascontiguousarray(np.stack([dag.c_cpu, dag.c_gpu], 1)))
    n = dag.n
    out = dict(ia=np.zeros(n, np.int32), ie=np.zeros(n, np.int32), worker=np.zeros(n, np.int32),
               start=np.zeros(n, np.int64), end=np.zeros(n, np.int64), makespan=np.zeros(1, np.int64))
    try:
        _lib.insp_attributes(h, 0, out["ia"], out["ie"])
        _lib.insp_simulate(h, out["ia"], out["ie"], out["worker"], out["start"], out["end"], out["makespan"])
    finally:
        _lib.insp_dag_destroy(h)
    return out


def _noalloc(dag, machine, ia, ie):
    import torch
    from paper_2404_03226_b300 import _lib
    dev = torch.device("cuda")
    x = _device_inputs(dag)
    n = dag.n
    d_ia = torch.from_numpy(ia).to(dev)
    d_ie = torch.from_numpy(ie).to(dev)
    worker = torch.full((n,), -7, dtype=torch.int32, device=dev)
    start = torch.full((n,), -7, dtype=torch.int64, device=dev)
    end = torch.full((n,), -7, dtype=torch.int64, device=dev)
    mk = torch.full((1,), -7, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    _lib.insp_simulate_noalloc(n, x["row_ptr"], x["col_idx"], x["type"], 1, None, x["task_cost"], machine.n_cpu,
                               machine.n_gpu, machine.xfer_ns, None, d_ia, d_ie, worker, start, end, mk,
                               torch.cuda.current_stream())
    return dict(worker=worker.cpu().numpy(), start=start.cpu().numpy(), end=end.cpu().numpy(),
                makespan=mk.cpu().numpy())


def test_noalloc_matches_regular_entry_points_twice_in_a_row():
    big = inputs.layered(1, cfg=95, first=0, n_min=1800, n_max=1800).dag(0)   # wide pool, spills used
    small = inputs.cholesky8().dag(0)
    cases = [(big, inputs.MACHINE_LAYERED), (small, inputs.MACHINE_CHOLESKY8)]
    for dag, machine in cases:  # two calls in a row, the second over the first call's leftovers
        ref = _regular(dag, machine)
        got = _noalloc(dag, machine, ref["ia"], ref["ie"])
        for k in ("worker", "start", "end", "makespan"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_noalloc_rejects_oversized_dag_and_host_pointers():
    import torch
    from paper_2404_03226_b300 import _lib
    dev = torch.device("cuda")
    z32 = torch.zeros(4, dtype=torch.int32, device=dev)
    z64 = torch.ones(8, dtype=torch.int64, device=dev)
    z8 = torch.zeros(4, dtype=torch.uint8, device=dev)
    with pytest.raises(_lib.InspError) as e:
        _lib.insp_simulate_noalloc(_lib.INSP_NOALLOC_MAX_TASKS + 1, z32, z32, z8, 1, None, z64, 1, 1, 0, None,
                                   z32, z32, z32, z64, z64, z64)
    assert e.value.code == _lib.INSP_EINVAL and "scratch" in str(e.value)
    host = np.zeros(4, np.int32)
    with pytest.raises(_lib.InspError) as e:
        _lib.insp_simulate_noalloc(1, host, z32, z8, 1, None, z64, 1, 1, 0, None, z32, z32, z32, z64, z64, z64)
    assert e.value.code == _lib.INSP_EINVAL and "device pointer" in str(e.value)
