"""insp_simulate_noalloc, the entry point for callers that cannot allocate
device memory (for example code inside a framework whose allocator owns the
whole GPU, or a latency-critical loop that cannot absorb cudaMalloc's implicit
synchronisation).  It must give exactly the schedule of the regular entry
points while using only the library's fixed scratch array.

Checked through the C ABI: calls in a row on DAGs of different sizes (each
call runs over the scratch the previous one left behind) against
insp_dag_load_csr + insp_attributes + insp_simulate and against the oracle,
on per-task and per-type cost tables and on the three policies it accepts;
exact equality, the tolerance of every parity test here.  Validation errors
give the oracle's codes (a non-topological numbering is an error here, where
the regular load renumbers it), and the empty DAG works.  This file is named to
run last.
"""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

POLICIES = {"inspirit": (0, oracle.POLICY_INSPIRIT), "fifo": (1, oracle.POLICY_FIFO),
            "dmdap_ia": (3, oracle.POLICY_DMDAP_IA)}


def _costs(dag, type_table):
    """(n_types, type_cost, task_cost, type) in the layout the C ABI takes; with per-task costs
    there is one type and every task has type 0."""
    if type_table is None:
        return (1, None, np.ascontiguousarray(np.stack([dag.c_cpu, dag.c_gpu], 1), np.int64),
                np.zeros(max(dag.n, 1), np.uint8))
    tt = np.ascontiguousarray(type_table, np.int64)
    return tt.shape[0], tt, None, np.ascontiguousarray(dag.type if dag.n else np.zeros(1), np.uint8)


def _dev(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype)).to(torch.device("cuda"))


def _policy(name):
    from paper_2404_03226_b300 import _lib
    p = _lib.insp_policy()
    p.policy = POLICIES[name][0]
    return p


def _regular(dag, machine, type_table, policy):
    """Schedule from the existing single-DAG entry points (host arrays)."""
    from paper_2404_03226_b300 import _lib
    nt, tc, kc, ty = _costs(dag, type_table)
    M = _lib.insp_machine_create(machine.n_cpu, machine.n_gpu, machine.xfer_ns, _policy(policy))
    n = dag.n
    out = dict(ia=np.zeros(max(n, 1), np.int32), ie=np.zeros(max(n, 1), np.int32),
               worker=np.zeros(max(n, 1), np.int32), start=np.zeros(max(n, 1), np.int64),
               end=np.zeros(max(n, 1), np.int64), makespan=np.zeros(1, np.int64))
    try:
        h = _lib.insp_dag_load_csr(M, n, np.ascontiguousarray(dag.row_ptr, np.int32),
                                   np.ascontiguousarray(dag.col_idx, np.int32) if dag.col_idx.size
                                   else np.zeros(1, np.int32), ty, nt, tc, kc)
        try:
            _lib.insp_attributes(h, 0, out["ia"], out["ie"])
            _lib.insp_simulate(h, out["ia"], out["ie"], out["worker"], out["start"], out["end"], out["makespan"])
        finally:
            _lib.insp_dag_destroy(h)
    finally:
        _lib.insp_machine_destroy(M)
    return {k: v[:n] if k != "makespan" else v for k, v in out.items()}


def _noalloc(dag, machine, ia, ie, type_table=None, policy="inspirit"):
    import torch
    from paper_2404_03226_b300 import _lib
    n = dag.n
    nt, tc, kc, ty = _costs(dag, type_table)
    row_ptr = _dev(dag.row_ptr, np.int32)
    col_idx = _dev(dag.col_idx if dag.col_idx.size else np.zeros(1), np.int32)
    typ = _dev(ty, np.uint8)
    d_tc = None if tc is None else _dev(tc, np.int64)
    d_kc = None if kc is None else _dev(kc if n else np.ones((1, 2)), np.int64)
    d_ia = _dev(ia if n else np.zeros(1), np.int32)
    d_ie = _dev(ie if n else np.zeros(1), np.int32)
    worker = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    start = torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda")
    end = torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda")
    mk = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    _lib.insp_simulate_noalloc(n, row_ptr, col_idx, typ, nt, d_tc, d_kc, machine.n_cpu, machine.n_gpu,
                               machine.xfer_ns, _policy(policy), d_ia, d_ie, worker, start, end, mk,
                               torch.cuda.current_stream())
    return dict(worker=worker.cpu().numpy()[:n], start=start.cpu().numpy()[:n], end=end.cpu().numpy()[:n],
                makespan=mk.cpu().numpy())


def _oracle(dag, machine, policy):
    r = oracle.simulate(dag, machine, oracle.Policy(POLICIES[policy][1]))
    assert r["rc"] == 0
    return r


def _assert_same(got, ref, what):
    for k in ("worker", "start", "end"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{k} of {what}")
    assert int(got["makespan"][0]) == int(np.asarray(ref["makespan"]).reshape(-1)[0]), f"makespan of {what}"


def test_noalloc_matches_regular_entry_points_twice_in_a_row():
    big = inputs.layered(1, cfg=95, first=0, n_min=1800, n_max=1800).dag(0)   # wide pool, spills used
    small = inputs.cholesky8().dag(0)
    cases = [(big, inputs.MACHINE_LAYERED), (small, inputs.MACHINE_CHOLESKY8)]
    for dag, machine in cases:  # two calls in a row, the second over the first call's leftovers
        ref = _regular(dag, machine, None, "inspirit")
        got = _noalloc(dag, machine, ref["ia"], ref["ie"])
        _assert_same(got, ref, f"{dag.n}-task DAG")


def test_noalloc_type_costs_and_policies_match_the_oracle():
    """Per-type cost tables (the kernel stages them in shared memory) with 8 and 4 types, and the
    INSPIRIT, DMDA (FIFO) and DMDAP-by-ability policies, each against the oracle and the regular
    path; consecutive calls alternate between a large and a small DAG."""
    lay = inputs.layered(1, cfg=95, first=3, n_min=1500, n_max=1500)
    chol = inputs.cholesky8()
    cases = [(lay.dag(0), lay.type_cost[0], inputs.MACHINE_LAYERED),
             (chol.dag(0), chol.type_cost[0], inputs.MACHINE_CHOLESKY8)]
    for policy in POLICIES:
        for dag, table, machine in cases:
            assert table.shape[0] > 1
            ref = _oracle(dag, machine, policy)
            got = _noalloc(dag, machine, ref["ia"], ref["ie"], table, policy)
            _assert_same(got, ref, f"{dag.n}-task DAG, {policy}, oracle")
            reg = _regular(dag, machine, table, policy)
            _assert_same(got, reg, f"{dag.n}-task DAG, {policy}, regular path")


def test_noalloc_validation_and_empty_dag_as_the_regular_load():
    from paper_2404_03226_b300 import _lib
    m = inputs.MACHINE_CHOLESKY8
    bad = [
        inputs.Dag(3, np.array([0, 1, 1, 1], np.int32), np.array([0], np.int32), np.zeros(3, np.uint8),
                   np.ones(3, np.int64), np.ones(3, np.int64)),                     # self edge: not topological
        inputs.Dag(3, np.array([0, 0, 1, 1], np.int32), np.array([0], np.int32), np.zeros(3, np.uint8),
                   np.ones(3, np.int64), np.ones(3, np.int64)),                     # edge 1 -> 0
        inputs.Dag(3, np.array([0, 2, 2, 2], np.int32), np.array([2, 1], np.int32), np.zeros(3, np.uint8),
                   np.ones(3, np.int64), np.ones(3, np.int64)),                     # unsorted successors
        inputs.Dag(2, np.array([0, 1, 1], np.int32), np.array([1], np.int32), np.zeros(2, np.uint8),
                   np.array([0, 1], np.int64), np.ones(2, np.int64)),               # cost < 1
    ]
    # the regular load renumbers a non-topological DAG (or reports its cycle); this entry point,
    # which has no room for a renumbered copy, rejects it as the oracle's check does
    regular = [_lib.INSP_ECYCLE, None, _lib.INSP_EINVAL, _lib.INSP_EINVAL]
    for dag, want in zip(bad, regular):
        with pytest.raises(_lib.InspError) as got:
            _noalloc(dag, m, np.zeros(dag.n, np.int32), np.zeros(dag.n, np.int32))
        assert got.value.code == oracle.check_dag(dag, m.xfer_ns) != _lib.INSP_OK
        if want is None:
            _regular(dag, m, None, "inspirit")  # renumbered and evaluated
        else:
            with pytest.raises(_lib.InspError) as reg:
                _regular(dag, m, None, "inspirit")
            assert reg.value.code == want
    empty = inputs.Dag(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint8),
                       np.zeros(0, np.int64), np.zeros(0, np.int64))
    got = _noalloc(empty, m, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert int(got["makespan"][0]) == 0
    # a valid DAG right after the errors and the empty DAG
    dag = inputs.cholesky8().dag(0)
    ref = _oracle(dag, m, "inspirit")
    _assert_same(_noalloc(dag, m, ref["ia"], ref["ie"]), ref, "Cholesky 8x8 after the error cases")


def test_noalloc_rejects_oversized_dag_short_arrays_and_host_pointers():
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
    # an output array that ends inside the allocation's last bytes: the call must refuse it
    # before any kernel runs (the library bounds every array by its allocation's extent)
    from cuda.bindings import driver
    buf = torch.zeros(1 << 21, dtype=torch.uint8, device=dev)
    err, base, size = driver.cuMemGetAddressRange(buf.data_ptr())
    assert err == driver.CUresult.CUDA_SUCCESS
    tail = int(base) + int(size) - 8          # 8 bytes before the end of the allocation
    n = 4                                     # start needs 32 bytes
    dag_rp = torch.tensor([0, 0, 0, 0, 0], dtype=torch.int32, device=dev)
    with pytest.raises(_lib.InspError) as e:
        _lib.insp_simulate_noalloc(n, dag_rp, z32, z8, 1, None, z64, 1, 1, 0, None, z32, z32, z32, tail, z64, z64)
    assert e.value.code == _lib.INSP_EINVAL and "shorter" in str(e.value)
    with pytest.raises(TypeError):
        _lib.insp_simulate_noalloc(n, dag_rp.to(torch.int64), z32, z8, 1, None, z64, 1, 1, 0, None, z32, z32, z32,
                                   z64, z64, z64)
    torch.cuda.synchronize()
