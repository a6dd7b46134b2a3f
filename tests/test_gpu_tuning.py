"""Launch shapes and pipelining of the batched kernels (the library's
autotuner, no counterpart in the paper): under every tuning both the two-call
step and the pipelined evaluation step give the oracle's results bit for bit,
the autotuner returns a valid tuning, and out-of-range fields are rejected."""
import numpy as np
import pytest

import inputs
from helpers import compare_dag, edge_case_dags

pytestmark = pytest.mark.gpu

TUNINGS = [
    dict(groups=1, attr_overlap=0, ia_warps=8, ie_warps=4, ie_ring_mb=64, sim_warps=8, sim_queue=64, group_split=0,
         ia_block=0),
    dict(groups=3, attr_overlap=1, ia_warps=32, ie_warps=1, ie_ring_mb=1, sim_warps=1, sim_queue=32, group_split=0,
         ia_block=1),
    dict(groups=16, attr_overlap=0, ia_warps=32, ie_warps=16, ie_ring_mb=2048, sim_warps=8, sim_queue=128,
         group_split=0, ia_block=0),
    dict(groups=4, attr_overlap=1, ia_warps=3, ie_warps=8, ie_ring_mb=256, sim_warps=3, sim_queue=128, group_split=1,
         ia_block=1),
    dict(groups=1, attr_overlap=1, ia_warps=1, ie_warps=2, ie_ring_mb=8, sim_warps=5, sim_queue=32, group_split=0,
         ia_block=1),
    dict(groups=3, attr_overlap=0, ia_warps=16, ie_warps=16, ie_ring_mb=512, sim_warps=4, sim_queue=64, group_split=1,
         ia_block=0),
    dict(groups=2, attr_overlap=1, ia_warps=16, ie_warps=8, ie_ring_mb=256, sim_warps=8, sim_queue=512, group_split=0,
         ia_block=1),
    dict(groups=1, attr_overlap=0, ia_warps=8, ie_warps=4, ie_ring_mb=128, sim_warps=3, sim_queue=256, group_split=0,
         ia_block=0),
    dict(groups=2, attr_overlap=0, ia_warps=8, ie_warps=4, ie_ring_mb=128, sim_warps=5, sim_queue=1024, group_split=0,
         ia_block=1),
    dict(groups=3, attr_overlap=1, ia_warps=16, ie_warps=4, ie_ring_mb=512, sim_warps=2, sim_queue=32, group_split=2,
         ia_block=0),
    dict(groups=2, attr_overlap=0, ia_warps=8, ie_warps=8, ie_ring_mb=256, sim_warps=4, sim_queue=64, group_split=2,
         ia_block=1),
]


def _batch():
    return inputs.concat([inputs.layered(40, cfg=41, n_min=1, n_max=900), inputs.concat_dags(edge_case_dags())])


def _run(B, fused=False, unit_time=None):
    import torch
    if fused:
        ia, ie, s = B.evaluate(unit_time)
    else:
        ia, ie = B.attributes(unit_time)
        s = B.simulate(ia, ie)
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    return dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(), start=s.start.cpu().numpy(),
                end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())


@pytest.mark.parametrize("k", range(len(TUNINGS)))
@pytest.mark.parametrize("fused", [False, True])
def test_every_tuning_matches_oracle(k, fused):
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    B = P.DagBatch(M, b)
    B.tuning = TUNINGS[k]
    assert B.tuning == TUNINGS[k]
    out = _run(B, fused)
    for d in range(b.ndag):
        compare_dag(b, d, out, m)


@pytest.mark.parametrize("wide", [False, True])
def test_pipelined_step_with_unit_times(wide):
    """Caller unit times: narrow ones keep the pipelined pull sweep, wide ones
    (>= 2^31 ns) take the global sweep in one group."""
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    rng = np.random.default_rng(8)
    ut = rng.integers(1, 3_000_000, b.ndag).astype(np.int64)
    ut[::7] = 0  # defaults
    if wide:
        ut[1] = (1 << 31) + 5
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.tuning = TUNINGS[3]
    out = _run(B, True, ut)
    ref = _run(B, False, ut)
    for f in out:
        np.testing.assert_array_equal(out[f], ref[f], err_msg=f)
    for d in range(0, b.ndag, 3):
        compare_dag(b, d, out, m, unit_time=int(ut[d]) if ut[d] > 0 else None)


def test_pipelined_step_more_groups_than_dags():
    import paper_2404_03226_b300 as P
    b, m = inputs.concat_dags(edge_case_dags()[:3]), inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.tuning = TUNINGS[2]
    out = _run(B, True)
    for d in range(b.ndag):
        compare_dag(b, d, out, m)


def test_autotune_keeps_results():
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    B = P.DagBatch(M, b)
    r0 = _run(B)
    t = B.autotune()
    assert t == B.tuning
    assert t["sim_queue"] in (32, 64, 128, 256, 512, 1024) and 1 <= t["sim_warps"] <= 8 and 1 <= t["ie_warps"] <= 8
    r1 = _run(B)
    for f in r0:
        np.testing.assert_array_equal(r0[f], r1[f], err_msg=f)


def test_tuning_rejects_out_of_range():
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    good = B.tuning
    for field, bad in (("groups", 0), ("groups", 17), ("attr_overlap", 2), ("ia_warps", 0), ("ia_warps", 33),
                       ("ie_warps", 17), ("ie_ring_mb", 0), ("sim_warps", 0), ("sim_queue", 48), ("group_split", 3),
                       ("ia_block", 2)):
        t = dict(good, **{field: bad})
        with pytest.raises(P.InspError):
            B.tuning = t
        assert B.tuning == good


def test_machine_tuning_applies_to_later_batches():
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    M.set_tuning(TUNINGS[2])
    B = P.DagBatch(M, b)
    assert B.tuning == TUNINGS[2]
    out = _run(B)
    for d in range(0, b.ndag, 5):
        compare_dag(b, d, out, m)
    with pytest.raises(P.InspError):
        M.set_tuning(dict(TUNINGS[0], sim_queue=7))


@pytest.mark.parametrize("queue", [32, 128, 512, 1024])
def test_large_ready_pools(queue):
    """Tiled DAGs hold hundreds of ready tasks at once: a 512- or 1024-entry pool keeps them
    in shared memory, a 32-entry one spills most of them, a 128-entry one keeps per-worker
    bitmaps of its shared part and spills the rest; all give the oracle's schedule."""
    import paper_2404_03226_b300 as P
    b = inputs.concat([inputs.tiled(inputs.KIND_CHOLESKY, 16, 2), inputs.tiled(inputs.KIND_QR, 12, 1)])
    m = inputs.MACHINE_TILED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.tuning = dict(TUNINGS[0], sim_queue=queue, sim_warps=2)
    out = _run(B, True)
    for d in range(b.ndag):
        compare_dag(b, d, out, m)


def test_simulation_cta_that_does_not_fit_is_an_error():
    """Eight warps of 1024-entry pools exceed a CTA's shared memory: the evaluation reports
    INSP_EINVAL instead of launching, and the batch stays usable."""
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.tuning = dict(TUNINGS[0], sim_warps=8, sim_queue=1024)
    with pytest.raises(P.InspError):
        _run(B, True)
    B.tuning = TUNINGS[0]
    out = _run(B, True)
    for d in range(0, b.ndag, 7):
        compare_dag(b, d, out, m)


@pytest.mark.parametrize("ia_block", [0, 1])
@pytest.mark.parametrize("groups", [1, 3])
def test_repeated_structures_share_ability(ia_block, groups):
    """Instances of one tiled structure with different per-task costs (inspiring ability depends
    on the structure alone, so it is computed once per structure and copied), mixed with unique
    DAGs, in both ability sweeps, one group or pipelined groups, two-call and fused steps."""
    import paper_2404_03226_b300 as P
    b = inputs.concat([inputs.tiled(inputs.KIND_CHOLESKY, 16, 5, cfg=42), inputs.layered(7, cfg=43, n_max=700),
                       inputs.tiled(inputs.KIND_LU, 8, 3, cfg=44), inputs.tiled(inputs.KIND_QR, 8, 1, cfg=45)])
    m = inputs.MACHINE_TILED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    from paper_2404_03226_b300 import _lib
    assert _lib.insp_batch_structures(B.handle) == 1 + 7 + 1 + 1  # Cholesky-16, 7 layered, LU-8, QR-8
    B.tuning = dict(TUNINGS[0], groups=groups, ia_block=ia_block)
    for fused in (False, True):
        out = _run(B, fused)
        for d in range(b.ndag):
            compare_dag(b, d, out, m)


@pytest.mark.parametrize("ia_block", [0, 1])
def test_ability_by_target_blocks_on_larger_dags(ia_block):
    """DAGs of one to three 8192-id target blocks (layered of 8,300 to 12,000 tasks, LU and QR at 32
    tiles; Cholesky at 48 tiles, 19,600 tasks, above the whole-row limit, so it takes the blocks
    in both modes)."""
    import paper_2404_03226_b300 as P
    b = inputs.concat([inputs.layered(2, cfg=46, n_min=8300, n_max=12000),
                       inputs.tiled(inputs.KIND_CHOLESKY, 48, 1, cfg=47), inputs.tiled(inputs.KIND_LU, 32, 1, cfg=47),
                       inputs.tiled(inputs.KIND_QR, 32, 1, cfg=47)])
    m = inputs.MACHINE_TILED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.tuning = dict(TUNINGS[0], ia_block=ia_block, ia_warps=32)
    out = _run(B)
    for d in range(b.ndag):
        compare_dag(b, d, out, m)


@pytest.mark.parametrize("machine", [inputs.Machine(32, 8, 20000), inputs.Machine(60, 4, 1000)])
@pytest.mark.parametrize("queue", [128, 1024])
def test_pool_bitmaps_with_two_workers_per_lane(machine, queue):
    """Machines of more than 32 workers (every lane owns two) with pools of 128+ shared-memory
    entries, where pops walk per-worker bitmaps: wide ready pools (a 300-way fan-out, wide
    layered DAGs, a Cholesky DAG) bit-exact against the oracle."""
    import paper_2404_03226_b300 as P
    b = inputs.concat([inputs.layered(6, cfg=51, n_min=400, n_max=1500, w_min=48, w_max=64),
                       inputs.concat_dags(edge_case_dags()), inputs.tiled(inputs.KIND_CHOLESKY, 12, 1, cfg=52)])
    B = P.DagBatch(P.Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns), b)
    B.tuning = dict(TUNINGS[0], sim_warps=2, sim_queue=queue)
    for fused in (False, True):
        out = _run(B, fused)
        for d in range(b.ndag):
            compare_dag(b, d, out, machine)
