"""Launch shapes of the batched kernels (the library's autotuner, no
counterpart in the paper): every tuning gives the oracle's results bit for
bit, the autotuner returns a valid tuning, and out-of-range fields are
rejected."""
import numpy as np
import pytest

import inputs
from helpers import compare_dag, edge_case_dags

pytestmark = pytest.mark.gpu

TUNINGS = [
    dict(ia_bin_tasks=0, ia_warps_small=8, ia_warps_large=8, ie_warps=4, ie_ring_mb=64, sim_warps=8, sim_queue=64),
    dict(ia_bin_tasks=300, ia_warps_small=2, ia_warps_large=32, ie_warps=1, ie_ring_mb=1, sim_warps=1, sim_queue=32),
    dict(ia_bin_tasks=0, ia_warps_small=32, ia_warps_large=32, ie_warps=16, ie_ring_mb=2048, sim_warps=8,
         sim_queue=128),
    dict(ia_bin_tasks=100000, ia_warps_small=5, ia_warps_large=3, ie_warps=8, ie_ring_mb=256, sim_warps=3,
         sim_queue=128),
    dict(ia_bin_tasks=1, ia_warps_small=1, ia_warps_large=7, ie_warps=2, ie_ring_mb=8, sim_warps=5, sim_queue=32),
]


def _batch():
    return inputs.concat([inputs.layered(40, cfg=41, n_min=1, n_max=900), inputs.concat_dags(edge_case_dags())])


def _run(B):
    import torch
    ia, ie = B.attributes()
    s = B.simulate(ia, ie)
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    return dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(), start=s.start.cpu().numpy(),
                end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())


@pytest.mark.parametrize("k", range(len(TUNINGS)))
def test_every_tuning_matches_oracle(k):
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    B = P.DagBatch(M, b)
    B.tuning = TUNINGS[k]
    assert B.tuning == TUNINGS[k]
    out = _run(B)
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
    assert t["sim_queue"] in (32, 64, 128) and 1 <= t["sim_warps"] <= 8 and 1 <= t["ie_warps"] <= 8
    r1 = _run(B)
    for f in r0:
        np.testing.assert_array_equal(r0[f], r1[f], err_msg=f)


def test_tuning_rejects_out_of_range():
    import paper_2404_03226_b300 as P
    b, m = _batch(), inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    good = B.tuning
    for field, bad in (("ia_warps_small", 0), ("ia_warps_large", 33), ("ie_warps", 17), ("ie_ring_mb", 0),
                       ("sim_warps", 0), ("sim_queue", 48), ("ia_bin_tasks", -1)):
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
