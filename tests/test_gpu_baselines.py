"""The DMDAP baselines and the push/pop trace on the GPU against the oracle:
bottom levels element by element, schedules of the static-priority policies
bit for bit, and every push and pop record of the trace."""
import numpy as np
import pytest

import inputs
import oracle
from helpers import compare_dag, edge_case_dags, gpu_run, machine_policy

pytestmark = pytest.mark.gpu

MACHINES = [inputs.MACHINE_LAYERED, inputs.Machine(1, 0, 0), inputs.Machine(3, 2, 7), inputs.Machine(60, 4, 1000)]


def _batch():
    return inputs.concat([inputs.layered(24, cfg=61, n_min=1, n_max=700), inputs.concat_dags(edge_case_dags())])


@pytest.mark.parametrize("m", MACHINES)
def test_bottom_level_matches_oracle(m):
    import torch
    import paper_2404_03226_b300 as P
    b = _batch()
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    bl = B.bottom_level()
    torch.cuda.synchronize()
    got = bl.cpu().numpy()
    for d in range(b.ndag):
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        np.testing.assert_array_equal(got[tb:te], oracle.bottom_level(b.dag(d), m), err_msg=f"DAG {d}")
    # host output array
    host = np.zeros(max(b.n_total, 1), np.int64)
    from paper_2404_03226_b300 import _lib
    _lib.insp_bottom_level_batch(B.handle, host)
    np.testing.assert_array_equal(host[:b.n_total], got)


@pytest.mark.parametrize("policy", ["dmdap_ia", "dmdap_bl"])
@pytest.mark.parametrize("m", MACHINES)
def test_dmdap_schedules_match_oracle(policy, m):
    b = _batch()
    g = gpu_run(b, m, policy)
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, m, policy)


@pytest.mark.parametrize("policy", ["dmdap_ia", "dmdap_bl"])
def test_dmdap_tiled_and_pipelined(policy):
    """Per-task costs (tiled Cholesky) and the pipelined evaluation step."""
    import torch
    import paper_2404_03226_b300 as P
    b = inputs.concat([inputs.tiled(inputs.KIND_CHOLESKY, 8, 3), inputs.tiled(inputs.KIND_QR, 6, 2)])
    m = inputs.MACHINE_TILED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns, machine_policy(policy)), b)
    B.tuning = dict(groups=3, attr_overlap=1, ia_warps=8, ie_warps=4, ie_ring_mb=64, sim_warps=2, sim_queue=32)
    ia, ie, s = B.evaluate()
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    out = dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(), start=s.start.cpu().numpy(),
               end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())
    for d in range(b.ndag):
        compare_dag(b, d, out, m, policy)
    per = gpu_run(b, m, policy, per_dag=True)
    np.testing.assert_array_equal(per["start"], out["start"])


@pytest.mark.parametrize("policy", ["inspirit", "fifo", "dmdap_ia", "dmdap_bl"])
def test_trace_matches_oracle(policy):
    import torch
    import paper_2404_03226_b300 as P
    b = _batch()
    m = inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns, machine_policy(policy)), b)
    ia, ie = B.attributes()
    s, tr = B.simulate_trace(ia, ie)
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    tr = {k: v.cpu().numpy() for k, v in tr.items()}
    pol = oracle.Policy({"inspirit": 0, "fifo": 1, "dmdap_ia": 3, "dmdap_bl": 4}[policy])
    for d in range(b.ndag):
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        r = oracle.simulate(b.dag(d), m, pol, trace=True)["trace"]
        for mine, ref in (("push_time", "push_t"), ("push_task", "push_task"), ("push_worker", "push_worker"),
                          ("push_nready", "push_nready"), ("pop_time", "t"), ("pop_task", "task"),
                          ("pop_worker", "worker"), ("pop_nready", "nready"), ("pop_mode", "mode")):
            np.testing.assert_array_equal(tr[mine][tb:te], r[ref], err_msg=f"{mine} of DAG {d}")
    # the schedule is the untraced one
    plain = B.simulate(ia, ie)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(plain.start.cpu().numpy(), s.start.cpu().numpy())
