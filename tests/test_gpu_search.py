"""The unit-time search on the GPU against the oracle, DAG by DAG: random
layered DAGs (random and degree types), edge cases, tiled DAGs with per-task
costs, a cap on k, and candidates wide enough to take the global efficiency
sweep."""
import numpy as np
import pytest

import inputs
import oracle
from helpers import edge_case_dags

pytestmark = pytest.mark.gpu


def _search(batch, k_max, machine=inputs.MACHINE_LAYERED):
    import torch
    import paper_2404_03226_b300 as P
    B = P.DagBatch(P.Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns), batch)
    ut = B.unit_time_search(k_max)
    torch.cuda.synchronize()
    return B, ut.cpu().numpy()


@pytest.mark.parametrize("typing", ["random", "degree"])
def test_search_layered(typing):
    b = inputs.layered(30, cfg=71, n_min=1, n_max=500, typing=typing)
    _, got = _search(b, 16)
    for d in range(b.ndag):
        assert got[d] == oracle.unit_time_search(b.dag(d), 16)[0], f"DAG {d}"


@pytest.mark.parametrize("k_max", [0, 2, 5, 20])
def test_search_edge_cases_and_caps(k_max):
    dags = edge_case_dags() + [inputs.make_dag(0, [], [], []),
                               inputs.make_dag(40, [(i, i + 1) for i in range(39)], [9] * 40, [3] * 40)]
    b = inputs.concat_dags(dags)
    _, got = _search(b, k_max)
    for d in range(b.ndag):
        assert got[d] == oracle.unit_time_search(b.dag(d), k_max)[0], f"DAG {d}"


def test_search_tiled_per_task_costs():
    b = inputs.concat([inputs.tiled(inputs.KIND_CHOLESKY, 8, 2), inputs.tiled(inputs.KIND_LU, 5, 2)])
    _, got = _search(b, 12, inputs.MACHINE_TILED)
    for d in range(b.ndag):
        assert got[d] == oracle.unit_time_search(b.dag(d), 12)[0], f"DAG {d}"


def test_search_wide_candidates_and_use():
    """GPU costs near 2^24 ns: candidates pass 2^31 and the global sweep takes over;
    the searched T then feeds the attributes."""
    import torch
    rng = np.random.default_rng(3)
    dags = [inputs.make_dag(300, [(i, i + 1) for i in range(299)], [1 << 25] * 300, [1 << 24] * 300),
            inputs.make_dag(50, [(u, v) for u in range(50) for v in range(u + 1, min(50, u + 4))],
                            rng.integers(1 << 22, 1 << 23, 50), rng.integers(1 << 22, 1 << 24, 50))]
    b = inputs.concat_dags(dags)
    B, got = _search(b, 16)
    want = [oracle.unit_time_search(b.dag(d), 16)[0] for d in range(b.ndag)]
    np.testing.assert_array_equal(got, want)
    assert got[0] == (1 << 24) << 9  # chain of 300: 2^9 >= 300
    ia, ie = B.attributes(got)
    torch.cuda.synchronize()
    ie = ie.cpu().numpy()
    for d in range(b.ndag):
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        np.testing.assert_array_equal(ie[tb:te], oracle.ie(b.dag(d), int(got[d])))
