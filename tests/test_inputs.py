"""The seeded workload generators: sizes, determinism and CSR invariants."""
import numpy as np
import pytest

import inputs


def _check_csr(b):
    for d in range(b.ndag):
        g = b.dag(d)
        assert g.row_ptr[0] == 0 and np.all(np.diff(g.row_ptr) >= 0)
        for u in range(g.n):
            row = g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]
            assert np.all(row > u) and np.all(np.diff(row) > 0)
        assert g.c_cpu.min() >= 1 and g.c_gpu.min() >= 1


@pytest.mark.parametrize("kind,N,n,m", [(0, 8, 120, 252), (0, 16, 816, 2040), (0, 32, 5984, 16368),
                                        (1, 16, 1496, 3960), (1, 32, 11440, 32240),
                                        (2, 16, 1496, 4080), (2, 32, 11440, 32736)])
def test_tiled_sizes(kind, N, n, m):
    b = inputs.tiled(kind, N, 1, perturb=False)
    assert (b.n_total, b.m_total) == (n, m) == (inputs.tiled_count(kind, N), m)
    _check_csr(b)


def test_tiled_perturbation_range():
    b = inputs.tiled(inputs.KIND_CHOLESKY, 16, 2)
    base = inputs.CHOLESKY_COST[b.type.astype(int)]
    ratio = b.task_cost / base
    assert ratio.min() >= 0.8 and ratio.max() <= 1.2
    assert not np.array_equal(b.task_cost[:816], b.task_cost[816:])  # instances differ


def test_layered_shape_and_determinism():
    b = inputs.layered(64)
    sizes = b.sizes()
    assert sizes.min() >= 50 and sizes.max() <= 2000
    assert 10 < b.m_total / b.n_total < 30
    _check_csr(b)
    b2 = inputs.layered(8, first=3)
    for i in range(8):
        assert np.array_equal(b.dag(3 + i).col_idx, b2.dag(i).col_idx)
        assert np.array_equal(b.type_cost[3 + i], b2.type_cost[i])
    # every non-first-layer task has a predecessor: only the first layer (<= 64) is parentless
    for d in range(8):
        g = b.dag(d)
        indeg = np.bincount(g.col_idx, minlength=g.n)
        assert (indeg == 0).sum() <= 64


def test_layered_costs():
    b = inputs.layered(256)
    cpu = b.type_cost[:, :, 0].ravel()
    gpu = b.type_cost[:, :, 1].ravel()
    assert 60_000 < np.median(cpu) < 160_000  # log-normal around 100 us
    r = cpu / gpu
    assert r.min() > 0.45 and r.max() < 21


def test_layered_degree_typing():
    """Degree typing keeps the random layered shapes and gives every task the
    type 4 * bucket(in-degree) + bucket(out-degree), buckets {0}, {1}, {2,3}, {4..}."""
    r = inputs.layered(12, cfg=2)
    g = inputs.layered(12, cfg=2, typing="degree")
    assert g.n_types == 16
    assert np.array_equal(r.row_ptr, g.row_ptr) and np.array_equal(r.col_idx, g.col_idx)
    _check_csr(g)

    def bucket(k):
        return np.select([k == 0, k == 1, k <= 3], [0, 1, 2], 3)

    for d in range(g.ndag):
        x = g.dag(d)
        indeg = np.bincount(x.col_idx, minlength=x.n)
        outdeg = np.diff(x.row_ptr)
        np.testing.assert_array_equal(x.type, 4 * bucket(indeg) + bucket(outdeg))
    assert (g.type_cost[:, :, 0] >= 1).all() and (g.type_cost[:, :, 1] >= 1).all()
    assert len(np.unique(g.type)) > 6
