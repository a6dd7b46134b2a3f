"""CPU pins of the oracle's scorer-training restatement: central finite
differences, the integer inference network, straight-through estimators where
quantisation is the identity, and a closed form of AdamW."""
import numpy as np
import pytest

import inputs
import oracle


def _rand(rng, dims, scale=0.3):
    return rng.normal(0, scale, oracle.mlp_nweights_dims(*dims))


@pytest.mark.parametrize("seed", range(4))
def test_smooth_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    dims = (16, 4, 4)
    w = _rand(rng, dims)
    x = rng.uniform(0, 3, (9, 16))
    t = rng.normal(0, 1, 9)
    loss, g = oracle.mlp_loss_grad(w, x, t, dims, mode=0)
    eps = 1e-6
    fd = np.zeros_like(w)
    for i in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd[i] = (oracle.mlp_loss_grad(wp, x, t, dims, 0)[0] - oracle.mlp_loss_grad(wm, x, t, dims, 0)[0]) / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-3, atol=1e-6)
    assert loss > 0


def test_quantised_forward_is_the_integer_network():
    rng = np.random.default_rng(11)
    for _ in range(10):
        k = rng.integers(-128, 129, oracle.mlp_nweights()).astype(np.int16)
        f = rng.integers(0, 256, 16)
        y = oracle.mlp_score(k, f) / 64.0
        loss, _ = oracle.mlp_loss_grad(k / 64.0, f[None, :], np.array([y]), mode=1)
        assert loss == 0.0
        # off-grid real weights round to the same network
        loss, _ = oracle.mlp_loss_grad(k / 64.0 + rng.uniform(-0.007, 0.007, k.size), f[None, :], np.array([y]), mode=1)
        assert loss == 0.0


def test_straight_through_gradient_equals_smooth_where_quantisation_is_identity():
    rng = np.random.default_rng(3)
    dims = (16, 8, 8)
    w = rng.integers(-1, 2, oracle.mlp_nweights_dims(*dims)).astype(np.float64)  # integers: on the grid
    x = rng.integers(0, 4, (12, 16)).astype(np.float64)                            # integer pre-activations
    t = rng.normal(0, 5, 12)
    l0, g0 = oracle.mlp_loss_grad(w, x, t, dims, mode=0)
    l1, g1 = oracle.mlp_loss_grad(w, x, t, dims, mode=1)
    assert l0 == pytest.approx(l1, rel=1e-12)
    assert np.allclose(g0, g1, rtol=1e-12, atol=1e-12)


def test_straight_through_blocks_weights_outside_the_grid():
    dims = (16, 4, 4)
    w = np.zeros(oracle.mlp_nweights_dims(*dims))
    w[0] = 3.0  # 64 w = 192 > 128: clamped, no gradient
    x = np.ones((2, 16))
    _, g = oracle.mlp_loss_grad(w, x, np.array([1.0, 2.0]), dims, mode=1)
    assert g[0] == 0.0


def test_adamw_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2, so
    every step moves a weight by lr * sign(g) (no decay)."""
    w = np.array([1.0, -2.0, 0.5])
    m, v = np.zeros(3), np.zeros(3)
    g = np.array([0.3, -4.0, 1e-3])
    lr = 0.01
    for t in range(1, 6):
        oracle.adamw(w, m, v, g, t, lr, eps=1e-12)
    assert np.allclose(w, np.array([1.0, -2.0, 0.5]) - 5 * lr * np.sign(g), atol=1e-9)
    # decoupled decay with a zero gradient shrinks geometrically
    w2 = np.array([2.0]); m2 = np.zeros(1); v2 = np.zeros(1)
    for t in range(1, 4):
        oracle.adamw(w2, m2, v2, np.zeros(1), t, 0.1, wd=0.5)
    assert w2[0] == pytest.approx(2.0 * 0.95 ** 3)


def test_features_hand_computed():
    """The 16 scorer features of the candidates at two pops, each value computed by hand."""
    import json
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    g = json.load(open(os.path.join(gold, "features_hand_computed.json")))
    case = [c for c in json.load(open(os.path.join(gold, "sim_hand_traced.json")))["cases"] if c["name"] == g["dag"]][0]
    d = inputs.make_dag(case["n"], case["edges"], case["c_cpu"], case["c_gpu"])
    m = inputs.Machine(*case["machine"])
    for pop in g["pops"]:
        pol = oracle.Policy(oracle.POLICY_INSPIRIT)
        for k, v in case["policy_params"].items():
            setattr(pol, k, v)
        r = oracle.simulate(d, m, pol, unit_time=pop["unit_time"] or None, feat_pop=pop["pop"], feat_cap=8)
        assert list(r["feat_task"]) == pop["tasks"], pop["_why"]
        np.testing.assert_array_equal(r["feat"], np.array(pop["features"]), err_msg=pop["_why"])
