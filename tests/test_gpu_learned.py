"""The learned proposal scorer on the GPU: tensor-core scoring and the learned
pop bit-exact against the oracle's integer network, rollout controls (forced
pick, candidate features) against the oracle's trace, training gradients and
AdamW against the oracle's fp64 restatement, and a small end-to-end training
run with the plain-INSPIRIT fallback."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _bf16_bits(k):
    f = (np.asarray(k, np.float64) / 64.0).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def _weights(seed, spread=128):
    rng = np.random.default_rng(seed)
    return rng.integers(-spread, spread + 1, oracle.mlp_nweights()).astype(np.int16)


def test_scorer_eval_matches_integer_network():
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    rng = np.random.default_rng(1)
    M = P.Machine(2, 1, 0)
    for seed, spread in ((0, 128), (1, 8), (2, 1)):
        k = _weights(seed, spread)
        _lib.insp_set_scorer(M.handle, _bf16_bits(k))
        feat = rng.integers(0, 256, (1000, 16)).astype(np.int32)
        feat[:5] = 0
        feat[5:10] = 255
        d_feat = torch.from_numpy(feat).cuda()
        out = torch.empty(1000, dtype=torch.int64, device="cuda")
        _lib.insp_scorer_eval(M.handle, d_feat, 1000, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        exp = np.array([oracle.mlp_score(k, f) for f in feat])
        np.testing.assert_array_equal(got, exp)


def test_scorer_eval_many_tiles_ragged_and_clamped():
    """The tensor-core scoring over more 128-row tiles than the persistent grid has CTAs (four
    per SM), a ragged last tile and features outside [0, 255] (clamped): sampled rows against
    the oracle's integer network, every row scored (no timeout sentinel)."""
    import time
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    M = P.Machine(2, 1, 0)
    k = _weights(4, 64)
    _lib.insp_set_scorer(M.handle, _bf16_bits(k))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = sms * 4 * 128 * 2 + 77
    rng = np.random.default_rng(5)
    feat = rng.integers(-40, 300, (n, 16)).astype(np.int32)
    d_feat = torch.from_numpy(feat).cuda()
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    _lib.insp_scorer_eval(M.handle, d_feat, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert not (got == _lib.INSP_SCORE_TIMEOUT).any()
    rows = np.unique(np.concatenate([np.arange(0, n, 211), np.arange(n - 300, n), np.arange(0, 300)]))
    exp = np.array([oracle.mlp_score(k, np.clip(feat[r], 0, 255)) for r in rows])
    np.testing.assert_array_equal(got[rows], exp)
    # rows that are not 16-byte aligned (one int32 in): per-thread loads instead of bulk copies
    flat = torch.empty(n * 16 + 1, dtype=torch.int32, device="cuda")
    flat[1:] = d_feat.reshape(-1)
    out2 = torch.full((n,), 7, dtype=torch.int64, device="cuda")
    _lib.insp_scorer_eval(M.handle, flat[1:], n, out2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out2.cpu().numpy(), got)
    t0 = time.perf_counter()
    for _ in range(10):
        _lib.insp_scorer_eval(M.handle, d_feat, n, out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / 10
    print(f"\nscoring {n} rows on the tensor cores: {dt * 1e3:.3f} ms ({n / dt / 1e9:.2f} G rows/s)")


def test_set_scorer_rejects_off_grid_weights():
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    M = P.Machine(2, 1, 0)
    bits = _bf16_bits(_weights(3))
    bad = bits.copy()
    bad[7] = np.float32(1.0 / 3.0).view(np.uint32) >> 16
    with pytest.raises(_lib.InspError):
        _lib.insp_set_scorer(M.handle, bad)
    big = bits.copy()
    big[0] = np.float32(4.0).view(np.uint32) >> 16  # k = 256
    with pytest.raises(_lib.InspError):
        _lib.insp_set_scorer(M.handle, big)


def _gpu_learned(batch, machine, k):
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    pol = P.insp_policy()
    pol.policy = P.INSP_POLICY_LEARNED
    M = P.Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns, pol)
    _lib.insp_set_scorer(M.handle, _bf16_bits(k))
    B = P.DagBatch(M, batch)
    ia, ie = B.attributes()
    s = B.simulate(ia, ie)
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    return s


@pytest.mark.parametrize("seed,spread", [(10, 128), (11, 6), (12, 2)])
def test_learned_simulation_matches_oracle(seed, spread):
    k = _weights(seed, spread)
    b = inputs.concat([inputs.layered(12, cfg=96, n_min=20, n_max=700), inputs.concat_dags(
        [inputs.make_dag(40, [], np.arange(1, 41), np.arange(40, 0, -1))])])
    m = inputs.MACHINE_LAYERED
    s = _gpu_learned(b, m, k)
    pol = oracle.Policy(oracle.POLICY_LEARNED)
    for d in range(b.ndag):
        g = b.dag(d)
        r = oracle.simulate(g, m, pol, mlp_weights=k)
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        np.testing.assert_array_equal(s.worker.cpu().numpy()[tb:te], r["worker"], err_msg=f"DAG {d}")
        np.testing.assert_array_equal(s.start.cpu().numpy()[tb:te], r["start"], err_msg=f"DAG {d}")
        assert int(s.makespan.cpu()[d]) == r["makespan"]


def test_rollout_features_and_forced_pick_match_oracle():
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    b = inputs.layered(10, cfg=97, n_min=60, n_max=500)
    m = inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    B = P.DagBatch(M, b)
    ia, ie = B.attributes()
    n, nd, cap = b.n_total, b.ndag, 8
    sizes = b.sizes()
    pop = (np.arange(nd) * 7919 % np.maximum(sizes, 1)).astype(np.int32)
    dev = torch.device("cuda")
    bufs = [torch.empty(n, dtype=t, device=dev) for t in (torch.int32, torch.int64, torch.int64)]
    mk = torch.empty(nd, dtype=torch.int64, device=dev)
    ftask = torch.full((nd, cap), -1, dtype=torch.int32, device=dev)
    feat = torch.zeros((nd, cap, 16), dtype=torch.int32, device=dev)
    fn = torch.zeros(nd, dtype=torch.int32, device=dev)
    d_pop = torch.from_numpy(pop).to(dev)
    _lib.insp_simulate_rollout(B.handle, ia, ie, *bufs, mk, None, None, d_pop, cap, ftask, feat, fn)
    torch.cuda.synchronize()
    fn_h, ft_h, f_h = fn.cpu().numpy(), ftask.cpu().numpy(), feat.cpu().numpy()
    forced = np.array([ft_h[d, fn_h[d] - 1] if fn_h[d] > 0 else -1 for d in range(nd)], np.int32)
    mk2 = torch.empty(nd, dtype=torch.int64, device=dev)
    _lib.insp_simulate_rollout(B.handle, ia, ie, *bufs, mk2, d_pop, torch.from_numpy(forced).to(dev))
    torch.cuda.synchronize()
    w2, s2 = bufs[0].cpu().numpy(), bufs[1].cpu().numpy()
    for d in range(nd):
        g = b.dag(d)
        r = oracle.simulate(g, m, feat_pop=int(pop[d]), feat_cap=cap)
        assert fn_h[d] == len(r["feat_task"])
        np.testing.assert_array_equal(ft_h[d, :fn_h[d]], r["feat_task"])
        np.testing.assert_array_equal(f_h[d, :fn_h[d]], r["feat"])
        rf = oracle.simulate(g, m, force=(int(pop[d]), int(forced[d])))
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        np.testing.assert_array_equal(w2[tb:te], rf["worker"])
        np.testing.assert_array_equal(s2[tb:te], rf["start"])
        assert int(mk2.cpu()[d]) == rf["makespan"]


@pytest.mark.parametrize("dims,mode", [((16, 4, 4), 0), ((16, 4, 4), 1), ((16, 64, 64), 0), ((16, 64, 64), 1)])
def test_training_gradient_matches_oracle(dims, mode):
    import torch
    from paper_2404_03226_b300 import _lib
    rng = np.random.default_rng(sum(dims) + mode)
    nw = oracle.mlp_nweights_dims(*dims)
    w = rng.normal(0, 0.1, nw).astype(np.float32)
    w[dims[0] * dims[1]:dims[0] * dims[1] + dims[1]] = 1.5  # live first-layer units
    n = 300
    x = rng.integers(0, 20, (n, dims[0])).astype(np.float32)
    t = rng.normal(0, 2, n).astype(np.float32)
    dev = torch.device("cuda")
    dw, dx, dt = (torch.from_numpy(a).to(dev) for a in (w, x, t))
    g = torch.zeros(nw, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.empty(n * (2 * dims[1] + 2 * dims[2] + 2), dtype=torch.float32, device=dev)
    _lib.insp_scorer_train_grad(dims[0], dims[1], dims[2], dw, mode, n, dx, dt, work, g, loss)
    torch.cuda.synchronize()
    l_ref, g_ref = oracle.mlp_loss_grad(w.astype(np.float64), x, t, dims, mode)
    assert float(loss.cpu()[0]) == pytest.approx(l_ref, rel=1e-5)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(g.cpu().numpy(), g_ref, rtol=1e-4, atol=1e-5 * scale)
    # deterministic: the same call gives the same bits
    g2 = torch.zeros_like(g)
    _lib.insp_scorer_train_grad(dims[0], dims[1], dims[2], dw, mode, n, dx, dt, work, g2, loss)
    assert torch.equal(g, g2)


def test_adamw_and_quantize_match_oracle():
    import torch
    from paper_2404_03226_b300 import _lib
    rng = np.random.default_rng(4)
    nw = 1000
    w = rng.normal(0, 1, nw)
    m, v = np.zeros(nw), np.zeros(nw)
    dev = torch.device("cuda")
    dw = torch.from_numpy(w.astype(np.float32)).to(dev)
    dm, dv = torch.zeros(nw, device=dev), torch.zeros(nw, device=dev)
    wr = w.astype(np.float32).astype(np.float64)
    for t in range(1, 6):
        g = rng.normal(0, 1, nw)
        dg = torch.from_numpy(g.astype(np.float32)).to(dev)
        _lib.insp_adamw(nw, dw, dm, dv, dg, t, 0.01, 0.9, 0.999, 1e-8, 0.01)
        oracle.adamw(wr, m, v, g.astype(np.float32).astype(np.float64), t, 0.01, wd=0.01)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dw.cpu().numpy(), wr, rtol=1e-5, atol=1e-6)
    q = torch.empty(nw, dtype=torch.int16, device=dev)
    grid = torch.from_numpy(rng.uniform(-2.5, 2.5, nw).astype(np.float32)).to(dev)
    _lib.insp_scorer_quantize(nw, grid, q)
    torch.cuda.synchronize()
    bits = q.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    got = bits.view(np.float32).astype(np.float64) * 64
    k = grid.cpu().numpy().astype(np.float64) * 64
    exp = np.clip(np.sign(k) * np.floor(np.abs(k) + 0.5), -128, 128)
    np.testing.assert_array_equal(got, exp)


def test_small_training_run_and_fallback():
    from paper_2404_03226_b300 import scorer
    train = inputs.layered(384, cfg=4, first=0, n_max=600)
    held = inputs.layered(128, cfg=4, first=1 << 20, n_max=600)
    m = inputs.MACHINE_LAYERED
    roll = scorer.collect_rollouts(train, m, seed=5)
    assert len(roll.target) > 500
    w, q, hist = scorer.train(roll, epochs=8, batch=1024, seed=5)
    assert hist[-1] < hist[0]
    res = scorer.evaluate(held, m, q)
    chosen = res["mean_makespan_learned"] if res["policy"] == "learned" else res["mean_makespan_inspirit"]
    assert chosen <= res["mean_makespan_inspirit"]


def test_shipped_scorer_on_held_out_dags():
    """The trained scorer shipped with the library (layered workload, 100k
    training DAGs) against plain INSPIRIT on the 4096 held-out DAGs: when the
    learned policy is shipped it must not lose on average; otherwise the plain
    priority is the fallback."""
    from paper_2404_03226_b300 import scorer
    bits, shipped = scorer.load_trained()
    held = inputs.layered(4096, cfg=4, first=1 << 20)
    res = scorer.evaluate(held, inputs.MACHINE_LAYERED, bits)
    print(f"held-out gain of the learned scorer: {res['gain_pct']:.3f}% "
          f"(wins {res['wins']}, losses {res['losses']}), shipped: {shipped}")
    if shipped == "learned":
        assert res["mean_makespan_learned"] <= res["mean_makespan_inspirit"]
    else:
        assert shipped.startswith("inspirit")


def test_training_checkpoint_resume_is_exact(tmp_path):
    """Training interrupted after 2 epochs and resumed from its checkpoint ends
    with the same bits as 4 uninterrupted epochs."""
    from paper_2404_03226_b300 import scorer
    train = inputs.layered(96, cfg=4, first=7, n_max=400)
    roll = scorer.collect_rollouts(train, inputs.MACHINE_LAYERED, seed=9)
    w_full, q_full, h_full = scorer.train(roll, epochs=4, batch=512, seed=3)
    ck = str(tmp_path / "ck.npz")
    scorer.train(roll, epochs=2, batch=512, seed=3, checkpoint=ck)
    w_res, q_res, h_res = scorer.train(roll, epochs=4, batch=512, seed=3, checkpoint=ck)
    np.testing.assert_array_equal(w_res, w_full)
    np.testing.assert_array_equal(q_res, q_full)
    assert h_res == h_full


@pytest.mark.parametrize("dims,mode", [((16, 4, 4), 0), ((16, 4, 4), 1), ((16, 64, 64), 0), ((16, 64, 64), 1),
                                       ((32, 64, 64), 1), ((7, 13, 5), 0), ((7, 13, 5), 1)])
def test_training_gradient_on_tensor_cores_matches_oracle(dims, mode):
    """The tensor-core form (BF16 mma.sync, FP32 accumulation) against the oracle's fp64
    gradient, at the tolerance of the FP32 path: each FP32 operand enters as hi + lo BF16 parts
    and each product drops only lo*lo, below 2^-16 of the product, so the relative error of a
    product stays under 2^-16 (1.5e-5) and the FP32 sums over up to a few hundred terms keep
    the gradient within rtol 1e-4 (atol 1e-5 of the largest gradient for cancelling sums).  In
    the quantisation-aware mode (1) the forward pass is exact, so the loss matches to 1e-6;
    the smooth mode (0) carries the split error into the loss (1e-4).  300 samples: a ragged
    last tile.  Deterministic, and close to the FP32 form."""
    import torch
    from paper_2404_03226_b300 import _lib
    rng = np.random.default_rng(sum(dims) * 7 + mode)
    nw = oracle.mlp_nweights_dims(*dims)
    w = rng.normal(0, 0.1, nw).astype(np.float32)
    w[dims[0] * dims[1]:dims[0] * dims[1] + dims[1]] = 1.5  # live first-layer units
    n = 300
    x = rng.integers(0, 20, (n, dims[0])).astype(np.float32)
    t = rng.normal(0, 2, n).astype(np.float32)
    dev = torch.device("cuda")
    dw, dx, dt = (torch.from_numpy(a).to(dev) for a in (w, x, t))
    g = torch.zeros(nw, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    part = torch.empty(((n + 15) // 16) * (nw + 1), dtype=torch.float32, device=dev)
    _lib.insp_scorer_train_grad_tc(dims[0], dims[1], dims[2], dw, mode, n, dx, dt, part, g, loss)
    torch.cuda.synchronize()
    l_ref, g_ref = oracle.mlp_loss_grad(w.astype(np.float64), x, t, dims, mode)
    assert float(loss.cpu()[0]) == pytest.approx(l_ref, rel=1e-6 if mode else 1e-4)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(g.cpu().numpy(), g_ref, rtol=1e-4, atol=1e-5 * scale)
    g2 = torch.zeros_like(g)
    _lib.insp_scorer_train_grad_tc(dims[0], dims[1], dims[2], dw, mode, n, dx, dt, part, g2, loss)
    assert torch.equal(g, g2)
    work = torch.empty(n * (2 * dims[1] + 2 * dims[2] + 2), dtype=torch.float32, device=dev)
    g3 = torch.zeros_like(g)
    _lib.insp_scorer_train_grad(dims[0], dims[1], dims[2], dw, mode, n, dx, dt, work, g3, loss)
    np.testing.assert_allclose(g.cpu().numpy(), g3.cpu().numpy(), rtol=1e-4, atol=1e-5 * scale)


def test_training_time_tensor_cores_vs_fp32():
    """Both forms on one minibatch of the trainer's shape (4096 samples, 16 -> 64 -> 64 -> 1,
    quantisation-aware): the tensor-core form is timed beside the FP32 one (printed) and gives
    the same gradient within the tolerance above."""
    import torch
    from paper_2404_03226_b300 import _lib, scorer
    rng = np.random.default_rng(11)
    nw = oracle.mlp_nweights_dims(16, 64, 64)
    n = 4096
    dev = torch.device("cuda")
    w = torch.from_numpy(scorer.init_weights(3)).to(dev)
    x = torch.from_numpy(rng.integers(0, 256, (n, 16)).astype(np.float32)).to(dev)
    t = torch.from_numpy(rng.normal(0, 2, n).astype(np.float32)).to(dev)
    g1, g2 = torch.zeros(nw, device=dev), torch.zeros(nw, device=dev)
    loss = torch.zeros(1, device=dev)
    part = torch.empty(((n + 15) // 16) * (nw + 1), device=dev)
    work = torch.empty(n * (2 * 64 + 2 * 64 + 2), device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(3):
        _lib.insp_scorer_train_grad_tc(16, 64, 64, w, 1, n, x, t, part, g1, loss)
        _lib.insp_scorer_train_grad(16, 64, 64, w, 1, n, x, t, work, g2, loss)
    ev[0].record()
    for _ in range(20):
        _lib.insp_scorer_train_grad_tc(16, 64, 64, w, 1, n, x, t, part, g1, loss)
    ev[1].record()
    ev[2].record()
    for _ in range(20):
        _lib.insp_scorer_train_grad(16, 64, 64, w, 1, n, x, t, work, g2, loss)
    ev[3].record()
    torch.cuda.synchronize()
    tc, fp = ev[0].elapsed_time(ev[1]) / 20, ev[2].elapsed_time(ev[3]) / 20
    print(f"gradient of a 4096-sample minibatch: tensor cores {tc:.3f} ms, FP32 CUDA cores {fp:.3f} ms")
    scale = float(g2.abs().max())
    np.testing.assert_allclose(g1.cpu().numpy(), g2.cpu().numpy(), rtol=1e-4, atol=1e-5 * scale)
