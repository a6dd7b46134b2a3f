"""Training driver of the learned proposal scorer (no counterpart in the paper).

Rollouts come from the simulator itself (insp_simulate_rollout): for every
training DAG a decision point (a pop) is drawn, the candidates of the popping
worker's queue are recorded with their 16 features, and the run is repeated
once per candidate with that candidate forced at the decision point.  A
candidate's target is the relative makespan gain, in percent, of forcing it
over the plain INSPIRIT run, centred on the mean over that decision's
candidates (the scorer ranks candidates of one pop, so only their relative
gains matter).  The MLP 16 -> 64 -> 64 -> 1 is trained on the
GPU by the library's kernels (insp_scorer_train_grad in quantisation-aware
mode, insp_adamw), then rounded to the BF16 grid (insp_scorer_quantize) and
installed with insp_set_scorer.  The plain INSPIRIT priority stays the
fallback: the learned policy is used only if its mean makespan on a
validation split is no worse.

torch is used for device buffers only; numpy only assembles labels.
"""
from __future__ import annotations

from dataclasses import dataclass

import os

import numpy as np

from . import _lib

IN, H = 16, 64
NW = IN * H + H + H * H + H + H + 1
CAP = 8


def _policy(kind: int) -> _lib.insp_policy:
    p = _lib.insp_policy()
    p.policy = kind
    return p


@dataclass
class Rollouts:
    feat: np.ndarray     # [N, 16] int32
    target: np.ndarray   # [N] float32, % makespan gain of forcing the candidate
    dag: np.ndarray      # [N] index of the DAG the row came from


def collect_rollouts(batch, machine, seed: int, cap: int = CAP) -> Rollouts:
    """One decision point per DAG of `batch` (an inputs.Batch-like object)."""
    import torch
    from . import DagBatch, Machine
    M = Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns, _policy(_lib.INSP_POLICY_INSPIRIT))
    B = DagBatch(M, batch)
    nd, n = B.ndag, B.n_tasks
    dev = torch.device("cuda")
    ia, ie = B.attributes()
    sizes = np.diff(np.asarray(batch.task_base))
    rng = np.random.default_rng(seed)
    pop = np.floor(rng.random(nd) * np.maximum(sizes, 1)).astype(np.int32)
    d_pop = torch.from_numpy(pop).to(dev)
    worker = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    start = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    end = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    mk0 = torch.empty(nd, dtype=torch.int64, device=dev)
    ftask = torch.full((nd, cap), -1, dtype=torch.int32, device=dev)
    feat = torch.zeros((nd, cap, IN), dtype=torch.int32, device=dev)
    fn = torch.zeros(nd, dtype=torch.int32, device=dev)
    _lib.insp_simulate_rollout(B.handle, ia, ie, worker, start, end, mk0, None, None, d_pop, cap, ftask, feat, fn)
    mks = []
    for r in range(cap):
        mk = torch.empty(nd, dtype=torch.int64, device=dev)
        force_task = ftask[:, r].contiguous()
        _lib.insp_simulate_rollout(B.handle, ia, ie, worker, start, end, mk, d_pop, force_task)
        mks.append(mk)
    torch.cuda.synchronize()
    if _lib.insp_batch_status(B.handle) != 0:
        raise RuntimeError("rollout simulation failed: " + _lib.last_error())
    mk0 = mk0.cpu().numpy().astype(np.float64)
    fn = fn.cpu().numpy()
    feat = feat.cpu().numpy()
    mk = np.stack([m.cpu().numpy() for m in mks], 1).astype(np.float64)
    rows_f, rows_t, rows_d = [], [], []
    for d in np.nonzero(fn >= 2)[0]:
        k = int(fn[d])
        gain = (mk0[d] - mk[d, :k]) / mk0[d] * 100.0
        rows_f.append(feat[d, :k])
        rows_t.append(gain - gain.mean())
        rows_d.append(np.full(k, d))
    if not rows_f:
        return Rollouts(np.zeros((0, IN), np.int32), np.zeros(0, np.float32), np.zeros(0, np.int64))
    return Rollouts(np.concatenate(rows_f).astype(np.int32), np.concatenate(rows_t).astype(np.float32),
                    np.concatenate(rows_d))


def init_weights(seed: int) -> np.ndarray:
    """Small random weights with positive biases (floor activations need
    positive pre-activations to pass gradients)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(NW, np.float32)
    o = 0
    w[o:o + IN * H] = rng.normal(0, 0.08, IN * H); o += IN * H
    w[o:o + H] = 2.0; o += H
    w[o:o + H * H] = rng.normal(0, 0.06, H * H); o += H * H
    w[o:o + H] = 2.0; o += H
    w[o:o + H] = rng.normal(0, 0.05, H); o += H
    w[o] = 0.0
    return w


def train(roll: Rollouts, epochs: int = 30, batch: int = 4096, lr: float = 2e-3, seed: int = 0,
          w0: np.ndarray | None = None, log=None, checkpoint: str | None = None):
    """Quantisation-aware training on the GPU, the loss and gradient of each
    minibatch on the tensor cores (insp_scorer_train_grad_tc: BF16 mma.sync,
    FP32 accumulation, FP32 master weights), then AdamW; returns (fp32 master
    weights, BF16 grid weights as uint16, per-epoch mean loss).

    checkpoint: a .npz path written after every epoch (fp32 weights, AdamW
    moments, step, epoch, seed, loss history); if it exists when training
    starts, training resumes from it.  The gradient reduction is deterministic
    and the epoch permutations are replayed from the seed, so a resumed run
    ends with the same bits as an uninterrupted one."""
    import torch
    dev = torch.device("cuda")
    n = len(roll.target)
    x = torch.from_numpy(roll.feat.astype(np.float32)).to(dev)
    y = torch.from_numpy(roll.target.astype(np.float32)).to(dev)
    w = torch.from_numpy(init_weights(seed) if w0 is None else w0.astype(np.float32)).to(dev)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    g = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    bs = min(batch, n)
    part = torch.empty(((bs + 15) // 16) * (NW + 1), dtype=torch.float32, device=dev)  # per-tile partials
    rng = np.random.default_rng(seed + 1)
    t = 0
    hist = []
    first = 0
    if checkpoint and os.path.exists(checkpoint):
        ck = np.load(checkpoint)
        if int(ck["seed"]) != seed or int(ck["nweights"]) != NW:
            raise ValueError(f"checkpoint {checkpoint} belongs to another run")
        w.copy_(torch.from_numpy(ck["w"]))
        m.copy_(torch.from_numpy(ck["m"]))
        v.copy_(torch.from_numpy(ck["v"]))
        t, first, hist = int(ck["step"]), int(ck["epoch"]), [float(x) for x in ck["hist"]]
        for _ in range(first):  # the permutations of the epochs already done
            rng.permutation(n)
    for ep in range(first, epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        losses = []
        for s0 in range(0, n - bs + 1, bs):
            idx = perm[s0:s0 + bs]
            xb = x[idx].contiguous()
            yb = y[idx].contiguous()
            _lib.insp_scorer_train_grad_tc(IN, H, H, w, 1, bs, xb, yb, part, g, loss)
            t += 1
            _lib.insp_adamw(NW, w, m, v, g, t, lr)
            losses.append(loss)
        ep_loss = float(torch.stack(losses).mean()) if losses else float("nan")
        hist.append(ep_loss)
        if log:
            log(f"epoch {ep}: loss {ep_loss:.4f}")
        if checkpoint:
            tmp = checkpoint + ".tmp.npz"
            np.savez(tmp, w=w.cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(), step=t, epoch=ep + 1, seed=seed,
                     nweights=NW, hist=np.array(hist))
            os.replace(tmp, checkpoint)
    q = torch.empty(NW, dtype=torch.int16, device=dev)
    _lib.insp_scorer_quantize(NW, w, q)
    torch.cuda.synchronize()
    return w.cpu().numpy(), q.cpu().numpy().view(np.uint16), hist


def evaluate(batch, machine, bf16_weights) -> dict:
    """Mean makespan of the plain INSPIRIT priority and of the learned scorer
    on `batch`; the policy to ship is the learned one only if it is no worse."""
    import torch
    from . import DagBatch, Machine
    res = {}
    for name, kind in (("inspirit", _lib.INSP_POLICY_INSPIRIT), ("learned", _lib.INSP_POLICY_LEARNED)):
        M = Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns, _policy(kind))
        if kind == _lib.INSP_POLICY_LEARNED:
            _lib.insp_set_scorer(M.handle, np.ascontiguousarray(bf16_weights, np.uint16))
        B = DagBatch(M, batch)
        ia, ie = B.attributes()
        s = B.simulate(ia, ie)
        torch.cuda.synchronize()
        if _lib.insp_batch_status(B.handle) != 0:
            raise RuntimeError(_lib.last_error())
        res[name] = s.makespan.cpu().numpy()
    mean_plain = float(res["inspirit"].mean())
    mean_learned = float(res["learned"].mean())
    return {"mean_makespan_inspirit": mean_plain, "mean_makespan_learned": mean_learned,
            "gain_pct": (mean_plain - mean_learned) / mean_plain * 100.0,
            "wins": int((res["learned"] < res["inspirit"]).sum()),
            "losses": int((res["learned"] > res["inspirit"]).sum()),
            "policy": "learned" if mean_learned <= mean_plain else "inspirit (fallback)",
            "makespan_inspirit": res["inspirit"], "makespan_learned": res["learned"]}


TRAINED = __import__("os").path.join(__import__("os").path.dirname(__file__), "scorer_k.txt")


def load_trained(path: str = TRAINED) -> tuple[np.ndarray, str]:
    """(BF16 bit patterns, shipped policy) of the scorer trained by main()."""
    policy = "learned"
    with open(path) as f:
        for line in f:
            if line.startswith("# policy shipped:"):
                policy = line.split(":", 1)[1].strip()
            elif line.strip() and not line.startswith("#"):
                k = np.array([int(t) for t in line.split()], np.int64)
    f32 = (k.astype(np.float64) / 64.0).astype(np.float32)
    return (f32.view(np.uint32) >> 16).astype(np.uint16), policy


def score_throughput(rows: int, steps: int = 20, warmup: int = 3, seed: int = 0) -> dict:
    """Batched scoring (insp_scorer_eval, tcgen05 MMAs) of `rows` random feature rows with the
    shipped weights, timed with CUDA events over `steps` calls after `warmup`; 72 bytes per row
    (16 int32 features in, one int64 score out) and 2 x (16 x 64 + 64 x 64 + 64) flops."""
    import torch
    from . import Machine
    M = Machine(2, 1, 0)
    bits, _ = load_trained()
    _lib.insp_set_scorer(M.handle, bits)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    feat = torch.randint(0, 256, (rows, IN), dtype=torch.int32, device="cuda", generator=g)
    out = torch.empty(rows, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        _lib.insp_scorer_eval(M.handle, feat, rows, out, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(steps):
        _lib.insp_scorer_eval(M.handle, feat, rows, out, s)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"rows": rows, "ms": round(ms, 4), "rows_per_s": rows / ms * 1e3, "GB_s": rows * 72 / ms / 1e6,
            "TFLOP_s": rows * 2 * (IN * H + H * H + H) / ms / 1e9,
            "timeouts": int((out == _lib.INSP_SCORE_TIMEOUT).sum())}


def main(argv=None) -> None:
    """Train on rollouts of layered DAGs and evaluate on held-out ones:
    python -m paper_2404_03226_b300.scorer --train 100000 --eval 4096 --out FILE
    or time the batched scoring: python -m paper_2404_03226_b300.scorer --score-rows 16777216"""
    import argparse
    import json
    import sys
    import time
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import inputs  # seeded workload generators (repository root)
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=100000)
    ap.add_argument("--val", type=int, default=2048)
    ap.add_argument("--eval", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--chunk", type=int, default=8192)
    ap.add_argument("--decisions", type=int, default=4, help="decision points drawn per training DAG")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--out", default="")
    ap.add_argument("--checkpoint", default="", help="training checkpoint (.npz), resumed from if present")
    ap.add_argument("--score-rows", type=int, default=0, help="only time batched scoring of this many rows")
    a = ap.parse_args(argv)
    if a.score_rows:
        print(json.dumps(score_throughput(a.score_rows)))
        return
    m = inputs.MACHINE_LAYERED
    t0 = time.time()
    parts = []
    for first in range(0, a.train, a.chunk):
        b = inputs.layered(min(a.chunk, a.train - first), cfg=4, first=first)
        for r in range(a.decisions):
            parts.append(collect_rollouts(b, m, seed=(a.seed + first) * 16 + r))
    roll = Rollouts(np.concatenate([p.feat for p in parts]), np.concatenate([p.target for p in parts]),
                    np.concatenate([p.dag for p in parts]))
    t1 = time.time()
    w, q, hist = train(roll, epochs=a.epochs, lr=a.lr, seed=a.seed, log=lambda s: print(s, file=sys.stderr),
                       checkpoint=a.checkpoint or None)
    t2 = time.time()
    val = evaluate(inputs.layered(a.val, cfg=4, first=1 << 19), m, q)       # seed set A, not trained on
    held = evaluate(inputs.layered(a.eval, cfg=4, first=1 << 20), m, q)     # seed set B
    use = "learned" if val["mean_makespan_learned"] <= val["mean_makespan_inspirit"] else "inspirit (fallback)"
    rep = {"train_dags": a.train, "rollout_rows": int(len(roll.target)), "epochs": a.epochs,
           "loss_first": hist[0], "loss_last": hist[-1], "rollout_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
           "validation": {k: v for k, v in val.items() if not k.startswith("makespan_")},
           "policy_shipped": use,
           "held_out": {k: v for k, v in held.items() if not k.startswith("makespan_")},
           "held_out_gain_pct_of_shipped": held["gain_pct"] if use == "learned" else 0.0}
    print(json.dumps(rep))
    if a.out:
        k = np.round((q.astype(np.uint32) << 16).view(np.float32) * 64).astype(np.int64)
        with open(a.out, "w") as f:
            f.write("# learned scorer, grid numerators k (weight = k/64), layout W1[16][64] b1 W2[64][64] b2 W3[64] b3\n")
            f.write(f"# python -m paper_2404_03226_b300.scorer --train {a.train} --val {a.val} --eval {a.eval} "
                    f"--epochs {a.epochs} --decisions {a.decisions} --lr {a.lr} --seed {a.seed}\n")
            f.write(f"# policy shipped: {use}\n")
            f.write(" ".join(str(int(x)) for x in k) + "\n")


if __name__ == "__main__":
    main()
