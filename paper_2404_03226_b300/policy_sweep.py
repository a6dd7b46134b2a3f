"""Sweep of the Nready controller's parameters (Sec. 4.4 names task_window,
s_inc, s_dec, dec_step, c and the ascending slope k_inc but gives no values)
over resident DAGs, every point one batched simulation on the GPU.

The attributes (inspiring ability and efficiency) do not depend on the
controller, so they are computed once per batch; each grid point then sets the
batch's policy (insp_batch_set_policy) and simulates every DAG.  The point
with the lowest mean makespan on a validation batch is then scored on a
held-out batch beside DMDA (FIFO pop), the default parameters and DMDAP by
inspiring ability, so the reported gain is not the selection's own.

    python -m paper_2404_03226_b300.policy_sweep [--val 2048] [--held 4096]
"""
from __future__ import annotations

import itertools
import json

import numpy as np

from . import _lib


def grid(P: int) -> list[dict]:
    """Parameter points for P workers: task_window, s_inc and s_dec (dec_step = s_dec) at P/2, P,
    2P (task_window also 4P), the slack c at 1, P/2, P, and k_inc at 1, 4 or 16 times the
    default of P tasks per unit time (k_factor 1 keeps each DAG's own default)."""
    pts = []
    for tw, si, sd, c, kf in itertools.product((P // 2 or 1, P, 2 * P, 4 * P), (P // 2 or 1, P, 2 * P),
                                                (P // 2 or 1, P, 2 * P), (1, max(1, P // 2), P), (1, 4, 16)):
        pts.append(dict(task_window=tw, s_inc=si, s_dec=sd, dec_step=sd, c=c, k_factor=kf))
    return pts


def _policy(kind: int, pt: dict | None, P: int, T_med: int):
    p = _lib.insp_policy()
    p.policy = kind
    if pt:
        p.task_window, p.s_inc, p.s_dec, p.dec_step, p.c = (pt["task_window"], pt["s_inc"], pt["s_dec"],
                                                             pt["dec_step"], pt["c"])
        if pt["k_factor"] != 1:  # k_inc = k_factor x P tasks per T (T: the batch's median unit time)
            p.k_inc_tasks = pt["k_factor"] * P
            p.k_inc_ns = T_med
    return p


def mean_makespans(batch, machine, points, extra=()):
    """Mean makespan of every grid point (INSPIRIT) and of the extra (name, policy kind) pairs
    on one resident batch; attributes computed once."""
    import torch
    from . import DagBatch, Machine
    P = machine.n_cpu + machine.n_gpu
    M = Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns)
    B = DagBatch(M, batch)
    ia, ie = B.attributes()
    torch.cuda.synchronize()
    # the per-DAG default unit times are 4 x the lower median GPU cost; one representative T for
    # the explicit k_inc points (the default points use each DAG's own T)
    cg = batch.task_cost[:, 1] if batch.task_cost is not None else None
    T_med = int(4 * np.median(cg)) if cg is not None else int(4 * np.median(batch.type_cost[:, :, 1]))
    out = {}

    def run(name, pol):
        _lib.insp_batch_set_policy(B.handle, pol)
        s = B.simulate(ia, ie)
        torch.cuda.synchronize()
        if _lib.insp_batch_status(B.handle) != 0:
            raise RuntimeError(_lib.last_error())
        out[name] = float(s.makespan.double().mean())

    for k, pt in enumerate(points):
        run(k, _policy(_lib.INSP_POLICY_INSPIRIT, pt, P, T_med))
    for name, kind in extra:
        run(name, _policy(kind, None, P, T_med))
    return out


def main(argv=None) -> None:
    import argparse
    import os
    import sys
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import inputs  # seeded workload generators (repository root)
    ap = argparse.ArgumentParser()
    ap.add_argument("--val", type=int, default=2048)
    ap.add_argument("--held", type=int, default=4096)
    a = ap.parse_args(argv)
    m = inputs.MACHINE_LAYERED
    P = m.n_cpu + m.n_gpu
    pts = grid(P)
    t0 = time.time()
    val = mean_makespans(inputs.layered(a.val, cfg=4, first=1 << 19), m, pts)
    best = min(range(len(pts)), key=lambda k: val[k])
    t1 = time.time()
    base = [("default", _lib.INSP_POLICY_INSPIRIT), ("dmda_fifo", _lib.INSP_POLICY_FIFO),
            ("dmdap_ia", _lib.INSP_POLICY_DMDAP_IA)]
    held = mean_makespans(inputs.layered(a.held, cfg=4, first=1 << 20), m, [pts[best]], base)
    ref = held["dmda_fifo"]
    dflt = next(k for k, pt in enumerate(pts) if pt == dict(task_window=P, s_inc=P, s_dec=P, dec_step=P,
                                                             c=max(1, P // 2), k_factor=1))
    rep = {"points": len(pts), "sweep_seconds": round(t1 - t0, 2), "best_on_validation": pts[best],
           "validation_best_vs_default": val[best] / val[dflt],
           "held_out_mean_makespan_ns": {"best": held[0], "default": held["default"], "dmda_fifo": ref,
                                          "dmdap_ia": held["dmdap_ia"]},
           "held_out_vs_dmda": {"best": held[0] / ref, "default": held["default"] / ref,
                                "dmdap_ia": held["dmdap_ia"] / ref}}
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
