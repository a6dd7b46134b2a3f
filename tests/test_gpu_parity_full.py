"""Full-workload parity of the CUDA path with the oracle, and the hand-traced
schedules on the GPU.

- Every one of the 4096 layered DAGs of the headline workload, bit-exact
  (attributes and schedule), in the launch the benchmark times.
- Every DAG of the tiled Cholesky / LU / QR batch at 16 and 32 tiles (1,536
  DAGs), and single LU and QR DAGs at 64 tiles (89,440 tasks) and QR at 32.
- The shipped learned scorer on 256 held-out layered DAGs plus DAGs whose
  ready pool outgrows the shared-memory queue, bit-exact against the
  oracle's integer network.
- The hand-traced schedules of the oracle's pins (efficiency and
  efficiency-with-locality picks, the default slope threshold at an explicit
  unit time), run through the C ABI and compared with the hand-derived values.
The oracle runs on all host cores (one DAG per thread)."""
import json
import os

import numpy as np
import pytest

import inputs
import oracle
from helpers import compare_many, gpu_run, oracle_many

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_headline_workload_every_dag_bit_exact():
    import torch
    import paper_2404_03226_b300 as P
    b = inputs.layered4096()
    m = inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.autotune()
    ia, ie, s = B.evaluate()
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    g = dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(), start=s.start.cpu().numpy(),
             end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())
    compare_many(b, g, m, oracle_many(b, range(b.ndag), m))


def test_tiled_16_32_batch_every_dag_bit_exact():
    b = inputs.tiled_workload(Ns=(16, 32))
    m = inputs.MACHINE_TILED
    assert b.ndag == 1536
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    compare_many(b, g, m, oracle_many(b, range(b.ndag), m))


@pytest.mark.parametrize("kind,N", [(inputs.KIND_QR, 32), (inputs.KIND_LU, 64), (inputs.KIND_QR, 64)])
def test_tiled_single_dags_bit_exact(kind, N):
    b = inputs.tiled(kind, N, 1, cfg=3, first=77)
    m = inputs.MACHINE_TILED
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    compare_many(b, g, m, oracle_many(b, [0], m))


def _shipped_weights():
    from paper_2404_03226_b300 import scorer
    bits, policy = scorer.load_trained()
    k = np.round((bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64) * 64).astype(np.int16)
    return bits, k, policy


def test_shipped_scorer_on_held_out_dags_bit_exact():
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    bits, k, _ = _shipped_weights()
    held = inputs.layered(256, cfg=4, first=1 << 20)
    wide = inputs.concat_dags([inputs.make_dag(300, [(0, v) for v in range(1, 300)],
                                               np.arange(1, 301) * 1000, np.arange(300, 0, -1) * 500)])
    chol = inputs.tiled(inputs.KIND_CHOLESKY, 16, 1, cfg=3, first=5)
    for b, m in ((held, inputs.MACHINE_LAYERED), (wide, inputs.MACHINE_LAYERED), (chol, inputs.MACHINE_TILED)):
        pol = P.insp_policy()
        pol.policy = P.INSP_POLICY_LEARNED
        M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns, pol)
        _lib.insp_set_scorer(M.handle, bits)
        B = P.DagBatch(M, b)
        ia, ie = B.attributes()
        s = B.simulate(ia, ie)
        torch.cuda.synchronize()
        assert (B.status() == 0).all()
        g = dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(),
                 start=s.start.cpu().numpy(), end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())
        res = oracle_many(b, range(b.ndag), m, "learned", mlp_weights=k)
        compare_many(b, g, m, res)
        if b is not held:  # the ready pool outgrows the shared-memory queue (sim_queue entries)
            r = oracle.simulate(b.dag(0), m, oracle.Policy(oracle.POLICY_LEARNED), mlp_weights=k, trace=True)
            assert int(r["trace"]["nready"].max()) > B.tuning["sim_queue"]


def test_hand_traced_schedules_on_the_gpu():
    import torch
    import paper_2404_03226_b300 as P
    g = json.load(open(os.path.join(GOLD, "sim_hand_traced.json")))
    names = {"inspirit": P.INSP_POLICY_INSPIRIT, "fifo": P.INSP_POLICY_FIFO, "dmdap_ia": P.INSP_POLICY_DMDAP_IA,
             "dmdap_bl": P.INSP_POLICY_DMDAP_BL}
    for case in g["cases"]:
        dag = inputs.make_dag(case["n"], case["edges"], case["c_cpu"], case["c_gpu"])
        b = inputs.concat_dags([dag])
        mach = case["machine"]
        for pname in case["policies"]:
            pol = P.insp_policy()
            pol.policy = names[pname]
            for key, v in case.get("policy_params", {}).items():
                setattr(pol, key, v)
            B = P.DagBatch(P.Machine(*mach, pol), b)
            ut = None if "unit_time" not in case else np.array([case["unit_time"]], np.int64)
            ia, ie = B.attributes(ut)
            s, tr = B.simulate_trace(ia, ie)
            torch.cuda.synchronize()
            assert (B.status() == 0).all()
            what = f"{case['name']} ({pname})"
            assert list(s.worker.cpu().numpy()) == case["worker"], what
            assert list(s.start.cpu().numpy()) == case["start"], what
            assert list(s.end.cpu().numpy()) == case["end"], what
            assert int(s.makespan.cpu()[0]) == case["makespan"], what
            if "order" in case:
                assert list(tr["pop_task"].cpu().numpy()) == case["order"], what
            if "modes" in case:
                assert list(tr["pop_mode"].cpu().numpy()) == case["modes"], what
