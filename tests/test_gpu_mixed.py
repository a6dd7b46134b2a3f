"""The mixed-size stress workload on the GPU (32 CPU + 8 GPU workers, so every lane of the
simulation warp owns two workers): a sample of the workload's own DAGs bit-exact against the
oracle in one batch with the workload's two ~200,000-task golden DAGs, whose attributes and
schedules must hash to the digests the oracle wrote (tests/golden/mixed_200k.json), under both
ability sweeps; and the plain and learned policies on the sample."""
import hashlib
import json
import os

import numpy as np
import pytest

import inputs
import oracle
from helpers import compare_many, oracle_many

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "mixed_200k.json")


def _sample_indices(k=40, cap=15000):
    sizes = inputs.mixed_sizes(2000)
    return [i for i in range(2000) if sizes[i] <= cap][:k]


_CACHE = {}


def _oracle_sample(b, m, n):
    """Oracle results of the sample (the first n DAGs of b), computed once for both sweeps."""
    if "plain" not in _CACHE:
        _CACHE["plain"] = oracle_many(b, range(n), m)
    return _CACHE["plain"]


def _run(b, m, policy=None, tuning=None, scorer=None):
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns, policy)
    if scorer is not None:
        _lib.insp_set_scorer(M.handle, scorer)
    B = P.DagBatch(M, b)
    if tuning:
        B.tuning = dict(B.tuning, **tuning)
    ia, ie, s = B.evaluate()
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    return dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(), start=s.start.cpu().numpy(),
                end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())


@pytest.mark.parametrize("ia_block", [0, 1])
def test_mixed_sample_and_200k_golden_dags(ia_block):
    gold = json.load(open(GOLD))["dags"]
    idx = _sample_indices()
    parts = [inputs.mixed(1, first=i) for i in idx] + [inputs.mixed(1, first=g["index"]) for g in gold.values()]
    b = inputs.concat_batches(parts)
    m = inputs.MACHINE_MIXED
    g = _run(b, m, tuning=dict(ia_block=ia_block))
    compare_many(b, g, m, _oracle_sample(b, m, len(idx)))
    dt = {"ia": "<i4", "ie": "<i4", "worker": "<i4", "start": "<i8", "end": "<i8"}
    for k, (name, want) in enumerate(gold.items()):
        d = len(idx) + k
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        assert te - tb == want["n"]
        for f, t in dt.items():
            got = np.ascontiguousarray(g[f][tb:te], t)
            np.testing.assert_array_equal(got[want["sample_tasks"]], want["sample"][f], err_msg=f"{f} of {name}")
            assert hashlib.sha256(got.tobytes()).hexdigest() == want["sha256"][f], f"{f} of {name}"
        assert int(g["makespan"][d]) == want["makespan"], name


def test_mixed_sample_learned_policy():
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import scorer
    bits, _ = scorer.load_trained()
    k = np.round((bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64) * 64).astype(np.int16)
    idx = _sample_indices(16, cap=12000)
    b = inputs.concat_batches([inputs.mixed(1, first=i) for i in idx])
    m = inputs.MACHINE_MIXED
    pol = P.insp_policy()
    pol.policy = P.INSP_POLICY_LEARNED
    g = _run(b, m, policy=pol, scorer=bits)
    compare_many(b, g, m, oracle_many(b, range(b.ndag), m, "learned", mlp_weights=k))
