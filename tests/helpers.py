"""Shared helpers for the parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
import numpy as np

import inputs
import oracle


def machine_policy(policy_name):
    from paper_2404_03226_b300 import insp_policy
    p = insp_policy()
    p.policy = {"inspirit": 0, "fifo": 1, "dmdap_ia": 3, "dmdap_bl": 4}[policy_name]
    return p


def gpu_run(batch, machine, policy="inspirit", unit_time=None, per_dag=False):
    """Attributes + simulation on the GPU; returns numpy arrays."""
    import torch
    import paper_2404_03226_b300 as P
    m = P.Machine(machine.n_cpu, machine.n_gpu, machine.xfer_ns, machine_policy(policy))
    b = P.DagBatch(m, batch)
    ia, ie = b.attributes(unit_time)
    s = b.simulate(ia, ie, per_dag=per_dag)
    torch.cuda.synchronize()
    st = b.status()
    out = dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(),
               start=s.start.cpu().numpy(), end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy(), status=st)
    return out


def oracle_dag(batch, d, machine, policy="inspirit", unit_time=None):
    g = batch.dag(d)
    pol = oracle.Policy({"inspirit": oracle.POLICY_INSPIRIT, "fifo": oracle.POLICY_FIFO,
                         "dmdap_ia": oracle.POLICY_DMDAP_IA, "dmdap_bl": oracle.POLICY_DMDAP_BL}[policy])
    return g, oracle.simulate(g, machine, pol, unit_time=unit_time)


def compare_dag(batch, d, gpu, machine, policy="inspirit", unit_time=None):
    """Element-by-element equality of DAG d's attributes and schedule."""
    g, r = oracle_dag(batch, d, machine, policy, unit_time)
    tb, te = int(batch.task_base[d]), int(batch.task_base[d + 1])
    assert r["rc"] == 0
    np.testing.assert_array_equal(gpu["ia"][tb:te], r["ia"], err_msg=f"ia of DAG {d}")
    np.testing.assert_array_equal(gpu["ie"][tb:te], r["ie"], err_msg=f"ie of DAG {d}")
    np.testing.assert_array_equal(gpu["worker"][tb:te], r["worker"], err_msg=f"worker of DAG {d}")
    np.testing.assert_array_equal(gpu["start"][tb:te], r["start"], err_msg=f"start of DAG {d}")
    np.testing.assert_array_equal(gpu["end"][tb:te], r["end"], err_msg=f"end of DAG {d}")
    assert int(gpu["makespan"][d]) == r["makespan"], f"makespan of DAG {d}"


def valid(batch, d, gpu, machine):
    g = batch.dag(d)
    tb, te = int(batch.task_base[d]), int(batch.task_base[d + 1])
    return oracle.validate(g, machine, gpu["worker"][tb:te], gpu["start"][tb:te], gpu["end"][tb:te],
                           int(gpu["makespan"][d]))


def edge_case_dags():
    """Small DAGs covering degenerate shapes (all with per-task costs)."""
    rng = np.random.default_rng(77)
    D = []
    D.append(inputs.make_dag(1, [], [5], [3]))                                      # single task
    D.append(inputs.make_dag(33, [], rng.integers(1, 50, 33), rng.integers(1, 50, 33)))  # independent, ragged block
    D.append(inputs.make_dag(40, [(i, i + 1) for i in range(39)], [7] * 40, [3] * 40))     # chain
    star = [(0, v) for v in range(1, 300)]
    D.append(inputs.make_dag(300, star, rng.integers(1, 100, 300), rng.integers(1, 100, 300)))  # wide release
    fan_in = [(u, 299) for u in range(299)]
    D.append(inputs.make_dag(300, fan_in, rng.integers(1, 100, 300), rng.integers(1, 100, 300)))
    full = [(u, v) for u in range(24) for v in range(u + 1, 24)]
    D.append(inputs.make_dag(24, full, rng.integers(1, 30, 24), rng.integers(1, 30, 24)))  # fully connected
    eq = [(u, v) for u in range(60) for v in range(u + 1, min(60, u + 9)) if (u * 7 + v) % 3 == 0]
    D.append(inputs.make_dag(60, eq, [10] * 60, [10] * 60))  # equal costs: many simultaneous events
    return D


def oracle_many(batch, idx, machine, policy="inspirit", unit_time=None, mlp_weights=None, threads=None):
    """Oracle results of the listed DAGs on a thread pool over the host cores
    (the oracle's C calls release the interpreter lock); unit_time is None, an
    int, or a per-DAG array."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    pol = oracle.Policy({"inspirit": oracle.POLICY_INSPIRIT, "fifo": oracle.POLICY_FIFO,
                         "learned": oracle.POLICY_LEARNED, "dmdap_ia": oracle.POLICY_DMDAP_IA,
                         "dmdap_bl": oracle.POLICY_DMDAP_BL}[policy])

    def one(d):
        T = None if unit_time is None else int(np.asarray(unit_time).reshape(-1)[d] if np.ndim(unit_time) else unit_time)
        return oracle.simulate(batch.dag(int(d)), machine, pol, unit_time=T, mlp_weights=mlp_weights)

    with ThreadPoolExecutor(threads or os.cpu_count() or 1) as ex:
        return dict(zip([int(d) for d in idx], ex.map(one, idx)))


def compare_many(batch, gpu, machine, results, with_attributes=True):
    """Element-by-element equality of every DAG in `results` (from oracle_many)."""
    for d, r in results.items():
        tb, te = int(batch.task_base[d]), int(batch.task_base[d + 1])
        assert r["rc"] == 0, f"oracle rc of DAG {d}"
        keys = ("ia", "ie", "worker", "start", "end") if with_attributes else ("worker", "start", "end")
        for k in keys:
            np.testing.assert_array_equal(gpu[k][tb:te], r[k], err_msg=f"{k} of DAG {d}")
        assert int(gpu["makespan"][d]) == r["makespan"], f"makespan of DAG {d}"
