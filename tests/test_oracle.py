"""CPU pins of the oracle against facts that do not come from the oracle itself:
the paper's worked statements, closed forms, brute force by path enumeration,
hand-traced schedules and controller steps, bounds and an exhaustive optimum."""
import json
import os

import numpy as np
import pytest

import inputs
import oracle
from oracle import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_dag(rng, n, p, cmax=50):
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
    return inputs.make_dag(n, edges, rng.integers(1, cmax, n), rng.integers(1, cmax, n))


def _chain(n, c_cpu, c_gpu):
    return inputs.make_dag(n, [(i, i + 1) for i in range(n - 1)], [c_cpu] * n, [c_gpu] * n)


# ------------------------------------------------------------ inspiring ability
def test_ia_paper_statements():
    g = json.load(open(os.path.join(GOLD, "attributes_paper.json")))
    for case in g["cases"]:
        n = case["n"]
        edges = [(u, v) for u in range(n) for v in range(u + 1, n)] if case["edges"] == "complete" else case["edges"]
        d = inputs.make_dag(n, edges, [1] * n, [1] * n)
        ia = oracle.ia(d)
        if "ia" in case:
            assert list(ia) == case["ia"], case["name"]
        if "ia_source" in case:
            assert ia[0] == case["ia_source"]


def test_ia_closed_forms():
    for n in (1, 2, 7, 40):
        assert list(oracle.ia(_chain(n, 3, 1))) == [n - 1 - i for i in range(n)]
    diamond = inputs.make_dag(4, [(0, 1), (0, 2), (1, 3), (2, 3)], [1] * 4, [1] * 4)
    assert list(oracle.ia(diamond)) == [3, 1, 1, 0]  # a path count would give 4 for task 0
    indep = inputs.make_dag(5, [], [1] * 5, [1] * 5)
    assert list(oracle.ia(indep)) == [0] * 5


def test_ia_cholesky8_source():
    d = inputs.cholesky8().dag(0)
    ia = oracle.ia(d)
    assert d.n == 120 and ia[0] == 119  # every task depends on the first POTRF
    assert ia[-1] == 0  # the last POTRF has no successor


@pytest.mark.parametrize("seed", range(12))
def test_ia_matches_path_enumeration(seed):
    rng = np.random.default_rng(seed)
    d = _rand_dag(rng, int(rng.integers(1, 13)), float(rng.uniform(0.1, 0.6)))
    assert list(oracle.ia(d)) == brute.ia(d)


# --------------------------------------------------------- inspiring efficiency
@pytest.mark.parametrize("seed", range(12))
def test_ie_matches_path_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    d = _rand_dag(rng, int(rng.integers(1, 12)), float(rng.uniform(0.1, 0.6)), cmax=20)
    for T in (1, 10, 25, 60, 200):
        assert list(oracle.ie(d, T)) == brute.ie(d, T), T


def test_ie_limits():
    """Too small a unit time gives zero, a large one converges to IA (Sec. 4.2)."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        d = _rand_dag(rng, 30, 0.15)
        big = int(d.c_gpu.sum())
        assert list(oracle.ie(d, big)) == list(oracle.ia(d))
        # every counted task finishes after at least two executions (v and itself)
        assert not oracle.ie(d, int(d.c_gpu.min())).any()


def test_ie_chain_closed_form():
    for n, c, T in [(10, 5, 23), (10, 5, 5), (10, 5, 50), (12, 7, 1000), (6, 3, 2)]:
        ie = oracle.ie(_chain(n, 100, c), T)
        assert list(ie) == [max(0, min(n - 1 - i, T // c - 1)) for i in range(n)]


def test_ie_uses_longest_path():
    # 0 -> 1 -> 2 and 0 -> 2: task 2 is reached at 2 over the short path but
    # only at 12 over the long one; it fits in T=5 only under a shortest-path
    # reading, so its inspiring efficiency count from task 0 is 0.
    d = inputs.make_dag(3, [(0, 1), (0, 2), (1, 2)], [1, 1, 1], [1, 10, 1])
    assert list(oracle.ie(d, 5)) == [0, 0, 0]
    assert list(oracle.ie(d, 12)) == [2, 1, 0]


def test_default_unit_time():
    d = inputs.make_dag(4, [], [1] * 4, [3, 1, 2, 5])
    assert oracle.default_unit_time(d) == 8  # 4 x lower median (2)
    d = inputs.make_dag(3, [], [1] * 3, [9, 1, 4])
    assert oracle.default_unit_time(d) == 16


# ------------------------------------------------------------- the controller
def test_controller_hand_traced():
    g = json.load(open(os.path.join(GOLD, "controller_hand_traced.json")))
    for seqn in g["sequences"]:
        pol = oracle.Policy(0, **seqn["policy"])
        st = oracle.Ctrl(0, 0, 0, 0, oracle.MODE_FIFO, oracle.STATE_INC)
        for k, step in enumerate(seqn["steps"]):
            oracle.ctrl_step(st, pol, step["cur"], step["now"])
            got = dict(mode=st.mode, peak=st.peak, count=st.count, prev_n=st.prev_n, prev_t=st.prev_t)
            exp = {key: step[key] for key in got}
            assert got == exp, (k, step["_why"])


def test_policy_defaults():
    p = oracle.resolve_policy(oracle.Policy(), 10, 12345)
    assert (p.task_window, p.s_inc, p.s_dec, p.dec_step, p.c, p.k_inc_tasks, p.k_inc_ns) == (10, 10, 10, 10, 5, 10, 12345)
    p = oracle.resolve_policy(oracle.Policy(0, 3, 0, 0, 0, 0, 0, 0), 1, 7)
    assert (p.task_window, p.c, p.k_inc_tasks) == (3, 1, 1)


# ------------------------------------------------------------- the simulation
def _policy(name):
    return oracle.Policy({"inspirit": oracle.POLICY_INSPIRIT, "fifo": oracle.POLICY_FIFO,
                          "dmdap_ia": oracle.POLICY_DMDAP_IA, "dmdap_bl": oracle.POLICY_DMDAP_BL}[name])


def test_simulation_hand_traced():
    g = json.load(open(os.path.join(GOLD, "sim_hand_traced.json")))
    for case in g["cases"]:
        d = inputs.make_dag(case["n"], case["edges"], case["c_cpu"], case["c_gpu"])
        m = inputs.Machine(*case["machine"])
        for pname in case["policies"]:
            pol = _policy(pname)
            for k, v in case.get("policy_params", {}).items():
                setattr(pol, k, v)
            r = oracle.simulate(d, m, pol, unit_time=case.get("unit_time"), trace=True)
            assert r["rc"] == 0
            assert list(r["worker"]) == case["worker"], (case["name"], pname)
            assert list(r["start"]) == case["start"], (case["name"], pname)
            assert list(r["end"]) == case["end"], (case["name"], pname)
            assert r["makespan"] == case["makespan"]
            if "order" in case:
                assert list(r["trace"]["task"]) == case["order"]
            if "modes" in case:
                assert list(r["trace"]["mode"]) == case["modes"]


@pytest.mark.parametrize("policy", ["inspirit", "fifo"])
def test_one_worker_sums(policy):
    """A chain, or independent tasks, on one worker: makespan = sum of costs."""
    rng = np.random.default_rng(3)
    for n in (1, 5, 33):
        costs = rng.integers(1, 1000, n)
        chain = inputs.make_dag(n, [(i, i + 1) for i in range(n - 1)], costs, costs)
        indep = inputs.make_dag(n, [], costs, costs)
        for d in (chain, indep):
            for m in (inputs.Machine(1, 0, 77), inputs.Machine(0, 1, 77)):
                assert oracle.simulate(d, m, _policy(policy))["makespan"] == int(costs.sum())


def test_chain_on_one_kind():
    """A chain where the GPU is always faster stays on the GPU: makespan = sum of GPU costs."""
    n = 17
    d = _chain(n, 100, 7)
    r = oracle.simulate(d, inputs.Machine(4, 1, 1000), _policy("inspirit"))
    assert r["makespan"] == 7 * n and set(r["worker"]) == {4}


@pytest.mark.parametrize("P,n,c", [(3, 10, 7), (4, 4, 5), (5, 23, 11), (8, 1, 3)])
def test_identical_workers_independent_tasks(P, n, c):
    d = inputs.make_dag(n, [], [c] * n, [c] * n)
    for pol in ("fifo", "inspirit"):
        assert oracle.simulate(d, inputs.Machine(P, 0, 0), _policy(pol))["makespan"] == -(-n // P) * c


def _lower_bound(d, m):
    cmin = np.minimum(d.c_cpu, d.c_gpu) if m.n_gpu and m.n_cpu else (d.c_cpu if m.n_cpu else d.c_gpu)
    cp = np.zeros(d.n, np.int64)
    for u in range(d.n - 1, -1, -1):
        succ = d.col_idx[d.row_ptr[u]:d.row_ptr[u + 1]]
        cp[u] = cmin[u] + (cp[succ].max() if len(succ) else 0)
    return max(int(cp.max()) if d.n else 0, -(-int(cmin.sum()) // m.n_workers))


@pytest.mark.parametrize("seed", range(10))
def test_random_schedules_valid_and_bounded(seed):
    rng = np.random.default_rng(1000 + seed)
    d = _rand_dag(rng, int(rng.integers(2, 60)), float(rng.uniform(0.02, 0.3)), cmax=100)
    m = inputs.Machine(int(rng.integers(1, 4)), int(rng.integers(0, 3)), int(rng.integers(0, 40)))
    for pol in ("inspirit", "fifo"):
        r = oracle.simulate(d, m, _policy(pol))
        assert r["rc"] == 0
        assert oracle.validate(d, m, r["worker"], r["start"], r["end"], r["makespan"]) == (0, -1)
        assert r["makespan"] >= _lower_bound(d, m)


@pytest.mark.parametrize("seed", range(12))
def test_exhaustive_optimum(seed):
    """makespan >= exact optimum >= lower bound on DAGs of 2 to 10 tasks (seeds 8-11: 9 or 10 tasks)."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 9)) if seed < 8 else int(rng.integers(9, 11))
    d = _rand_dag(rng, n, 0.3, cmax=30)
    m = inputs.Machine(int(rng.integers(1, 3)), 1, int(rng.integers(0, 10)))
    best = oracle.optimum(d, m)
    assert best >= _lower_bound(d, m)
    for pol in ("inspirit", "fifo", "dmdap_ia", "dmdap_bl"):
        assert oracle.simulate(d, m, _policy(pol))["makespan"] >= best


@pytest.mark.parametrize("seed", range(6))
def test_optimum_matches_listing_every_schedule(seed):
    """The branch and bound equals a plain listing of every assignment and topological order (<= 6 tasks)."""
    rng = np.random.default_rng(2100 + seed)
    d = _rand_dag(rng, int(rng.integers(2, 7)), 0.35, cmax=20)
    m = inputs.Machine(int(rng.integers(1, 3)), int(rng.integers(0, 2)), int(rng.integers(0, 12)))
    assert oracle.optimum(d, m) == brute.optimum(d, m)


def test_optimum_known_cases():
    # two independent tasks of 5 on two workers: 5; a chain of three 2-ns tasks
    # across CPU/GPU with a 100 ns transfer: stays on one worker, 6
    assert oracle.optimum(inputs.make_dag(2, [], [5, 5], [5, 5]), inputs.Machine(1, 1, 0)) == 5
    assert oracle.optimum(_chain(3, 2, 2), inputs.Machine(1, 1, 100)) == 6
    assert oracle.optimum(_chain(3, 9, 2), inputs.Machine(1, 1, 100)) == 6


def test_validator_catches_planted_errors():
    d = inputs.make_dag(3, [(0, 1), (1, 2)], [4, 4, 4], [2, 2, 2])
    m = inputs.Machine(1, 1, 10)
    r = oracle.simulate(d, m, _policy("fifo"))
    w, s, e = r["worker"].copy(), r["start"].copy(), r["end"].copy()
    assert oracle.validate(d, m, w, s, e, r["makespan"])[0] == 0
    s2, e2 = s.copy(), e.copy()
    s2[2] -= 1; e2[2] -= 1
    assert oracle.validate(d, m, w, s2, e2, r["makespan"] - 1)[0] == 3
    w2 = w.copy(); w2[1] = 0
    assert oracle.validate(d, m, w2, s, e, r["makespan"])[0] == 2
    assert oracle.validate(d, m, w, s, e, r["makespan"] + 1)[0] == 5


def test_cholesky8_bounds_and_validity():
    d = inputs.cholesky8().dag(0)
    m = inputs.MACHINE_CHOLESKY8
    for pol in ("inspirit", "fifo"):
        r = oracle.simulate(d, m, _policy(pol))
        assert oracle.validate(d, m, r["worker"], r["start"], r["end"], r["makespan"]) == (0, -1)
        assert r["makespan"] >= 2_040_000  # critical path at the fastest cost: 2040 us
    assert _lower_bound(d, m) == 2_040_000


def test_check_dag_errors():
    good = inputs.make_dag(3, [(0, 1), (1, 2)], [1, 1, 1], [1, 1, 1])
    assert oracle.check_dag(good) == oracle.OK
    bad = inputs.make_dag(3, [(0, 1)], [1, 0, 1], [1, 1, 1])
    assert oracle.check_dag(bad) == oracle.EINVAL
    back = inputs.Dag(2, np.array([0, 0, 1], np.int32), np.array([0], np.int32), np.zeros(2, np.uint8),
                      np.ones(2, np.int64), np.ones(2, np.int64))
    assert oracle.check_dag(back) == oracle.ENOTTOPO
    dup = inputs.Dag(2, np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32), np.zeros(2, np.uint8),
                     np.ones(2, np.int64), np.ones(2, np.int64))
    assert oracle.check_dag(dup) == oracle.EINVAL
    huge = inputs.make_dag(2, [], [1 << 53, (1 << 53) + 1], [1, 1])
    assert oracle.check_dag(huge) == oracle.EOVERFLOW


# ----------------------------------------------------------------- the scorer
def test_mlp_score_closed_form():
    nw = oracle.mlp_nweights()
    assert nw == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    w = np.zeros(nw, np.int16)
    assert oracle.mlp_score(w, np.zeros(16, np.int32)) == 0
    # one path: W1[0][0] = 64 (1.0), W2[0][0] = 64, W3[0] = 128 (2.0), b3 = 5
    W1 = 0; b1 = 16 * 64; W2 = b1 + 64; b2 = W2 + 64 * 64; W3 = b2 + 64; b3 = W3 + 64
    w[W1 + 0] = 64; w[W2 + 0] = 64; w[W3 + 0] = 128; w[b3] = 5
    f = np.zeros(16, np.int32); f[0] = 7
    assert oracle.mlp_score(w, f) == 128 * 7 + 5
    f[0] = 200; w[W1 + 0] = 128  # hidden 400 clamps at 255, then 255
    assert oracle.mlp_score(w, f) == 128 * 255 + 5
    w[b1 + 0] = -100 * 64  # negative pre-activation: relu gives 0
    assert oracle.mlp_score(w, f) == 128 * 255 + 5 - 0 if 400 - 100 >= 255 else True
    w[W1 + 0] = 1; w[b1 + 0] = -63  # (200 - 63) / 64 = 2.14 -> floor 2
    assert oracle.mlp_score(w, f) == 128 * 2 + 5


def test_mlp_score_matches_float_network():
    """The integer restatement equals an fp64 evaluation of the same network."""
    rng = np.random.default_rng(5)
    nw = oracle.mlp_nweights()
    for _ in range(20):
        k = rng.integers(-128, 129, nw).astype(np.int16)
        f = rng.integers(0, 256, 16)
        W1 = k[:1024].reshape(16, 64) / 64.0; b1 = k[1024:1088] / 64.0
        W2 = k[1088:5184].reshape(64, 64) / 64.0; b2 = k[5184:5248] / 64.0
        W3 = k[5248:5312] / 64.0; b3 = k[5312] / 64.0
        h1 = np.clip(np.floor(np.maximum(f @ W1 + b1, 0)), 0, 255)
        h2 = np.clip(np.floor(np.maximum(h1 @ W2 + b2, 0)), 0, 255)
        assert oracle.mlp_score(k, f) == int(round((h2 @ W3 + b3) * 64))


# ---------------------------------------------- DMDAP baselines and the trace
@pytest.mark.parametrize("seed", range(6))
def test_bottom_level_matches_path_enumeration(seed):
    rng = np.random.default_rng(3000 + seed)
    d = _rand_dag(rng, int(rng.integers(1, 14)), float(rng.uniform(0.1, 0.5)), cmax=1000)
    for m in (inputs.Machine(1, 0, 0), inputs.Machine(4, 1, 777), inputs.Machine(8, 2, 20000),
              inputs.Machine(0, 3, 5), inputs.Machine(3, 3, 1)):
        np.testing.assert_array_equal(oracle.bottom_level(d, m), brute.bottom_level(d, m))


def test_bottom_level_closed_forms():
    """A chain of n equal tasks: rank(i) = (n - i) * wbar + (n - 1 - i) * cbar; with
    8 CPUs + 2 GPUs, 34 of the 100 ordered worker pairs sit on distinct nodes."""
    n = 9
    d = _chain(n, 300, 40)
    m = inputs.Machine(8, 2, 1000)
    wbar, cbar = (8 * 300 + 2 * 40) // 10, 1000 * 34 // 100
    np.testing.assert_array_equal(oracle.bottom_level(d, m), [(n - i) * wbar + (n - 1 - i) * cbar for i in range(n)])
    # one worker: no transfer between distinct nodes, wbar = the CPU cost
    np.testing.assert_array_equal(oracle.bottom_level(d, inputs.Machine(1, 0, 5)), [(n - i) * 300 for i in range(n)])


@pytest.mark.parametrize("policy", ["dmdap_ia", "dmdap_bl"])
def test_dmdap_one_worker_sums_and_validity(policy):
    rng = np.random.default_rng(11)
    costs = rng.integers(1, 1000, 20)
    indep = inputs.make_dag(20, [], costs, costs)
    assert oracle.simulate(indep, inputs.Machine(1, 0, 5), _policy(policy))["makespan"] == int(costs.sum())
    for seed in range(6):
        r2 = np.random.default_rng(4000 + seed)
        d = _rand_dag(r2, int(r2.integers(2, 50)), float(r2.uniform(0.03, 0.3)), cmax=100)
        m = inputs.Machine(int(r2.integers(1, 4)), int(r2.integers(0, 3)), int(r2.integers(0, 40)))
        r = oracle.simulate(d, m, _policy(policy), trace=True)
        assert r["rc"] == 0
        assert oracle.validate(d, m, r["worker"], r["start"], r["end"], r["makespan"]) == (0, -1)
        assert r["makespan"] >= _lower_bound(d, m)
        assert set(r["trace"]["mode"]) == {oracle.MODE_ABILITY if policy == "dmdap_ia" else oracle.MODE_PRIO}


@pytest.mark.parametrize("policy", ["inspirit", "fifo", "dmdap_bl"])
def test_push_pop_trace_consistent(policy):
    """The push/pop trace (Nready time piling): every task is pushed once and
    popped once, on the worker it was pushed to; pushes at an event time come
    before that time's pops, so Nready after the k-th push is k + 1 minus the
    pops at earlier times, and Nready before a pop is the pushes up to its time
    minus the earlier pops; times never decrease."""
    rng = np.random.default_rng(21)
    for _ in range(5):
        d = _rand_dag(rng, int(rng.integers(5, 70)), float(rng.uniform(0.03, 0.25)), cmax=60)
        m = inputs.Machine(int(rng.integers(1, 5)), int(rng.integers(0, 3)), int(rng.integers(0, 30)))
        r = oracle.simulate(d, m, _policy(policy), trace=True)
        tr = r["trace"]
        n = d.n
        assert len(tr["push_task"]) == n and len(tr["task"]) == n
        assert sorted(tr["push_task"]) == list(range(n)) and sorted(tr["task"]) == list(range(n))
        np.testing.assert_array_equal(tr["push_worker"], r["worker"][tr["push_task"]])
        np.testing.assert_array_equal(tr["worker"], r["worker"][tr["task"]])
        assert (np.diff(tr["push_t"]) >= 0).all() and (np.diff(tr["t"]) >= 0).all()
        for k in range(n):
            pops_before = int((tr["t"] < tr["push_t"][k]).sum())
            assert tr["push_nready"][k] == k + 1 - pops_before
        for j in range(n):
            pushes = int((tr["push_t"] <= tr["t"][j]).sum())
            assert tr["nready"][j] == pushes - j
        # a task is popped no earlier than it was pushed
        pushed_at = dict(zip(tr["push_task"], tr["push_t"]))
        assert all(t >= pushed_at[x] for x, t in zip(tr["task"], tr["t"]))


# ------------------------------------------------------- unit-time search
@pytest.mark.parametrize("n", [1, 2, 5, 8, 9, 33])
def test_unit_time_search_chain_closed_form(n):
    """Chain of n tasks of GPU cost c: IA and the layers take n distinct values,
    and IE at T = c 2^k takes min(n, 2^k) values, so the search stops at the
    first k with 2^k >= n."""
    c = 7
    d = _chain(n, 50, c)
    k = int(np.ceil(np.log2(n))) if n > 1 else 0
    assert oracle.unit_time_search(d, 16) == (c << k, k)
    if k > 1:  # a cap below the answer returns the last candidate
        assert oracle.unit_time_search(d, k - 1) == (c << (k - 1), k - 1)


def test_unit_time_search_special_cases():
    # independent tasks: IA is all 0 (one value), so the first candidate (the lower median) suffices
    d = inputs.make_dag(6, [], [9] * 6, [5, 1, 8, 3, 3, 20])
    assert oracle.unit_time_search(d) == (3, 0)
    # empty DAG
    assert oracle.unit_time_search(inputs.make_dag(0, [], [], [])) == (1, 0)


@pytest.mark.parametrize("seed", range(6))
def test_unit_time_search_matches_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(2, 12))
    d = _rand_dag(rng, n, float(rng.uniform(0.15, 0.5)), cmax=40)
    d = inputs.make_dag(n, [(u, int(v)) for u in range(n) for v in d.col_idx[d.row_ptr[u]:d.row_ptr[u + 1]]],
                        d.c_cpu, d.c_gpu, type=rng.integers(0, 3, n))
    med = int(np.sort(d.c_gpu)[(n - 1) // 2])
    lay = brute.layers(d)
    target = min(len({(lay[i], int(d.type[i])) for i in range(n)}), len(set(brute.ia(d))))
    want = None
    for k in range(12):
        if len(set(brute.ie(d, med << k))) >= target:
            want = (med << k, k)
            break
    assert want is not None
    assert oracle.unit_time_search(d, 11) == want


# ----------------------------------------------------------------- renumbering
def _shuffled(d, rng):
    """The same DAG under a random relabelling (rows re-sorted): usually not topological."""
    perm = rng.permutation(d.n).astype(np.int32)
    return oracle.relabel(d, perm)


def test_renumber_hand_example_and_topological_identity():
    # old edges 2->0, 2->3, 0->1, 3->1: round 0 {2}, round 1 {0, 3}, round 2 {1}
    d = inputs.make_dag(4, [], [1] * 4, [1] * 4)
    d = inputs.Dag(4, np.array([0, 1, 1, 3, 4], np.int32), np.array([1, 0, 3, 1], np.int32), np.zeros(4, np.uint8),
                   np.ones(4, np.int64), np.ones(4, np.int64))
    rc, new = oracle.renumber(d)
    assert rc == oracle.OK and list(new) == [1, 3, 0, 2]
    # ids already topological stay as they are (even where Kahn rounds would reorder: 0->1, 2 isolated)
    chain = inputs.make_dag(3, [(0, 1)], [1] * 3, [1] * 3)
    assert list(oracle.renumber(chain)[1]) == [0, 1, 2]


@pytest.mark.parametrize("seed", range(8))
def test_renumber_is_kahn_rounds_by_path_enumeration(seed):
    """On shuffled random DAGs: a permutation, a topological order, and sorted by (round, old id)
    where the round is the most edges on a path from a source (enumerated by brute force)."""
    rng = np.random.default_rng(3000 + seed)
    d = _shuffled(_rand_dag(rng, int(rng.integers(2, 25)), 0.25), rng)
    rc, new = oracle.renumber(d)
    assert rc == oracle.OK
    assert sorted(new) == list(range(d.n))
    for u in range(d.n):
        for v in d.col_idx[d.row_ptr[u]:d.row_ptr[u + 1]]:
            assert new[u] < new[v]
    layer = brute.layers(d)
    order = sorted(range(d.n), key=lambda t: (layer[t], t))
    assert [int(new[t]) for t in order] == list(range(d.n))


def test_renumber_reports_cycles_and_bad_rows():
    two = inputs.Dag(2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.zeros(2, np.uint8),
                     np.ones(2, np.int64), np.ones(2, np.int64))
    self_loop = inputs.Dag(2, np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.zeros(2, np.uint8),
                           np.ones(2, np.int64), np.ones(2, np.int64))
    deep = inputs.Dag(5, np.array([0, 1, 2, 3, 4, 4], np.int32), np.array([1, 2, 3, 1], np.int32),
                      np.zeros(5, np.uint8), np.ones(5, np.int64), np.ones(5, np.int64))  # 1 -> 2 -> 3 -> 1
    for d in (two, self_loop, deep):
        assert oracle.renumber(d)[0] == oracle.ECYCLE
    dup = inputs.Dag(2, np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32), np.zeros(2, np.uint8),
                     np.ones(2, np.int64), np.ones(2, np.int64))
    assert oracle.renumber(dup)[0] == oracle.EINVAL


def test_relabel_keeps_attributes_and_schedule_validity():
    """A relabelled DAG is the same DAG: IA and IE follow their tasks (closed under the
    relabelling), and the renumbered DAG's schedule mapped back is valid for the original."""
    rng = np.random.default_rng(7)
    d = _rand_dag(rng, 40, 0.15)
    s = _shuffled(d, rng)
    rc, new = oracle.renumber(s)
    assert rc == oracle.OK
    r = oracle.relabel(s, new)
    m = inputs.Machine(2, 1, 5)
    res = oracle.simulate(r, m)
    back = {k: np.asarray(res[k])[new] for k in ("worker", "start", "end", "ia")}
    assert oracle.validate(s, m, back["worker"], back["start"], back["end"], res["makespan"]) == (0, -1)
    assert list(back["ia"]) == brute.ia(s)
