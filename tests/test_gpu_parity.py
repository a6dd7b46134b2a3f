"""Parity of the CUDA path (through the C ABI) with the oracle: bit-exact
inspiring ability / efficiency, worker, start, end and makespan."""
import numpy as np
import pytest

import inputs
import oracle
from helpers import compare_dag, edge_case_dags, gpu_run, valid

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", ["inspirit", "fifo"])
def test_cholesky8(policy):
    b = inputs.cholesky8()
    m = inputs.MACHINE_CHOLESKY8
    g = gpu_run(b, m, policy)
    assert (g["status"] == 0).all()
    compare_dag(b, 0, g, m, policy)


@pytest.mark.parametrize("policy", ["inspirit", "fifo"])
def test_layered_small_sizes(policy):
    """Layered DAGs spanning several 32-source blocks, ragged tails."""
    b = inputs.layered(48, cfg=90, n_min=1, n_max=300)
    m = inputs.MACHINE_LAYERED
    g = gpu_run(b, m, policy)
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, m, policy)


def test_layered_degree_typed():
    """The layered shapes with 16 task types by in/out degree."""
    b = inputs.layered(40, cfg=2, first=100, n_max=900, typing="degree")
    m = inputs.MACHINE_LAYERED
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, m)


@pytest.mark.parametrize("machine", [inputs.Machine(1, 0, 0), inputs.Machine(0, 1, 5), inputs.Machine(3, 2, 7),
                                     inputs.Machine(32, 8, 20000), inputs.Machine(60, 4, 1000)])
def test_edge_case_dags(machine):
    dags = edge_case_dags()
    b = inputs.concat_dags(dags)
    for policy in ("inspirit", "fifo"):
        g = gpu_run(b, machine, policy)
        assert (g["status"] == 0).all()
        for d in range(b.ndag):
            compare_dag(b, d, g, machine, policy)


def test_empty_dags_in_batch():
    dags = [inputs.make_dag(0, [], [], []), inputs.make_dag(3, [(0, 1)], [1, 2, 3], [3, 2, 1]),
            inputs.make_dag(0, [], [], [])]
    b = inputs.concat_dags(dags)
    m = inputs.Machine(2, 1, 4)
    g = gpu_run(b, m)
    assert list(g["makespan"][[0, 2]]) == [0, 0]
    compare_dag(b, 1, g, m)


@pytest.mark.parametrize("kind,N", [(inputs.KIND_CHOLESKY, 16), (inputs.KIND_LU, 8), (inputs.KIND_QR, 8)])
def test_tiled_per_task_costs(kind, N):
    b = inputs.tiled(kind, N, 3, cfg=91)
    m = inputs.MACHINE_TILED
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, m)


def test_explicit_unit_times_narrow_and_wide():
    b = inputs.layered(12, cfg=92, n_min=20, n_max=400)
    m = inputs.MACHINE_LAYERED
    rng = np.random.default_rng(0)
    for T in (rng.integers(1, 200_000, b.ndag), np.full(b.ndag, 3_000_000_000)):
        g = gpu_run(b, m, unit_time=T)
        for d in range(b.ndag):
            compare_dag(b, d, g, m, unit_time=int(T[d]))


@pytest.mark.parametrize("T", [65533, 65534, 65535, 65536])
def test_unit_times_at_the_16_bit_code_boundary(T):
    """The efficiency sweep keeps 16-bit codes when T <= 65534 and 32-bit ones above: path
    weights built to land on T - 1, T and T + 1 on both sides of that switch."""
    rng = np.random.default_rng(T)
    shapes = inputs.layered(10, cfg=94, n_min=40, n_max=300)
    costs = np.array([1, 2, 21844, 21845, 21846, 32766, 32767, 32768, 65533, 65534, 65535, 65536], np.int64)
    dags = []
    for d in range(shapes.ndag):
        g = shapes.dag(d)
        edges = [(u, int(v)) for u in range(g.n) for v in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]]
        cg = rng.choice(costs, g.n)
        dags.append(inputs.make_dag(g.n, edges, cg * 3, cg))
    b = inputs.concat_dags(dags)
    m = inputs.MACHINE_LAYERED
    g = gpu_run(b, m, unit_time=np.full(b.ndag, T))
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, m, unit_time=T)


def test_per_dag_launch_matches_batched():
    b = inputs.layered(16, cfg=93, n_max=600)
    m = inputs.MACHINE_LAYERED
    g1 = gpu_run(b, m)
    g2 = gpu_run(b, m, per_dag=True)
    for k in ("ia", "ie", "worker", "start", "end", "makespan"):
        np.testing.assert_array_equal(g1[k], g2[k])


def test_full_layered_workload_sampled():
    """All 4096 layered DAGs in the batched launch: every schedule valid and
    bounded, a sample (largest, smallest, spread) bit-exact vs the oracle."""
    b = inputs.layered4096()
    m = inputs.MACHINE_LAYERED
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    sizes = b.sizes()
    order = np.argsort(-sizes, kind="stable")
    sample = list(order[:3]) + list(order[-2:]) + list(range(0, b.ndag, 512))
    for d in sample:
        compare_dag(b, int(d), g, m)
    for d in range(0, b.ndag, 7):
        assert valid(b, d, g, m) == (0, -1)
    # repeat: deterministic
    g2 = gpu_run(b, m)
    np.testing.assert_array_equal(g["makespan"], g2["makespan"])
    np.testing.assert_array_equal(g["start"], g2["start"])
    # the benchmark's configuration: autotuned shapes, the pipelined evaluation step
    import torch
    import paper_2404_03226_b300 as P
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    B.autotune()
    ia, ie, s = B.evaluate()
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    for name, got in (("ia", ia), ("ie", ie), ("worker", s.worker), ("start", s.start), ("end", s.end),
                      ("makespan", s.makespan)):
        np.testing.assert_array_equal(got.cpu().numpy(), g[name], err_msg=name)


def test_load_errors():
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    m = P.Machine(2, 1, 10)
    good = inputs.make_dag(3, [(0, 1), (1, 2)], [1, 1, 1], [1, 1, 1])
    cases = []
    dup = inputs.Dag(2, np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32), np.zeros(2, np.uint8),
                     np.ones(2, np.int64), np.ones(2, np.int64))
    cases.append((dup, _lib.INSP_EINVAL))
    zero = inputs.make_dag(3, [(0, 1)], [1, 0, 1], [1, 1, 1])
    cases.append((zero, _lib.INSP_EINVAL))
    oob = inputs.Dag(2, np.array([0, 1, 1], np.int32), np.array([5], np.int32), np.zeros(2, np.uint8),
                     np.ones(2, np.int64), np.ones(2, np.int64))
    cases.append((oob, _lib.INSP_EINVAL))
    huge = inputs.make_dag(2, [], [1 << 53, (1 << 53) + 1], [1, 1])
    cases.append((huge, _lib.INSP_EOVERFLOW))
    for dag, code in cases:
        assert oracle.check_dag(dag, 10) == code  # the oracle agrees on the code
        with pytest.raises(_lib.InspError) as e:
            P.DagBatch(m, inputs.concat_dags([good, dag]))
        assert e.value.code == code
    bad_type = inputs.concat_dags([good])
    bad_type.task_cost = None
    bad_type.type = np.array([0, 3, 0], np.uint8)
    bad_type.type_cost = np.ones((1, 2, 2), np.int64)
    bad_type.n_types = 2
    with pytest.raises(_lib.InspError) as e:
        P.DagBatch(m, bad_type)
    assert e.value.code == _lib.INSP_EINVAL


def test_host_pointer_path_matches_device_path():
    """The C ABI with host arrays (staged by the library) gives the same result."""
    from paper_2404_03226_b300 import _lib
    import paper_2404_03226_b300 as P
    b = inputs.layered(8, cfg=94, n_max=500)
    m = inputs.MACHINE_LAYERED
    g = gpu_run(b, m)
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    B = P.DagBatch(M, b)
    n = b.n_total
    ia = np.zeros(n, np.int32); ie = np.zeros(n, np.int32)
    _lib.insp_attributes_batch(B.handle, None, ia, ie)
    w = np.zeros(n, np.int32); s = np.zeros(n, np.int64); e = np.zeros(n, np.int64); mk = np.zeros(b.ndag, np.int64)
    _lib.insp_simulate_batch(B.handle, ia, ie, w, s, e, mk)
    np.testing.assert_array_equal(ia, g["ia"]); np.testing.assert_array_equal(ie, g["ie"])
    np.testing.assert_array_equal(w, g["worker"]); np.testing.assert_array_equal(mk, g["makespan"])


def test_single_dag_entry_points():
    from paper_2404_03226_b300 import _lib
    import paper_2404_03226_b300 as P
    d = inputs.cholesky8().dag(0)
    m = inputs.MACHINE_CHOLESKY8
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    h = _lib.insp_dag_load_csr(M.handle, d.n, d.row_ptr, d.col_idx, None, 1, None,
                               np.ascontiguousarray(np.stack([d.c_cpu, d.c_gpu], 1)))
    try:
        ia = np.zeros(d.n, np.int32); ie = np.zeros(d.n, np.int32)
        _lib.insp_attributes(h, 0, ia, ie)
        w = np.zeros(d.n, np.int32); s = np.zeros(d.n, np.int64); e = np.zeros(d.n, np.int64)
        mk = np.zeros(1, np.int64)
        _lib.insp_simulate(h, ia, ie, w, s, e, mk)
    finally:
        _lib.insp_dag_destroy(h)
    r = oracle.simulate(d, m)
    np.testing.assert_array_equal(ia, r["ia"]); np.testing.assert_array_equal(ie, r["ie"])
    np.testing.assert_array_equal(w, r["worker"]); np.testing.assert_array_equal(s, r["start"])
    assert int(mk[0]) == r["makespan"]


def test_recorded_graph_replays_match_direct_calls():
    """A recorded evaluation step replayed several times (and interleaved with
    direct calls) reproduces the direct results: the step counters live on the
    device, so replays never reuse a stale done-flag epoch or record tag."""
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    b = inputs.layered(64, cfg=98, n_max=1500)
    m = inputs.MACHINE_LAYERED
    ref = gpu_run(b, m)
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    B = P.DagBatch(M, b)
    n, nd = b.n_total, b.ndag
    dev = torch.device("cuda")
    bufs = dict(ia=torch.empty(n, dtype=torch.int32, device=dev), ie=torch.empty(n, dtype=torch.int32, device=dev),
                worker=torch.empty(n, dtype=torch.int32, device=dev), start=torch.empty(n, dtype=torch.int64, device=dev),
                end=torch.empty(n, dtype=torch.int64, device=dev), makespan=torch.empty(nd, dtype=torch.int64, device=dev))
    s = torch.cuda.Stream()
    _lib.insp_batch_record(B.handle, bufs["ia"], bufs["ie"], bufs["worker"], bufs["start"], bufs["end"],
                           bufs["makespan"], s)
    for rep in range(3):
        for v in bufs.values():
            v.fill_(-1)
        torch.cuda.synchronize()
        _lib.insp_batch_replay(B.handle, s)
        s.synchronize()
        assert _lib.insp_batch_status(B.handle) == 0
        for k, v in bufs.items():
            np.testing.assert_array_equal(v.cpu().numpy(), ref[k], err_msg=f"{k}, replay {rep}")
        if rep == 1:  # a direct step between replays advances the device counters too
            _lib.insp_attributes_batch(B.handle, None, bufs["ia"], bufs["ie"], s)
            s.synchronize()
    with pytest.raises(_lib.InspError):
        _lib.insp_batch_record(B.handle, bufs["ia"], bufs["ie"], bufs["worker"], bufs["start"], bufs["end"],
                               bufs["makespan"], None)


def test_tiled_32_long_spans_take_the_pull_sweep():
    """Cholesky and LU at 32 tiles (edge spans up to ~1000 ids, window 1024)."""
    b = inputs.concat([inputs.tiled(inputs.KIND_CHOLESKY, 32, 1), inputs.tiled(inputs.KIND_LU, 32, 1)])
    m = inputs.MACHINE_TILED
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, m)


def test_tiled_64_cholesky_window_4096():
    """Cholesky at 64 tiles (45,760 tasks, edges spanning up to 2,078 ids: a 4096-row window and
    the sparse efficiency sweep; bitset rows of 715 words; hundreds of ready tasks)."""
    b = inputs.tiled(inputs.KIND_CHOLESKY, 64, 1)
    m = inputs.MACHINE_TILED
    g = gpu_run(b, m)
    assert (g["status"] == 0).all()
    compare_dag(b, 0, g, m)


def _shuffle_batch(batch, seed):
    """Every DAG of the batch under a random relabelling (not topological), and the new ids
    the oracle's renumbering gives each."""
    rng = np.random.default_rng(seed)
    dags, news = [], []
    for d in range(batch.ndag):
        g = batch.dag(d)
        s = oracle.relabel(g, rng.permutation(g.n).astype(np.int32)) if g.n > 1 else g
        dags.append(s)
        rc, new = oracle.renumber(s)
        assert rc == oracle.OK
        news.append(new)
    return dags, news


@pytest.mark.parametrize("host", [False, True])
def test_non_topological_numbering_is_renumbered(host):
    """DAGs given in a shuffled numbering (mixed with ones already topological) are renumbered
    at load by Kahn rounds; every per-task result comes back in the caller's numbering and
    equals the oracle's on the renumbered DAG, mapped back.  Two-call and fused steps, device
    and host outputs (per-task costs, which move with their tasks)."""
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    base = inputs.concat([inputs.layered(10, cfg=48, n_max=900), inputs.tiled(inputs.KIND_LU, 8, 2, cfg=49)])
    sh, news = _shuffle_batch(base, 5)
    keep = [base.dag(0), base.dag(3)]  # already topological: they keep their ids
    dags = sh[:6] + keep + sh[6:]
    news = news[:6] + [np.arange(d.n) for d in keep] + news[6:]
    b = inputs.concat_dags(dags)
    m = inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    n, nd = b.n_total, b.ndag
    refs = [oracle.simulate(oracle.relabel(g, nw), m) for g, nw in zip(dags, news)]

    def check(got, what):
        for d, (r, nw) in enumerate(zip(refs, news)):
            tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
            for k in ("ia", "ie", "worker", "start", "end"):
                np.testing.assert_array_equal(got[k][tb:te], np.asarray(r[k])[nw], err_msg=f"{k} of DAG {d}, {what}")
            assert int(got["makespan"][d]) == r["makespan"], f"makespan of DAG {d}, {what}"

    if host:
        out = dict(ia=np.zeros(n, np.int32), ie=np.zeros(n, np.int32), worker=np.zeros(n, np.int32),
                   start=np.zeros(n, np.int64), end=np.zeros(n, np.int64), makespan=np.zeros(nd, np.int64))
        _lib.insp_evaluate_batch(B.handle, None, *out.values())
        check(out, "fused, host")
        out2 = {k: np.zeros_like(v) for k, v in out.items()}
        _lib.insp_attributes_batch(B.handle, None, out2["ia"], out2["ie"])
        _lib.insp_simulate_batch(B.handle, out2["ia"], out2["ie"], out2["worker"], out2["start"], out2["end"],
                                 out2["makespan"])
        check(out2, "two calls, host")
    else:
        ia, ie, s = B.evaluate()
        torch.cuda.synchronize()
        assert (B.status() == 0).all()
        check(dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(),
                   start=s.start.cpu().numpy(), end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy()), "fused")
        ia, ie = B.attributes()
        s = B.simulate(ia, ie)
        torch.cuda.synchronize()
        check(dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(),
                   start=s.start.cpu().numpy(), end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy()),
              "two calls")
        # bottom levels follow their tasks too
        bl = B.bottom_level().cpu().numpy()
        for d, (g, nw) in enumerate(zip(dags, news)):
            tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
            np.testing.assert_array_equal(bl[tb:te], oracle.bottom_level(oracle.relabel(g, nw), m)[nw])
        with pytest.raises(_lib.InspError):
            B.simulate_trace(ia, ie)


def test_cycles_are_reported():
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    good = inputs.make_dag(3, [(0, 1), (1, 2)], [1, 1, 1], [1, 1, 1])
    cyc = inputs.Dag(3, np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 0], np.int32), np.zeros(3, np.uint8),
                     np.ones(3, np.int64), np.ones(3, np.int64))  # 0 -> 1 -> 2 -> 0
    assert oracle.renumber(cyc)[0] == oracle.ECYCLE
    with pytest.raises(_lib.InspError) as e:
        P.DagBatch(P.Machine(2, 1, 10), inputs.concat_dags([good, cyc]))
    assert e.value.code == _lib.INSP_ECYCLE


def test_renumbered_dags_with_per_type_costs():
    """Shuffled layered DAGs with per-type cost tables: the types move with their tasks."""
    import torch
    import paper_2404_03226_b300 as P
    base = inputs.layered(6, cfg=50, n_max=700)
    sh, news = _shuffle_batch(base, 9)
    nb = inputs.concat_dags(sh)
    b = inputs.Batch(nb.ndag, base.n_types, nb.task_base, nb.edge_base, nb.row_ptr, nb.col_idx, nb.type,
                     base.type_cost, None)
    m = inputs.MACHINE_LAYERED
    B = P.DagBatch(P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns), b)
    ia, ie, s = B.evaluate()
    torch.cuda.synchronize()
    assert (B.status() == 0).all()
    for d in range(b.ndag):
        g = b.dag(d)
        r = oracle.simulate(oracle.relabel(g, news[d]), m)
        tb, te = int(b.task_base[d]), int(b.task_base[d + 1])
        for k, v in (("ia", ia), ("ie", ie), ("worker", s.worker), ("start", s.start), ("end", s.end)):
            np.testing.assert_array_equal(v.cpu().numpy()[tb:te], np.asarray(r[k])[news[d]], err_msg=f"{k} of {d}")


def test_machine_destroyed_before_its_batches():
    """A machine destroyed while batches loaded on it are alive (a garbage collector may finalise
    the handles in either order): the batches stay usable, and the last one frees the machine."""
    import gc
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    b = inputs.layered(6, cfg=90, first=7, n_max=400)
    m = inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    batches = [P.DagBatch(M, b), P.DagBatch(M, b)]
    _lib.insp_machine_destroy(M.handle)
    M.handle = None
    while batches:
        B = batches.pop()
        ia, ie = B.attributes()
        s = B.simulate(ia, ie)
        torch.cuda.synchronize()
        assert (B.status() == 0).all()
        g = dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(),
                 start=s.start.cpu().numpy(), end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())
        for d in range(b.ndag):
            compare_dag(b, d, g, m)
        del B, s  # the first destroy leaves the machine to the second, which frees it
        gc.collect()


def test_concurrent_loads_from_host_threads():
    """Batches of one machine loaded from three host threads at once (each load on its batch's own
    stream, the machine's spare lists shared) while another batch evaluates, as the serving loop
    does: every schedule equals the oracle's."""
    import threading
    from types import SimpleNamespace
    import torch
    import paper_2404_03226_b300 as P
    from paper_2404_03226_b300 import _lib
    b = inputs.layered(24, cfg=90, first=11, n_max=500)
    m = inputs.MACHINE_LAYERED
    M = P.Machine(m.n_cpu, m.n_gpu, m.xfer_ns)
    running = P.DagBatch(M, b)
    ia0, ie0, s0 = running.evaluate(stream=torch.cuda.Stream())  # in flight while the loads run
    handles, errors = [None] * 3, []

    def load(k):
        try:
            handles[k] = _lib.insp_batch_load_csr(M.handle, b.ndag, np.ascontiguousarray(b.task_base, np.int64),
                                                  np.ascontiguousarray(b.edge_base, np.int64),
                                                  np.ascontiguousarray(b.row_ptr, np.int32),
                                                  np.ascontiguousarray(b.col_idx, np.int32),
                                                  np.ascontiguousarray(b.type, np.uint8), b.n_types,
                                                  np.ascontiguousarray(b.type_cost, np.int64), None)
        except Exception as exc:  # reported below
            errors.append(exc)

    threads = [threading.Thread(target=load, args=(k,)) for k in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    results = [(ia0, ie0, s0)]
    for h in handles:
        n = int(b.task_base[-1])
        ia = torch.empty(n, dtype=torch.int32, device="cuda"); ie = torch.empty_like(ia)
        w = torch.empty_like(ia); st = torch.empty(n, dtype=torch.int64, device="cuda"); en = torch.empty_like(st)
        mk = torch.empty(b.ndag, dtype=torch.int64, device="cuda")
        _lib.insp_evaluate_batch(h, None, ia, ie, w, st, en, mk)
        torch.cuda.synchronize()
        assert _lib.insp_batch_status(h) == 0
        results.append((ia, ie, SimpleNamespace(worker=w, start=st, end=en, makespan=mk)))
        _lib.insp_batch_destroy(h)
    for ia, ie, s in results:
        g = dict(ia=ia.cpu().numpy(), ie=ie.cpu().numpy(), worker=s.worker.cpu().numpy(),
                 start=s.start.cpu().numpy(), end=s.end.cpu().numpy(), makespan=s.makespan.cpu().numpy())
        for d in range(b.ndag):
            compare_dag(b, d, g, m)
