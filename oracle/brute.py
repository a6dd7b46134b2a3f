"""Brute-force second opinions for tiny DAGs (test infrastructure only).

Pure Python, deliberately different algorithms from ``oracle.c``:
  - inspiring ability by enumerating every path from a task (Sec. 4.2);
  - inspiring efficiency by enumerating every path and taking, for each
    reached task, the heaviest path weight (GPU times, both ends included)
    from the start of the source (Sec. 4.3 with the cone / longest-path
    reading);
  - the bottom level of the DMDAP baseline by enumerating every path to a
    sink, with the worker and pair means taken by listing workers and pairs;
Exponential in the worst case: only for DAGs of a few dozen tasks.
"""
from __future__ import annotations


def _succ(dag):
    return [list(dag.col_idx[dag.row_ptr[u]:dag.row_ptr[u + 1]]) for u in range(dag.n)]


def all_paths_from(dag, v):
    """Every path that starts at v, as a list of task lists (v included)."""
    succ = _succ(dag)
    out = []

    def rec(path):
        out.append(list(path))
        for s in succ[path[-1]]:
            path.append(int(s))
            rec(path)
            path.pop()

    rec([v])
    return out


def ia(dag):
    res = []
    for v in range(dag.n):
        ends = {p[-1] for p in all_paths_from(dag, v) if len(p) > 1}
        res.append(len(ends))
    return res


def ie(dag, T):
    res = []
    for v in range(dag.n):
        heaviest = {}
        for p in all_paths_from(dag, v):
            if len(p) == 1:
                continue
            w = sum(int(dag.c_gpu[x]) for x in p)
            u = p[-1]
            heaviest[u] = max(heaviest.get(u, w), w)
        res.append(sum(1 for u, w in heaviest.items() if w <= T))
    return res


def bottom_level(dag, machine):
    """HEFT upward rank by path enumeration: for each task, the heaviest path to
    a sink, weighing every task by its mean cost over the workers and every
    edge by the mean transfer cost over ordered worker pairs (both floored),
    the means taken by listing the workers and the pairs one by one."""
    workers = [0] * machine.n_cpu + [1] * machine.n_gpu  # kind of each worker
    P = len(workers)
    node = [0 if k == 0 else 1 + i for i, k in enumerate(workers)]  # CPUs share node 0
    distinct = sum(1 for a in range(P) for b in range(P) if node[a] != node[b])
    cbar = machine.xfer_ns * distinct // (P * P)

    def wbar(x):
        return sum(int(dag.c_cpu[x]) if k == 0 else int(dag.c_gpu[x]) for k in workers) // P

    succ = _succ(dag)
    res = []
    for v in range(dag.n):
        best = 0
        for p in all_paths_from(dag, v):
            if succ[p[-1]]:
                continue  # only paths that end at a sink
            best = max(best, sum(wbar(x) for x in p) + (len(p) - 1) * cbar)
        res.append(best)
    return res


def layers(dag):
    """Topological layer of every task: the most edges on any path from a
    source to it, by enumerating all paths from every source."""
    preds = [0] * dag.n
    for u in range(dag.n):
        for s in dag.col_idx[dag.row_ptr[u]:dag.row_ptr[u + 1]]:
            preds[int(s)] += 1
    best = [0] * dag.n
    for v in range(dag.n):
        if preds[v]:
            continue
        for p in all_paths_from(dag, v):
            best[p[-1]] = max(best[p[-1]], len(p) - 1)
    return best


def optimum(dag, machine):
    """Minimum makespan by listing every assignment of tasks to workers and
    every topological order: tasks are placed one by one in that order, each
    at the earliest time its worker is free and its data (with the transfer
    cost between memory nodes: CPUs share node 0, GPU g is node 1+g) has
    arrived.  Every schedule can be shifted left into one of these without a
    later end, so the minimum over them is the optimum.  Tiny DAGs only."""
    import itertools
    n, P = dag.n, machine.n_cpu + machine.n_gpu
    succ = _succ(dag)
    preds = [[u for u in range(n) if v in succ[u]] for v in range(n)]
    node = [0 if w < machine.n_cpu else 1 + w - machine.n_cpu for w in range(P)]

    def orders():
        def rec(done, seq):
            if len(seq) == n:
                yield list(seq)
                return
            for t in range(n):
                if t not in done and all(p in done for p in preds[t]):
                    done.add(t)
                    seq.append(t)
                    yield from rec(done, seq)
                    seq.pop()
                    done.remove(t)
        yield from rec(set(), [])

    topo = list(orders())
    best = None
    for assign in itertools.product(range(P), repeat=n):
        for order in topo:
            free = [0] * P
            end = [0] * n
            for t in order:
                w = assign[t]
                ready = max([end[p] + (machine.xfer_ns if node[assign[p]] != node[w] else 0) for p in preds[t]],
                            default=0)
                s = max(free[w], ready)
                end[t] = s + int(dag.c_cpu[t] if w < machine.n_cpu else dag.c_gpu[t])
                free[w] = end[t]
            mk = max(end) if n else 0
            best = mk if best is None else min(best, mk)
    return best or 0
