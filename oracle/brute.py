"""Brute-force second opinions for tiny DAGs (test infrastructure only).

Pure Python, deliberately different algorithms from ``oracle.c``:
  - inspiring ability by enumerating every path from a task (Sec. 4.2);
  - inspiring efficiency by enumerating every path and taking, for each
    reached task, the heaviest path weight (GPU times, both ends included)
    from the start of the source (Sec. 4.3 with the cone / longest-path
    reading);
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
