"""Write mixed_200k.json: the oracle's attributes and schedule of two ~200,000-task DAGs of the
mixed-size stress workload (a random layered one and a tiled one), on 32 CPU + 8 GPU workers
with the default INSPIRIT policy and unit time, as SHA-256 digests of the little-endian arrays
plus every 997th task's values.  Calls only the oracle and the input generators; takes tens of
minutes on one core per DAG (exact inspiring ability by a search from every task).

    python tests/golden/make_mixed_golden.py
"""
import hashlib
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import oracle  # noqa: E402

INDICES = {"layered": 562, "tiled": 19}  # first DAGs of the workload with a drawn size near 200,000
DTYPES = {"ia": "<i4", "ie": "<i4", "worker": "<i4", "start": "<i8", "end": "<i8"}


def digest(a, dt):
    return hashlib.sha256(np.ascontiguousarray(a, dt).tobytes()).hexdigest()


def one(item):
    name, idx = item
    b = inputs.mixed(1, first=idx)
    g = b.dag(0)
    t0 = time.time()
    r = oracle.simulate(g, inputs.MACHINE_MIXED)
    assert r["rc"] == 0
    sample = list(range(0, g.n, 997))
    return name, {"index": idx, "n": int(g.n), "m": int(g.m), "makespan": int(r["makespan"]),
                  "unit_time": int(r["unit_time"]),
                  "sha256": {k: digest(r[k], dt) for k, dt in DTYPES.items()},
                  "sample_tasks": sample, "sample": {k: [int(x) for x in np.asarray(r[k])[sample]] for k in DTYPES},
                  "oracle_seconds": round(time.time() - t0, 1)}


def main():
    with ThreadPoolExecutor(len(INDICES)) as ex:
        res = dict(ex.map(one, INDICES.items()))
    out = {"_what": ("Oracle results for DAGs of inputs.mixed(1, first=index) (the mixed-size stress workload), "
                     "machine 32 CPU + 8 GPU workers, 20 us transfer, INSPIRIT with default parameters and "
                     "the default unit time; written by make_mixed_golden.py from the oracle alone."),
           "dags": res}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mixed_200k.json")
    json.dump(out, open(path, "w"), indent=1)
    print(path)


if __name__ == "__main__":
    main()
