"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): every
rank takes its own window of DAGs (weak scaling, no data exchange) and the
job's throughput is the sum of tasks over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import inputs
    first = bench.rank_first_dag(rank, per_rank=8)
    b = inputs.layered(8, cfg=2, first=first)
    tasks, t = bench.combine_ranks(float(b.n_total), 1.0 + rank, dist, torch.device("cpu"))
    out[rank] = (first, b.n_total, tasks, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_without_overlap_and_combine():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (f0, n0, s0, t0), (f1, n1, s1, t1) = out[0], out[1]
    assert (f0, f1) == (0, 8)  # disjoint windows of the DAG stream
    assert s0 == s1 == float(n0 + n1)  # whole-job tasks
    assert t0 == t1 == 2.0  # slowest rank's time
    import inputs
    both = inputs.layered(16, cfg=2, first=0)
    assert n0 + n1 == both.n_total  # the two windows tile the 16-DAG prefix
