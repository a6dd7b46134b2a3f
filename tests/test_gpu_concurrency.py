"""Batches of one machine loaded on one host thread while another evaluates: the load runs
on its own stream, the machine's recycled buffers are handed out under a lock, and every
evaluation still matches the oracle."""
import queue
import threading

import numpy as np
import pytest

import inputs
import paper_2404_03226_b300 as P
from helpers import compare_dag

pytestmark = pytest.mark.gpu


def test_load_on_one_thread_while_another_evaluates():
    import torch
    m_desc = inputs.MACHINE_LAYERED
    m = P.Machine(m_desc.n_cpu, m_desc.n_gpu, m_desc.xfer_ns)
    batches = [inputs.layered(24, cfg=96 + k, n_min=20, n_max=700) for k in range(6)]
    slots = threading.Semaphore(2)
    q = queue.Queue()

    def loader():
        try:
            for b in batches:
                slots.acquire()
                q.put(P.DagBatch(m, b))
        except Exception as exc:
            q.put(exc)

    th = threading.Thread(target=loader, daemon=True)
    th.start()
    stream = torch.cuda.Stream()
    results = []
    for _ in batches:
        db = q.get()
        if isinstance(db, Exception):
            raise db
        ia, ie, sch = db.evaluate(stream=stream)
        stream.synchronize()
        results.append({"ia": ia.cpu().numpy(), "ie": ie.cpu().numpy(), "worker": sch.worker.cpu().numpy(),
                        "start": sch.start.cpu().numpy(), "end": sch.end.cpu().numpy(),
                        "makespan": sch.makespan.cpu().numpy(), "status": db.status()})
        del db
        slots.release()
    th.join()
    for b, g in zip(batches, results):
        assert (g["status"] == 0).all()
        for d in range(0, b.ndag, 3):
            compare_dag(b, d, g, m_desc)


def test_asynchronous_evaluation_into_pinned_host_memory():
    """insp_evaluate_batch_async returns once the step and its read-back are enqueued: after the
    stream syncs, the pinned host outputs equal the synchronous call's; pageable host outputs are
    refused (INSP_EINVAL) before any work is enqueued."""
    import torch
    from paper_2404_03226_b300 import _lib
    b = inputs.layered(20, cfg=97, n_min=30, n_max=600)
    m_desc = inputs.MACHINE_LAYERED
    m = P.Machine(m_desc.n_cpu, m_desc.n_gpu, m_desc.xfer_ns)
    db = P.DagBatch(m, b)
    ia_ref, ie_ref, sch = db.evaluate()
    torch.cuda.synchronize()
    n, nd = db.n_tasks, db.ndag
    pin = [torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
           torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int64).pin_memory(),
           torch.empty(n, dtype=torch.int64).pin_memory(), torch.empty(nd, dtype=torch.int64).pin_memory()]
    s = torch.cuda.Stream()
    _lib.insp_evaluate_batch_async(db.handle, None, *pin, s)
    s.synchronize()
    assert _lib.insp_batch_status(db.handle) == 0
    for got, ref in zip(pin, (ia_ref, ie_ref, sch.worker, sch.start, sch.end, sch.makespan)):
        np.testing.assert_array_equal(got.numpy(), ref.cpu().numpy())
    pageable = np.zeros(n, np.int32)
    with pytest.raises(P.InspError):
        _lib.insp_evaluate_batch_async(db.handle, None, pin[0], pin[1], pageable, pin[3], pin[4], pin[5], s)
