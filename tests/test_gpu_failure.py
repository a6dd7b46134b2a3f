"""Failure detection without a GPU fault: the bounded device-side wait gives up
with INSP_ETIMEOUT on a flag nothing sets, the context stays usable, and a
satisfied wait returns at once."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    import torch
    from paper_2404_03226_b300 import _lib
    with pytest.raises(_lib.InspError) as e:
        _lib.insp_selftest_wait(0, 1, 2000)
    assert e.value.code == 5  # INSP_ETIMEOUT
    _lib.insp_selftest_wait(7, 7, 1)  # already set: no poll needed
    # the context still runs real work afterwards
    from helpers import compare_dag, gpu_run
    b = inputs.layered(4, cfg=33, n_max=200)
    g = gpu_run(b, inputs.MACHINE_LAYERED)
    assert (g["status"] == 0).all()
    for d in range(b.ndag):
        compare_dag(b, d, g, inputs.MACHINE_LAYERED)
    torch.cuda.synchronize()


def test_bounded_wait_rejects_bad_limit():
    from paper_2404_03226_b300 import _lib
    with pytest.raises(_lib.InspError):
        _lib.insp_selftest_wait(0, 0, 0)
