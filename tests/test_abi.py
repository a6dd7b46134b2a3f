"""The C-ABI library loads on a machine without a GPU and exports every
entry point that include/inspirit.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "inspirit.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(insp_[a-z_0-9]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("insp_machine_create", "insp_dag_load_csr", "insp_attributes", "insp_simulate",
                 "insp_batch_load_csr", "insp_attributes_batch", "insp_simulate_batch", "insp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2404_03226_b300 import _lib
    L = _lib.lib()
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.so_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (insp_[a-z_0-9]+)", out))
    assert set(_declared()) <= exported
    # the binding wraps every declared entry point under the same name
    assert set(_declared()) <= set(_lib.symbols())


def test_last_error_is_empty_string_initially():
    from paper_2404_03226_b300 import _lib
    assert isinstance(_lib.last_error(), str)


def test_machine_argument_errors_without_gpu():
    from paper_2404_03226_b300 import _lib
    with pytest.raises(_lib.InspError) as e:
        _lib.insp_machine_create(0, 0, 10)
    assert e.value.code == _lib.INSP_EINVAL
    with pytest.raises(_lib.InspError):
        _lib.insp_machine_create(40, 40, 10)
    with pytest.raises(_lib.InspError):
        _lib.insp_machine_create(1, 1, -5)
    h = _lib.insp_machine_create(8, 2, 20000)
    _lib.insp_machine_destroy(h)


def test_binding_constants_match_the_header():
    """Constants the binding copies from include/inspirit.h stay equal to it."""
    from paper_2404_03226_b300 import _lib
    hdr = open(os.path.join(ROOT, "include", "inspirit.h")).read()
    defs = dict(re.findall(r"#define\s+(INSP_[A-Z_0-9]+)\s+(-?\d+)", hdr))
    assert int(defs["INSP_NOALLOC_MAX_TASKS"]) == _lib.INSP_NOALLOC_MAX_TASKS
    for name in ("INSP_OK", "INSP_EINVAL", "INSP_ENOTTOPO", "INSP_ENOMEM", "INSP_ECUDA", "INSP_ETIMEOUT",
                 "INSP_EOVERFLOW", "INSP_POLICY_INSPIRIT", "INSP_POLICY_FIFO", "INSP_POLICY_LEARNED",
                 "INSP_POLICY_DMDAP_IA", "INSP_POLICY_DMDAP_BL"):
        assert int(defs[name]) == getattr(_lib, name), name
    for code, name in _lib.ERROR_NAMES.items():
        assert int(defs[name]) == code, name
    assert re.search(r"#define\s+INSP_SCORE_TIMEOUT\s+INT64_MIN\b", hdr)
    assert _lib.INSP_SCORE_TIMEOUT == -(2 ** 63)


def test_scorer_eval_wrapper_checks_its_tensors():
    """The binding checks dtype, layout and length before taking raw pointers (no GPU needed:
    the checks run before the library is called)."""
    import torch
    from paper_2404_03226_b300 import _lib
    f32 = torch.zeros(4 * 16, dtype=torch.float32)
    i32 = torch.zeros(4 * 16, dtype=torch.int32)
    i64 = torch.zeros(4, dtype=torch.int64)
    with pytest.raises(TypeError):
        _lib.insp_scorer_eval(None, f32, 4, i64)
    with pytest.raises(TypeError):
        _lib.insp_scorer_eval(None, i32, 4, i64.to(torch.int32))
    with pytest.raises(ValueError):
        _lib.insp_scorer_eval(None, i32[: 3 * 16], 4, i64)
    with pytest.raises(ValueError):
        _lib.insp_scorer_eval(None, i32.view(16, 4).t(), 4, i64)
