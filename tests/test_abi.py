"""The C-ABI library builds, loads and exports every entry point that
include/epr.h declares.  CPU only: no call here touches a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "epr.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_22793_gb300 import build as B
    try:
        B._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("epr_plan_create", "epr_plan_destroy", "epr_forward", "epr_adjoint",
              "epr_precondition", "epr_solve_nonlocal", "epr_solve_local",
              "epr_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    from paper_2601_22793_gb300 import epr
    assert sorted(epr.SYMBOLS) == _declared()
    for n in _declared():
        assert callable(getattr(epr, n))


def test_status_strings_without_a_device(lib):
    lib.epr_status_string.restype = ctypes.c_char_p
    lib.epr_status_string.argtypes = [ctypes.c_int]
    for s in range(9):
        assert lib.epr_status_string(s)
    assert lib.epr_status_string(99) == b"unknown status"
    lib.epr_launch_count.restype = ctypes.c_longlong
    assert lib.epr_launch_count() >= 0


def test_plan_rejects_bad_sizes_before_touching_cuda(lib):
    from paper_2601_22793_gb300 import epr
    epr.load(os.path.join(ROOT, "paper_2601_22793_gb300", "libepr.so"))
    for nx, ny in ((100, 64), (64, 4), (8192, 64), (12, 64), (64, 20)):
        with pytest.raises(epr.EprError) as e:
            epr.epr_plan_create(nx, ny, 1e-5, 1.0, [60.0], [1e-7], [1e-10])
        assert e.value.status == epr.EPR_ERR_UNSUPPORTED_SIZE
    with pytest.raises(epr.EprError) as e:
        epr.epr_plan_create(64, 64, -1.0, 1.0, [60.0], [1e-7], [1e-10])
    assert e.value.status == epr.EPR_ERR_INVALID_ARG
    with pytest.raises(epr.EprError) as e:
        epr.epr_plan_create(64, 64, 1e-5, 1.0, [60.0], [1e-7], [1e-10], weights=[0.0])
    assert e.value.status == epr.EPR_ERR_INVALID_ARG
