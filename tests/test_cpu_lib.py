"""CPU-only checks of the C-ABI library: it loads, exports every entry point
include/bwt.h declares, and its host-only routines behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1109_2348_gb300 import _lib, bwt_inverse_check, datagen

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bwt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\*?(bwt_[a-z_]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_four_boundary_calls():
    names = declared_functions()
    for n in ("bwt_plan_create", "bwt_forward_batch", "bwt_inverse_check", "bwt_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_lib.EXPORTS) == names


def test_status_strings():
    lib = _lib.load()
    for code, name in enumerate(_lib.STATUS_NAMES):
        assert lib.bwt_status_string(code).decode() == name


def test_inverse_check_host():
    for src in (datagen.MARKOV3_Z96, datagen.RUNS16, datagen.CONST, datagen.PERIOD7):
        S = datagen.block(src, 5, 3000)
        L, p = oracle.bwt_block(S)
        assert bwt_inverse_check(L, p, S) == _lib.BWT_OK
        bad = L.copy()
        i = int(np.flatnonzero(bad != bad[0])[0]) if np.any(bad != bad[0]) else 0
        bad[0], bad[i] = bad[i], bad[0]
        if not np.array_equal(bad, L):
            assert bwt_inverse_check(bad, p, S) == _lib.BWT_EMISMATCH
    S = np.frombuffer(b"banana", dtype=np.uint8)
    L, p = oracle.bwt_block(S)
    assert bwt_inverse_check(L, 5, S) == _lib.BWT_EMISMATCH or p == 5
    assert bwt_inverse_check(L, -1, S) == _lib.BWT_EINVAL
    assert bwt_inverse_check(L, 6, S) == _lib.BWT_EINVAL
    L2 = L.copy()
    L2[0] = ord("z")
    assert bwt_inverse_check(L2, p, S) == _lib.BWT_EMISMATCH  # not a permutation


def test_plan_create_rejects_bad_descriptors_without_gpu():
    lib = _lib.load()
    h = ctypes.c_void_p()
    for desc in [
        _lib.PlanDesc(0, 100, 100, 0, 0, 0, None),
        _lib.PlanDesc(1, 0, 100, 0, 0, 0, None),
        _lib.PlanDesc(1, 1 << 32, 100, 0, 0, 0, None),
        _lib.PlanDesc(1, 100, 1 << 30, 0, 0, 0, None),
        _lib.PlanDesc(1, 100, 100, 9, 0, 0, None),
        _lib.PlanDesc(1, 100, 100, 8, 1000, 0, None),
    ]:
        assert lib.bwt_plan_create(ctypes.byref(desc), 0, ctypes.byref(h)) == _lib.BWT_EINVAL
        assert not h.value
    assert lib.bwt_plan_destroy(None) == _lib.BWT_OK


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES") is None and os.path.exists("/dev/nvidia0"),
                    reason="a GPU is present")
def test_plan_create_without_gpu_reports_cuda_error():
    lib = _lib.load()
    h = ctypes.c_void_p()
    desc = _lib.PlanDesc(1, 100, 100, 0, 0, 0, None)
    st = lib.bwt_plan_create(ctypes.byref(desc), 0, ctypes.byref(h))
    assert st in (_lib.BWT_ECUDA, _lib.BWT_EINVAL)
    assert not h.value


def test_debug_library_builds_and_exports_every_declared_symbol():
    """The -DBWT_DEBUG build (bounds checks that record BWT_EINTERNAL) compiles
    for sm_103a here and exports the same C ABI."""
    from paper_1109_2348_gb300 import _build
    so = _build.build_bwt(debug=True)
    lib = ctypes.CDLL(str(so))
    for n in declared_functions():
        assert hasattr(lib, n), n
    lib.bwt_status_string.restype = ctypes.c_char_p
    assert lib.bwt_status_string(_lib.BWT_EINTERNAL).decode() == "BWT_EINTERNAL"
