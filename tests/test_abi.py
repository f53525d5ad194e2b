"""The C-ABI library builds, loads and exports every entry point that
``include/fslbm.h`` declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fslbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fslbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_north_star_calls():
    names = _declared()
    for n in ("fslbm_create", "fslbm_init", "fslbm_step", "fslbm_observables", "fslbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2207_13962_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2207_13962_gb300 import fslbm
    assert sorted(fslbm.SYMBOLS) == _declared()
    lib.fslbm_version.restype = ctypes.c_char_p
    assert lib.fslbm_version().startswith(b"fslbm-gb300")


def test_params_default_and_invalid_create_need_no_gpu():
    from paper_2207_13962_gb300 import fslbm
    lib = fslbm.load()
    p = fslbm.fslbm_params()
    lib.fslbm_params_default(ctypes.byref(p))
    assert p.trt_magic == pytest.approx(3.0 / 16.0) and p.eps_phi == pytest.approx(1e-2)
    assert p.p_v0 == pytest.approx(1.0 / 3.0) and p.precision == 1
    dom = fslbm.fslbm_domain(0, 4, 4, (ctypes.c_int * 3)(0, 0, 0))
    h = ctypes.c_void_p()
    # rejected by argument validation before any CUDA call
    assert lib.fslbm_create(ctypes.byref(dom), 19, 1, 3, ctypes.byref(p), ctypes.byref(h)) == fslbm.EINVAL
    dom = fslbm.fslbm_domain(4, 4, 4, (ctypes.c_int * 3)(0, 0, 0))
    assert lib.fslbm_create(ctypes.byref(dom), 18, 1, 3, ctypes.byref(p), ctypes.byref(h)) == fslbm.EINVAL
    assert lib.fslbm_create(ctypes.byref(dom), 19, 1, 9, ctypes.byref(p), ctypes.byref(h)) == fslbm.EINVAL
    p.omega = 2.5
    assert lib.fslbm_create(ctypes.byref(dom), 19, 1, 3, ctypes.byref(p), ctypes.byref(h)) == fslbm.EINVAL
