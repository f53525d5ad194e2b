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


def test_header_declares_the_core_step_calls():
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


def test_memory_estimate_needs_no_gpu():
    """The admission estimate is host arithmetic: it grows with the domain
    and the stored precision, counts init's velocity staging, and rejects
    bad sizes and enums."""
    from paper_2207_13962_gb300 import fslbm
    lib = fslbm.load()
    e = {prec: fslbm.memory_estimate((64, 64, 64), 19, prec) for prec in ("FP64", "FP32", "FP16S", "BF16S")}
    assert e["FP64"] > e["FP32"] > e["FP16S"] == e["BF16S"]
    N = 64 ** 3
    # two FP32 PDF buffers alone take 2 * 19 * 4 bytes per cell
    assert e["FP32"] >= 2 * 19 * 4 * N
    assert fslbm.memory_estimate((64, 64, 64), 27, "FP32") > e["FP32"]
    # init stages the velocity field twice: as given and in the storage order
    assert fslbm.memory_estimate((64, 64, 64), 19, "FP32", with_velocity=True) == e["FP32"] + 2 * 24 * N
    assert fslbm.memory_estimate((128, 64, 64), 19, "FP32") > 1.9 * e["FP32"]
    b = ctypes.c_size_t(0)
    bad = fslbm.fslbm_domain(0, 4, 4, (ctypes.c_int * 3)(0, 0, 0))
    assert lib.fslbm_memory_estimate(ctypes.byref(bad), 19, 1, 0, ctypes.byref(b)) == fslbm.EINVAL
    dom = fslbm.fslbm_domain(4, 4, 4, (ctypes.c_int * 3)(0, 0, 0))
    assert lib.fslbm_memory_estimate(ctypes.byref(dom), 18, 1, 0, ctypes.byref(b)) == fslbm.EINVAL
    assert lib.fslbm_memory_estimate(ctypes.byref(dom), 19, 7, 0, ctypes.byref(b)) == fslbm.EINVAL
