"""fslbm_observables_noalloc: the observables reduction for callers that may
not allocate device memory (their memory belongs to another allocator, or an
allocation would stall a latency-critical loop).  It reads a state held in
caller-owned device buffers and keeps its partial sums in a fixed array of
the library.  Checked through the C ABI against fslbm_observables on the same
state, on two calls in a row (the second call reuses the array left by the
first).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


def test_noalloc_observables_match_allocating_entry_point(gpu_lib):
    import torch

    from paper_2207_13962_gb300 import fslbm
    torch.cuda.set_device(0)
    sc = S.random_interface(shape=(37, 21, 11), seed=5)
    ctx = fslbm.context_for(sc, precision="FP64")
    ctx.step(30)
    ref = ctx.observables()
    assert ref["status"] == 0
    r = ctx.read()
    dev = torch.device("cuda", 0)
    pdf = torch.from_numpy(np.ascontiguousarray(r["pdf"].reshape(-1))).to(dev)
    flags = torch.from_numpy(r["flags"]).to(dev)
    fill = torch.from_numpy(r["fill"]).to(dev)
    mass = torch.from_numpy(r["mass"]).to(dev)
    g = (C.c_double * 3)(*sc.g)
    dom = fslbm.fslbm_domain(*sc.shape, (C.c_int * 3)(*[int(x) for x in sc.periodic]))
    torch.cuda.synchronize()
    for _ in range(2):
        out = fslbm.fslbm_obs()
        st = gpu_lib.fslbm_observables_noalloc(C.byref(dom), sc.q, g, C.c_void_p(pdf.data_ptr()),
                                               C.c_void_p(flags.data_ptr()), C.c_void_p(fill.data_ptr()),
                                               C.c_void_p(mass.data_ptr()), C.byref(out), None)
        assert st == fslbm.OK
        for k in ("n_liquid", "n_interface", "n_gas", "n_obstacle"):
            assert getattr(out, k) == ref[k], k
        for k in ("total_mass", "liquid_volume", "max_u"):
            assert abs(getattr(out, k) - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
        assert out.nan_seen == 0
    # sizes outside the supported range are rejected before any GPU work
    bad = fslbm.fslbm_domain(1 << 16, 1 << 16, 1, (C.c_int * 3)(0, 0, 0))
    assert gpu_lib.fslbm_observables_noalloc(C.byref(bad), 19, g, C.c_void_p(pdf.data_ptr()),
                                             C.c_void_p(flags.data_ptr()), C.c_void_p(fill.data_ptr()),
                                             C.c_void_p(mass.data_ptr()), C.byref(out), None) == fslbm.EINVAL
    assert gpu_lib.fslbm_observables_noalloc(C.byref(dom), 18, g, C.c_void_p(pdf.data_ptr()),
                                             C.c_void_p(flags.data_ptr()), C.c_void_p(fill.data_ptr()),
                                             C.c_void_p(mass.data_ptr()), C.byref(out), None) == fslbm.EINVAL
    ctx.close()
