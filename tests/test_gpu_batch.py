"""Batches: uneven domains advanced by one launch per phase over a block table
(``fslbm_batch_*``).  The batched kernels run the same per-cell bodies as
the single-domain ones, so in FP64 (compiled without multiply-add
contraction) every member must match a copy of it stepped alone bit for bit,
whatever the mix of sizes, variants, parities and interleaved
single-context calls.  In FP32 the compiler may contract multiply-adds
differently in the two kernels, so FP32 members agree to FP32 rounding
(flags identical, PDFs within 1e-6).  The single-domain path itself is pinned
to the oracle by test_gpu_parity.py; one member here is also compared with
the oracle directly."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


def _mixed_fp64():
    return [S.random_interface(shape=(37, 21, 11), seed=7, variant="NBRC"),
            S.random_interface(shape=(24, 18, 9), seed=11, variant="NBKC", periodic=(True, True, False)),
            S.random_interface(shape=(16, 30, 7), seed=3, variant="OM"),
            S.random_interface(shape=(9, 13, 5), seed=5, variant="OM3"),
            S.taylor_bubble(nx=24, ny=24, nz=64, D=20, bubble_d=12, bubble_len=20, z0=12, z_ref=40.0,
                            g=2e-5, sigma=2e-3, nu=0.02),
            S.gravity_wave()]


def _assert_same(a, b, what):
    ra, rb = a.read(), b.read()
    for k in ("flags", "fill", "mass", "pdf"):
        np.testing.assert_array_equal(ra[k], rb[k], err_msg=f"{what}: {k}")


def test_batch_matches_members_alone_fp64(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    scs = _mixed_fp64()
    alone = [fslbm.context_for(sc, precision="FP64") for sc in scs]
    members = [fslbm.context_for(sc, precision="FP64") for sc in scs]
    # different parities: member 1 is three steps ahead when the batch starts
    alone[1].step(3)
    members[1].step(3)
    batch = fslbm.Batch(members)
    for _ in range(4):
        batch.step(10)
        for a in alone:
            a.step(10)
    st, per = batch.sync()
    assert st == fslbm.OK and per == [fslbm.OK] * len(scs)
    for k, (a, m) in enumerate(zip(alone, members)):
        _assert_same(a, m, f"member {k}")
        assert m.observables()["step"] == a.observables()["step"]
    Va, Pa = alone[4].bubbles()
    Vm, Pm = members[4].bubbles()
    np.testing.assert_array_equal(Va, Vm)
    np.testing.assert_array_equal(Pa, Pm)
    # interleaving: single-context steps between batch steps
    members[2].step(2)
    alone[2].step(2)
    batch.step(5)
    for a in alone:
        a.step(5)
    for k, (a, m) in enumerate(zip(alone, members)):
        _assert_same(a, m, f"member {k} after interleaving")
    assert batch.launches() == 45 * 11
    batch.close()


def test_batch_member_matches_oracle(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    scs = _mixed_fp64()
    members = [fslbm.context_for(sc, precision="FP64") for sc in scs]
    batch = fslbm.Batch(members)
    o = Oracle(*scs[0].shape, **S.make_oracle_kwargs(scs[0]))
    o.init(scs[0].fill, scs[0].flags, scs[0].velocity, scs[0].density)
    for s in range(1, 31):
        batch.step(1)
        o.step(1)
        if s % 10 == 0:
            ro, rg = o.read(), members[0].read()
            np.testing.assert_array_equal(rg["flags"], ro["flags"])
            fl = ro["flags"]
            fluid = (fl == S.LIQ) | (fl == S.IFACE)
            assert np.all(np.abs(rg["pdf"][:, fluid] - ro["pdf"][:, fluid]) <= 1e-12 * np.abs(ro["pdf"][:, fluid]))
            assert np.all(np.abs(rg["fill"] - ro["fill"]) <= 1e-12 * np.abs(ro["fill"]))
    batch.close()


def test_batch_fp32_d3q27_cylinders(gpu_lib):
    """Uneven cylindrical dam breaks, D3Q27, FP32 deviations (the batched
    workload's lattice and precision) at small sizes."""
    from paper_2207_13962_gb300 import fslbm
    Ls = [24, 31, 40, 17, 33]
    scs = [S.cylinder_dam_break(L=L, r_frac=0.2 + 0.04 * k, h_frac=0.35 - 0.03 * k, q=27, g=1e-4)
           for k, L in enumerate(Ls)]
    alone = [fslbm.context_for(sc, precision="FP32") for sc in scs]
    members = [fslbm.context_for(sc, precision="FP32") for sc in scs]
    batch = fslbm.Batch(members)
    batch.step(60)
    for a in alone:
        a.step(60)
    for k, (a, m) in enumerate(zip(alone, members)):
        ra, rm = a.read(), m.read()
        np.testing.assert_array_equal(ra["flags"], rm["flags"], err_msg=f"cylinder {k}")
        assert np.abs(ra["pdf"] - rm["pdf"]).max() <= 1e-6, f"cylinder {k}"
        assert np.abs(ra["fill"] - rm["fill"]).max() <= 1e-6, f"cylinder {k}"
    batch.close()


def test_batch_autotune_keeps_state_exact(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    scs = _mixed_fp64()[:3]
    alone = [fslbm.context_for(sc, precision="FP64") for sc in scs]
    members = [fslbm.context_for(sc, precision="FP64") for sc in scs]
    batch = fslbm.Batch(members)
    t = batch.autotune(steps=1)
    assert 1 <= t["bulk_blocks_per_sm"] <= 2 and t["band_blocks_per_sm"] in (1, 2, 4, 8)
    assert t["ms_per_step"] > 0 and batch.tuning()["bulk_blocks_per_sm"] == t["bulk_blocks_per_sm"]
    done = members[0].observables()["step"]
    assert done == 2 * 2 * 4  # (1 + 1) steps x 2 bulk shapes x 4 band shapes
    for a in alone:
        a.step(done)
    for k, (a, m) in enumerate(zip(alone, members)):
        _assert_same(a, m, f"member {k} after autotune")
    batch.close()


def test_batch_rejects_mixed_members(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.random_interface(shape=(10, 12, 6), seed=1)
    a = fslbm.context_for(sc, precision="FP64")
    b = fslbm.context_for(sc, precision="FP32")
    with pytest.raises(fslbm.FslbmError) as e:
        fslbm.Batch([a, b])
    assert e.value.status == fslbm.EINVAL
    with pytest.raises(fslbm.FslbmError) as e:
        fslbm.Batch([a, a])
    assert e.value.status == fslbm.EINVAL
    c = fslbm.Context((8, 8, 8), precision="FP64")
    with pytest.raises(fslbm.FslbmError) as e:
        fslbm.Batch([a, c])
    assert e.value.status == fslbm.ESTATE
