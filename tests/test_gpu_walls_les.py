"""Free-slip walls and the Smagorinsky model on the GPU against the oracle.

The rectangular dam break of Sec. 4.2 runs with free-slip walls at all
domain borders and the Smagorinsky model with C_S = 0.1 at omega = 1.9995;
these tests run that setup (scaled down) and mixed boundaries.  FP64 mode:
identical flags after every step, PDFs, fill levels and interface masses
within 1e-12 relative (the kernels keep the oracle's expression order).
"""
import numpy as np
import pytest

from oracle import Oracle, feq
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

FREE_SLIP = 2


def _close(a, b):
    return np.abs(a - b) <= 1e-12 * np.abs(b)


def _compare(o, g, step):
    ro, rg = o.read(), g.read()
    np.testing.assert_array_equal(rg["flags"], ro["flags"], err_msg=f"flags differ at step {step}")
    fl = ro["flags"]
    fluid = (fl == S.LIQ) | (fl == S.IFACE)
    iface = fl == S.IFACE
    assert _close(rg["fill"], ro["fill"]).all(), f"fill differs at step {step}"
    assert _close(rg["mass"][iface], ro["mass"][iface]).all(), f"mass differs at step {step}"
    assert _close(rg["pdf"][:, fluid], ro["pdf"][:, fluid]).all(), f"pdf differs at step {step}"


def _pair(sc, periodic, precision="FP64", **over):
    from paper_2207_13962_gb300 import fslbm
    kw = S.make_oracle_kwargs(sc, periodic=periodic, **over)
    o = Oracle(*sc.shape, **kw)
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    g = fslbm.context_for(sc, precision=precision, periodic=periodic, **over)
    return o, g


def _dam_break(q):
    return S.dam_break(nx=48, ny=32, nz=8, W=12, H=24, g=2e-4, q=q, variant="OM", collision="SRT")


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("variant", ["OM", "NBRC"])
def test_dam_break_free_slip_les(q, variant, gpu_lib):
    """All borders free-slip, SRT omega = 1.9995, Smagorinsky C_S = 0.1."""
    sc = _dam_break(q)
    o, g = _pair(sc, (FREE_SLIP,) * 3, variant=variant, omega=1.9995, smagorinsky_cs=0.1)
    M0 = o.total_mass()
    for s in range(1, 121):
        o.step(1)
        g.step(1)
        if s % 20 == 0:
            _compare(o, g, s)
    assert abs(g.observables()["total_mass"] - M0) <= 1e-12 * M0


@pytest.mark.parametrize("collision", ["SRT", "TRT"])
def test_mixed_boundaries_with_les(collision, gpu_lib):
    """Free-slip x, no-slip y, periodic z with obstacles, random velocities,
    surface tension and gravity (conversions both ways)."""
    sc = S.random_interface(shape=(29, 21, 9), seed=13, variant="OM3")
    o, g = _pair(sc, (FREE_SLIP, 0, 1), collision=collision, smagorinsky_cs=0.15)
    for s in range(1, 81):
        o.step(1)
        g.step(1)
        if s % 20 == 0:
            _compare(o, g, s)


@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_free_surface_slab_along_free_slip_walls(precision, gpu_lib):
    """The oracle's steady-state pin on the GPU: a slab moving along a
    free-slip floor and free-slip side walls under a free surface (D3Q27)."""
    from paper_2207_13962_gb300 import fslbm
    nx, ny, nz = 6, 9, 5
    U = (0.03, 0.0, 0.0)
    fl = np.full((nz, ny, nx), S.GAS, np.uint8)
    fill = np.zeros((nz, ny, nx))
    fl[:, :4, :], fill[:, :4, :] = S.LIQ, 1.0
    fl[:, 4, :], fill[:, 4, :] = S.IFACE, 0.5
    fluid = ((fl == S.LIQ) | (fl == S.IFACE)).reshape(-1)
    vel = np.concatenate([np.where(fluid, U[a], 0.0) for a in range(3)])
    g = fslbm.Context((nx, ny, nz), periodic=(1, FREE_SLIP, FREE_SLIP), q=27, variant="OM", omega=1.1,
                      precision=precision)
    g.init(fill.reshape(-1), fl.reshape(-1), vel, None)
    g.step(30)
    r = g.read()
    np.testing.assert_array_equal(r["flags"], fl.reshape(-1))
    tol = 1e-13 if precision == "FP64" else 1e-6
    assert np.abs(r["fill"][fluid] - fill.reshape(-1)[fluid]).max() <= tol
    assert np.abs(r["pdf"][:, fluid] - feq(27, 1.0, U)[:, None]).max() <= tol


def test_fp32_les_within_the_fp32_bound(gpu_lib):
    """FP32 deviations with the model: 3 steps of the free-slip dam break
    against the FP64 oracle, flags identical, PDFs within the FP32 bound of
    the other FP32 tests (25 u per step, u = 2^-24)."""
    sc = _dam_break(19)
    o, g = _pair(sc, (FREE_SLIP,) * 3, precision="FP32", omega=1.9995, smagorinsky_cs=0.1)
    o.step(3)
    g.step(3)
    ro, rg = o.read(), g.read()
    np.testing.assert_array_equal(rg["flags"], ro["flags"])
    fluid = (ro["flags"] == S.LIQ) | (ro["flags"] == S.IFACE)
    assert np.abs(rg["pdf"][:, fluid] - ro["pdf"][:, fluid]).max() <= 3 * 25 * 2.0 ** -24
    assert np.abs(rg["fill"] - ro["fill"]).max() <= 1e-4


def test_batch_with_free_slip_and_les_matches_alone(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    scs = [_dam_break(19), S.random_interface(shape=(17, 19, 7), seed=3, collision="SRT")]
    per = [(FREE_SLIP,) * 3, (1, 0, 1)]
    kw = dict(omega=1.9, smagorinsky_cs=0.1)
    alone = [fslbm.context_for(sc, precision="FP64", periodic=p, **kw) for sc, p in zip(scs, per)]
    members = [fslbm.context_for(sc, precision="FP64", periodic=p, **kw) for sc, p in zip(scs, per)]
    batch = fslbm.Batch(members)
    batch.step(40)
    for a in alone:
        a.step(40)
    for a, m in zip(alone, members):
        ra, rm = a.read(), m.read()
        for k in ("flags", "fill", "pdf"):
            np.testing.assert_array_equal(ra[k], rm[k])
    batch.close()
