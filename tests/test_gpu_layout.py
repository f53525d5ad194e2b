"""Storage order of the cells (fslbm_set_axis_order / fslbm_get_axis_order).

Inside a context any axis may be the contiguous one; the caller's cell index
x + nx (y + ny z), the direction labels and all arithmetic stay the same, so
the FP64 engine must give the oracle's results bit for bit in every storage
order, and bubbles must keep their numbering by lowest caller index.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

ORDERS = [(2, 0, 1), (1, 2, 0), (0, 2, 1)]


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


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("q", [19, 27])
def test_stress_domain_in_every_storage_order(order, q, gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.random_interface(shape=(37, 21, 11), seed=7, q=q, variant="OM3")
    o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    g = fslbm.context_for(sc, precision="FP64", axis_order=order)
    assert g.axis_order() == order
    for s in range(1, 61):
        o.step(1)
        g.step(1)
        if s % 15 == 0:
            _compare(o, g, s)
    g.close()


def _three_bubbles():
    """Liquid box (no-slip walls) with three gas bubbles whose order by lowest
    caller index (z first) differs from their order by lowest storage index
    when z or y is the contiguous axis."""
    nx, ny, nz = 20, 18, 16
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.ones((nz, ny, nx))
    for cx, cy, cz, r in ((14.0, 12.0, 4.0, 2.2), (5.0, 4.0, 11.0, 2.8), (13.0, 5.0, 8.0, 3.3)):
        d = np.sqrt((i + 0.5 - cx) ** 2 + (j + 0.5 - cy) ** 2 + (k + 0.5 - cz) ** 2)
        phi = np.minimum(phi, np.clip(d - r, 0.0, 1.0))
    periodic = (False, False, False)
    fill, flags = S.classify(phi, None, periodic, 19)
    return S.Scenario("three_bubbles", (nx, ny, nz), periodic, fill, flags, None, None, q=19,
                      collision="TRT", variant="OM", omega=1.6, g=(0.0, 0.0, -1e-4), sigma=2e-3,
                      bubble_model=True)


@pytest.mark.parametrize("order", [(0, 1, 2)] + ORDERS)
def test_bubbles_keep_their_numbering(order, gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = _three_bubbles()
    o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    g = fslbm.context_for(sc, precision="FP64", axis_order=order)
    V0o, _, _ = o.bubbles()
    V0g, _ = g.bubbles()
    assert len(V0o) == 3
    np.testing.assert_array_equal(V0g, V0o)  # the same volume under the same id
    for s in range(1, 31):
        o.step(1)
        g.step(1)
    _compare(o, g, 30)
    Vo, Po, _ = o.bubbles()
    Vg, Pg = g.bubbles()
    np.testing.assert_allclose(Vg, Vo, rtol=1e-13)
    np.testing.assert_allclose(Pg, Po, rtol=1e-13)
    g.close()


def test_automatic_order_follows_the_liquid(gpu_lib):
    """init keeps x contiguous for a domain whose liquid runs along x and
    makes the tube axis contiguous for a tube along z."""
    from paper_2207_13962_gb300 import fslbm
    wave = fslbm.context_for(S.gravity_wave(), precision="FP32")
    assert wave.axis_order() == (0, 1, 2)
    tube = S.taylor_bubble(nx=40, ny=40, nz=256, D=32, bubble_d=24, bubble_len=64, z0=32, z_ref=128.0)
    t = fslbm.context_for(tube, precision="FP32")
    assert t.axis_order() == (2, 0, 1)
    # the fields come back in the caller's cell order
    r = t.read(pdf=False)
    np.testing.assert_array_equal(r["flags"], tube.flags)
    np.testing.assert_array_equal(r["fill"][tube.flags == S.IFACE], tube.fill[tube.flags == S.IFACE])
    wave.close()
    t.close()


def test_checkpoint_in_another_storage_order(gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.random_interface(shape=(20, 18, 6), seed=2)
    a = fslbm.context_for(sc, precision="FP64", axis_order=(1, 2, 0))
    b = fslbm.context_for(sc, precision="FP64", axis_order=(1, 2, 0))
    a.step(40)
    b.step(20)
    buf = b.save()
    c = fslbm.context_for(sc, precision="FP64", axis_order=(1, 2, 0))
    c.load(buf)
    c.step(20)
    ra, rc = a.read(), c.read()
    for k in ("pdf", "fill", "flags", "mass"):
        np.testing.assert_array_equal(ra[k], rc[k])
    d = fslbm.context_for(sc, precision="FP64")  # x contiguous: another order
    with pytest.raises(fslbm.FslbmError) as e:
        d.load(buf)
    assert e.value.status == fslbm.EINVAL
    with pytest.raises(fslbm.FslbmError):
        d.set_axis_order((0, 0, 1))
