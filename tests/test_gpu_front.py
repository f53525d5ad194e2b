"""Seed-fill front detection on the device (``fslbm_front``; Sec. 4.3,
cylindrical dam break) against the oracle's breadth-first fill on the same
flags: the front mask, the count and the minimum and maximum radius are
identical (the radius is one correctly rounded square root of the same
operands), the mean radius agrees to relative 1e-12 (the device sums with
atomics in no fixed order)."""
import numpy as np
import pytest

from oracle import seed_fill_front
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


def _check(ctx, shape, periodic, layer, centre):
    got = ctx.front(layer, centre, mask=True)
    flags = ctx.read(pdf=False)["flags"]
    ref_mask, ref = seed_fill_front(flags, shape, layer, centre, periodic=periodic[:2])
    np.testing.assert_array_equal(got["mask"], ref_mask)
    assert got["count"] == ref["count"]
    assert got["r_min"] == ref["r_min"] and got["r_max"] == ref["r_max"]
    assert abs(got["r_mean"] - ref["r_mean"]) <= 1e-12 * max(ref["r_mean"], 1e-300)
    return got


@pytest.mark.parametrize("precision", ["FP32", "FP64"])
def test_cylinder_front_matches_oracle(precision, gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.cylinder_dam_break(L=48, r_frac=0.25, h_frac=0.35, g=1e-4, q=27)
    ctx = fslbm.context_for(sc, precision=precision)
    radii = []
    for steps in (0, 80, 120):
        ctx.step(steps)
        got = _check(ctx, sc.shape, sc.periodic, 0, (24.0, 24.0))
        assert got["count"] > 0
        radii.append(got["r_max"])
    # the column spreads on the floor
    assert radii[-1] > radii[0]
    ctx.close()


@pytest.mark.parametrize("order", [None, (2, 0, 1)])
def test_rough_surface_layers_match_oracle(order, gpu_lib):
    """Obstacles, a periodic x axis and every z-layer of a rough surface with
    a droplet; the storage order of the cells does not change the result."""
    from paper_2207_13962_gb300 import fslbm
    sc = S.random_interface(shape=(37, 21, 11), seed=5, variant="OM")
    ctx = fslbm.context_for(sc, precision="FP32", axis_order=order)
    ctx.step(10)
    for layer in range(sc.shape[2]):
        _check(ctx, sc.shape, sc.periodic, layer, (18.5, 10.5))
    with pytest.raises(fslbm.FslbmError) as e:
        ctx.front(sc.shape[2], (0.0, 0.0))
    assert e.value.status == fslbm.EINVAL
    ctx.close()
