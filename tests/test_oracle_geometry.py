"""Pins of the oracle's interface geometry (Sec. 2.2: smoothed fill level,
Parker-Youngs normal, curvature) by closed forms that hold for any correct
implementation:

* K8 smoothing is a symmetric kernel divided by its sum, so it reproduces
  constant and linear fill fields exactly (away from walls and faces).  A
  wrong normalisation, a missing stencil point or an asymmetric weight breaks
  this.
* The Parker-Youngs normal of a linear field phi = a + b.x is b / |b| (its
  weighted central differences are all proportional to b).  A transposed axis,
  a sign error or a dropped component breaks this.
* A planar field has zero curvature.
* The normal points into the liquid (towards growing fill level), and the
  curvature of a liquid sphere of radius R approaches 2 / R (sum of the
  principal curvatures, reading R7), of a gas sphere -2 / R.

The domains hold interface cells only, so every cell carries its own fill
level and the closed-layer condition holds trivially.
"""
import numpy as np
import pytest

from oracle import Oracle

SHAPE = (14, 13, 12)


def _geometry(phi, shape=SHAPE):
    nx, ny, nz = shape
    o = Oracle(nx, ny, nz)
    flags = np.full(nx * ny * nz, 1, np.uint8)  # interface everywhere
    o.init(phi.reshape(-1).astype(np.float64), flags, None, None)
    nhat, kappa, phis = o.geometry()
    return nhat.reshape(3, nz, ny, nx), kappa.reshape(nz, ny, nx), phis.reshape(nz, ny, nx)


def _interior(shape, d):
    nx, ny, nz = shape
    m = np.zeros((nz, ny, nx), bool)
    m[d:nz - d, d:ny - d, d:nx - d] = True
    return m


def _coords(shape):
    nx, ny, nz = shape
    return np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")


@pytest.mark.parametrize("b", [(0.02, -0.015, 0.01), (0.0, 0.0, 0.03), (-0.01, 0.025, 0.0)])
def test_linear_field_smoothing_normal_curvature(b):
    z, y, x = _coords(SHAPE)
    phi = 0.5 + b[0] * (x - 6.5) + b[1] * (y - 6.0) + b[2] * (z - 5.5)
    nhat, kappa, phis = _geometry(phi)
    # smoothing reads +-1, so cells 1 away from a face see only real cells
    m1 = _interior(SHAPE, 1)
    np.testing.assert_allclose(phis[m1], phi[m1], rtol=0, atol=1e-14)
    # the normal reads the smoothed field at +-1: 2 cells from a face
    m2 = _interior(SHAPE, 2)
    bn = np.array(b) / np.linalg.norm(b)
    for a in range(3):
        np.testing.assert_allclose(nhat[a][m2], bn[a], rtol=0, atol=1e-12)
    # the curvature reads the normal at +-1: 3 cells from a face
    m3 = _interior(SHAPE, 3)
    np.testing.assert_allclose(kappa[m3], 0.0, rtol=0, atol=1e-12)


def test_constant_field_is_reproduced_and_has_no_normal():
    phi = np.full((SHAPE[2], SHAPE[1], SHAPE[0]), 0.37)
    nhat, kappa, phis = _geometry(phi)
    # obstacles and faces take the centre's value, so a constant stays exact
    # everywhere, and its gradient vanishes: n^ = 0 by the len > 0 rule
    np.testing.assert_allclose(phis, 0.37, rtol=0, atol=1e-15)
    assert np.abs(nhat).max() == 0.0
    assert np.abs(kappa).max() == 0.0


@pytest.mark.parametrize("liquid_inside", [True, False])
def test_sphere_normal_direction_and_curvature(liquid_inside):
    # a smooth radial fill profile (width ~ 2 cells) around a sphere of
    # radius R; the curvature at cells near the surface approaches +-2/R
    shape = (40, 40, 40)
    R = 12.0
    z, y, x = _coords(shape)
    r = np.sqrt((x - 19.5) ** 2 + (y - 19.5) ** 2 + (z - 19.5) ** 2)
    inside = 0.5 * (1.0 - np.tanh((r - R) / 1.5))
    phi = inside if liquid_inside else 1.0 - inside
    nhat, kappa, _ = _geometry(phi, shape)
    shell = (np.abs(r - R) < 0.75) & _interior(shape, 4)
    # the normal points towards growing fill level: inward for a drop
    radial = np.stack([(x - 19.5) / r, (y - 19.5) / r, (z - 19.5) / r])
    dot = (nhat * radial).sum(0)[shell]
    sign = -1.0 if liquid_inside else 1.0
    assert np.all(sign * dot > 0.99)
    # kappa = -div(n^) is + the sum of the principal curvatures of the liquid
    # surface seen from the liquid: +2/R for a drop, -2/R for a bubble
    k = kappa[shell]
    expect = (2.0 / r[shell]) * (1.0 if liquid_inside else -1.0)
    assert np.abs(np.mean(k) - np.mean(expect)) < 0.1 * 2.0 / R


# ---------------------------------------------------------------------------
# Exact weights of the stencils (readings R16, R17), pinned by their impulse
# responses stored in tests/golden/.  Any other kernel shape, radius or
# normalisation, or other difference weights, changes these values.

def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        return json.load(fh)


def test_k8_impulse_response_on_a_block():
    from fractions import Fraction

    from oracle import k8_smooth
    g = _golden("k8_impulse.json")
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                b = np.zeros((3, 3, 3))
                b[oz + 1, oy + 1, ox + 1] = 1.0
                num, den = g["by_r2"][str(ox * ox + oy * oy + oz * oz)]
                # the weight and its sum are exact dyadic numbers, so the
                # one division rounds correctly: the result is exact to the
                # last bit
                assert k8_smooth(b) == float(Fraction(num, den)), (ox, oy, oz)


def test_k8_impulse_response_in_a_domain():
    """The step's smoothing of a fill-level impulse (one interface cell with
    phi = 1 among gas cells, periodic 5^3 domain)."""
    from fractions import Fraction
    g = _golden("k8_impulse.json")
    n = 5
    o = Oracle(n, n, n, periodic=(True, True, True))
    fill = np.zeros(n ** 3)
    flags = np.zeros(n ** 3, np.uint8)
    c = 2 + n * (2 + n * 2)
    fill[c], flags[c] = 1.0, 1
    o.init(fill, flags, None, None)
    _, _, phis = o.geometry()
    phis = phis.reshape(n, n, n)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                r2 = (x - 2) ** 2 + (y - 2) ** 2 + (z - 2) ** 2
                want = float(Fraction(*g["by_r2"][str(r2)])) if r2 <= 3 else 0.0
                assert phis[z, y, x] == want, (x, y, z)


def test_parker_youngs_impulse_response():
    from oracle import py_gradient
    g = _golden("parker_youngs_impulse.json")
    assert len(g["cases"]) == 27
    for case in g["cases"]:
        ox, oy, oz = case["offset"]
        b = np.zeros((3, 3, 3))
        b[oz + 1, oy + 1, ox + 1] = 1.0
        np.testing.assert_array_equal(py_gradient(b), np.array(case["gradient"], np.float64),
                                      err_msg=str(case["offset"]))
