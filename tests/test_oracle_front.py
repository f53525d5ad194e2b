"""Pins of the oracle's seed-fill front detection (Sec. 4.3, cylindrical dam
break; reading R23): the fill runs in one z-layer through gas and obstacle
cells over in-plane face neighbours, seeded on the layer's edge, and the
front is the set of interface cells with a reached gas face neighbour.

The oracle's breadth-first fill is checked against connected-component
labelling by scipy.ndimage (a library routine: 4-connected components of
the gas-or-obstacle mask that touch the edge) on random layers, and against
hand-built layers whose front is known: a disc (every ring cell is front),
an annulus (its inner ring is not: the hole does not connect to the edge),
a hole opened to the outside through an obstacle channel, and a hole that
reaches the edge only across a periodic face."""
import numpy as np
import pytest

from oracle import seed_fill_front

GAS, IFACE, LIQ, OBST = 0, 1, 2, 3


def _layered(layer2d, nz=3, k=1):
    """A flags volume of nz layers (gas elsewhere) with layer k = layer2d."""
    ny, nx = layer2d.shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[k] = layer2d
    return fl.reshape(-1), (nx, ny, nz)


def _library_front(layer2d, periodic):
    """The same front from scipy.ndimage.label (4-connectivity); periodic axes
    by labelling a 3x3 tiling and keeping the centre copy's labels."""
    ndimage = pytest.importorskip("scipy.ndimage")
    ny, nx = layer2d.shape
    outside = (layer2d == GAS) | (layer2d == OBST)
    reps = (3 if periodic[1] else 1, 3 if periodic[0] else 1)
    big = np.tile(outside, reps)
    lab, _ = ndimage.label(big, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    oy, ox = (ny if periodic[1] else 0), (nx if periodic[0] else 0)
    edge = np.zeros_like(outside)
    edge[0, :] = edge[-1, :] = True
    edge[:, 0] = edge[:, -1] = True
    seeds = set(np.unique(lab[oy:oy + ny, ox:ox + nx][edge & outside])) - {0}
    reached = np.isin(lab[oy:oy + ny, ox:ox + nx], list(seeds)) & (layer2d == GAS)
    front = np.zeros_like(outside)
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        sh = np.zeros_like(outside)
        src_y = np.arange(ny) + dy
        src_x = np.arange(nx) + dx
        vy = (src_y >= 0) & (src_y < ny) if not periodic[1] else np.ones(ny, bool)
        vx = (src_x >= 0) & (src_x < nx) if not periodic[0] else np.ones(nx, bool)
        yy, xx = np.meshgrid(src_y % ny, src_x % nx, indexing="ij")
        sh = reached[yy, xx] & vy[:, None] & vx[None, :]
        front |= sh
    return front & (layer2d == IFACE)


def _disc(n, r, centre=None, hole=None):
    c = (n / 2.0, n / 2.0) if centre is None else centre
    y, x = np.mgrid[0:n, 0:n] + 0.5
    d = np.hypot(x - c[0], y - c[1])
    lay = np.where(d < r, LIQ, GAS).astype(np.uint8)
    if hole is not None:
        lay[d < hole] = GAS
    # interface: liquid cells with a gas face neighbour
    liq = lay == LIQ
    gas = lay == GAS
    g = np.zeros_like(gas)
    g[1:, :] |= gas[:-1, :]
    g[:-1, :] |= gas[1:, :]
    g[:, 1:] |= gas[:, :-1]
    g[:, :-1] |= gas[:, 1:]
    lay[liq & g] = IFACE
    return lay


def test_disc_every_ring_cell_is_front():
    lay = _disc(40, 11.0)
    fl, shape = _layered(lay)
    front, st = seed_fill_front(fl, shape, 1, (20.0, 20.0))
    np.testing.assert_array_equal(front, lay == IFACE)
    r = np.hypot(np.nonzero(lay == IFACE)[1] + 0.5 - 20.0, np.nonzero(lay == IFACE)[0] + 0.5 - 20.0)
    assert st["count"] == r.size
    assert st["r_max"] == pytest.approx(r.max(), abs=0) and st["r_min"] == pytest.approx(r.min(), abs=0)
    assert st["r_mean"] == pytest.approx(r.mean(), rel=1e-15)
    # the ring lies within one cell inside the disc's radius
    assert 10.0 - 1e-12 <= st["r_min"] and st["r_max"] < 11.0


def test_annulus_inner_ring_is_not_front():
    lay = _disc(48, 16.0, hole=6.0)
    fl, shape = _layered(lay)
    front, st = seed_fill_front(fl, shape, 1, (24.0, 24.0))
    y, x = np.mgrid[0:48, 0:48] + 0.5
    d = np.hypot(x - 24.0, y - 24.0)
    outer = (lay == IFACE) & (d > 11.0)
    inner = (lay == IFACE) & (d < 11.0)
    assert inner.any() and outer.any()
    np.testing.assert_array_equal(front, outer)
    assert st["r_min"] > 15.0 - 1e-12


def test_obstacle_channel_opens_the_hole():
    lay = _disc(48, 16.0, hole=6.0)
    y, x = np.mgrid[0:48, 0:48] + 0.5
    # an obstacle channel from the hole to the right edge along y = 24
    lay[(np.abs(y - 24.5) < 0.6) & (x > 24.0)] = OBST
    fl, shape = _layered(lay)
    front, _ = seed_fill_front(fl, shape, 1, (24.0, 24.0))
    inner = (lay == IFACE) & (np.hypot(x - 24.0, y - 24.0) < 11.0)
    # inner-ring cells facing the (now reached) hole gas are front
    assert (front & inner).any()
    np.testing.assert_array_equal(front, _library_front(lay, (False, False)))


def test_periodic_face_connects():
    # a band of liquid across the whole width, a gas pocket above it that
    # touches the edge only through the top row, which is liquid except for
    # a gap that wraps around in x
    ny, nx = 20, 24
    lay = np.full((ny, nx), GAS, np.uint8)
    lay[5:15, :] = LIQ
    lay[8:12, 10:14] = GAS           # an enclosed pocket
    lay[4, :] = IFACE
    lay[15, :] = IFACE
    lay[7, 10:14] = IFACE
    lay[12, 10:14] = IFACE
    lay[8:12, 9] = IFACE
    lay[8:12, 14] = IFACE
    fl, shape = _layered(lay)
    for per in ((False, False), (True, False), (True, True)):
        front, _ = seed_fill_front(fl, shape, 1, (12.0, 10.0), periodic=per)
        np.testing.assert_array_equal(front, _library_front(lay, per))
        assert not front[7, 10:14].any()  # the pocket's rim never is


@pytest.mark.parametrize("seed", range(12))
def test_matches_library_labelling_on_random_layers(seed):
    rng = np.random.default_rng(seed)
    ny, nx = rng.integers(5, 30, 2)
    lay = rng.choice([GAS, IFACE, LIQ, OBST], size=(ny, nx), p=[0.4, 0.3, 0.2, 0.1]).astype(np.uint8)
    per = (bool(seed & 1), bool(seed & 2))
    fl, shape = _layered(lay, nz=2, k=seed % 2)
    front, st = seed_fill_front(fl, shape, seed % 2, (nx / 2.0, ny / 2.0), periodic=per)
    ref = _library_front(lay, per)
    np.testing.assert_array_equal(front, ref)
    assert st["count"] == int(ref.sum())


def test_other_layers_are_ignored_and_bad_layer_rejected():
    lay = _disc(30, 8.0)
    fl, shape = _layered(lay, nz=3, k=1)
    _, st0 = seed_fill_front(fl, shape, 0, (15.0, 15.0))
    assert st0["count"] == 0 and st0["r_max"] == 0.0
    with pytest.raises(ValueError):
        seed_fill_front(fl, shape, 3, (15.0, 15.0))
