"""Pins of the free-slip walls (reading R22) and the Smagorinsky model
(reading R21) of the oracle.

Free-slip (Sec. 2.1: PDFs reflected specularly, normal component reversed):
* a uniform flow along free-slip walls is an exact steady state (specular
  reflection maps f^eq(rho, U) onto itself when U is tangential), while the
  same flow between no-slip walls decays;
* a liquid slab moving uniformly along a free-slip floor and free-slip side
  walls, under a free surface, is an exact steady state too: at the side
  walls the specularly reflected PDFs that come from gas cells are missing
  and the free-surface BC (Eq. nm-fslbm-boundary-condition, Sec. 2.2)
  reconstructs them as f^eq(1, U).  On D3Q27 the corner directions carry
  c.U != 0, so bouncing them back instead leaves an O(U) error: with that
  mistake planted in the oracle the OM case fails (NBRC reconstructs those
  directions by the normal anyway).

Smagorinsky (Sec. 2.1, Eqs. nm-lbm-turbulence-viscosity to
nm-lbm-turublence-relaxation-time):
* with no non-equilibrium part the collision is the plain one;
* for a single cell with the non-equilibrium part A w_i c_ix c_iy (which
  changes neither density nor momentum) the momentum flux is Q_xy = Q_yx =
  A sum_i w_i c_ix^2 c_iy^2 = A c_s^4 = A / 9 and nothing else, so
  Qbar = sqrt(2 (Q_xy^2 + Q_yx^2)) = 2 A / 9; the relaxation time read back
  from the collision's output is the model's for that Qbar;
* mass is conserved and the momentum gains F, with the model on.
"""
import numpy as np
import pytest

from oracle import Oracle, collide, feq, lattice
from paper_2207_13962_gb300 import scenarios as S

FREE_SLIP = 2


def _liquid_box(shape, U):
    nx, ny, nz = shape
    N = nx * ny * nz
    vel = np.concatenate([np.full(N, U[0]), np.full(N, U[1]), np.full(N, U[2])])
    return np.ones(N), np.full(N, S.LIQ, np.uint8), vel


@pytest.mark.parametrize("q", [19, 27])
def test_uniform_flow_along_free_slip_walls_is_steady(q):
    shape = (8, 6, 5)
    U = (0.04, 0.0, 0.0)
    fill, flags, vel = _liquid_box(shape, U)
    o = Oracle(*shape, periodic=(1, FREE_SLIP, FREE_SLIP), q=q, omega=1.3)
    o.init(fill, flags, vel, None)
    o.step(40)
    f = o.read()["pdf"]
    np.testing.assert_allclose(f, np.repeat(feq(q, 1.0, U)[:, None], f.shape[1], 1), rtol=0, atol=1e-14)
    # between no-slip walls the same flow loses momentum
    n = Oracle(*shape, periodic=(1, 0, 0), q=q, omega=1.3)
    n.init(fill, flags, vel, None)
    n.step(40)
    _, u = n.moments()
    assert u[0].mean() < 0.9 * U[0]


def _slab(U, q=27):
    """Liquid slab y < 4 on a free-slip floor, interface row y = 4, gas
    above; periodic x, free-slip side walls in z; uniform velocity U."""
    nx, ny, nz = 6, 9, 5
    fl = np.full((nz, ny, nx), S.GAS, np.uint8)
    fill = np.zeros((nz, ny, nx))
    fl[:, :4, :] = S.LIQ
    fill[:, :4, :] = 1.0
    fl[:, 4, :] = S.IFACE
    fill[:, 4, :] = 0.5
    fluid = ((fl == S.LIQ) | (fl == S.IFACE)).reshape(-1)
    N = nx * ny * nz
    vel = np.concatenate([np.where(fluid, U[a], 0.0) for a in range(3)])
    return (nx, ny, nz), fill.reshape(-1), fl.reshape(-1), vel, fluid


@pytest.mark.parametrize("variant", ["NBRC", "OM"])
def test_free_surface_slab_along_free_slip_walls_is_steady(variant):
    U = (0.03, 0.0, 0.0)
    shape, fill, flags, vel, fluid = _slab(U)
    o = Oracle(*shape, periodic=(1, FREE_SLIP, FREE_SLIP), q=27, variant=variant, omega=1.1)
    o.init(fill, flags, vel, None)
    o.step(30)
    r = o.read()
    np.testing.assert_array_equal(r["flags"], flags)
    np.testing.assert_allclose(r["fill"][fluid], fill[fluid], rtol=0, atol=1e-13)
    f = r["pdf"][:, fluid]
    np.testing.assert_allclose(f, np.repeat(feq(27, 1.0, U)[:, None], f.shape[1], 1), rtol=0, atol=1e-13)


@pytest.mark.parametrize("q", [19, 27])
def test_les_reduces_to_plain_collision_at_zero_strain(q):
    u = np.array([0.03, -0.02, 0.01])
    fin = feq(q, 1.02, u)
    g = np.zeros(3)
    for coll in (0, 1):
        plain, _, _ = collide(q, coll, 1.7, 3.0 / 16.0, g, fin)
        les, _, _ = collide(q, coll, 1.7, 3.0 / 16.0, g, fin, cs=0.1)
        np.testing.assert_allclose(les, plain, rtol=1e-15, atol=1e-17)


@pytest.mark.parametrize("q", [19, 27])
def test_les_relaxation_time_from_the_momentum_flux(q):
    c, w, _ = lattice(q)
    c = c.astype(np.float64)
    rho, A, omega, cs = 1.03, 1e-2, 1.95, 0.3
    neq = A * w * c[:, 0] * c[:, 1]
    fin = feq(q, rho, np.zeros(3)) + neq
    out, r, u = collide(q, 0, omega, 0.0, np.zeros(3), fin, cs=cs)
    assert abs(r - rho) < 1e-15 and np.abs(u).max() < 1e-16  # neq carries no mass or momentum
    ratio = (out - feq(q, rho, np.zeros(3)))[neq != 0] / neq[neq != 0]
    tau_read = 1.0 / (1.0 - ratio)
    qbar = 2.0 * A / 9.0  # closed form of the momentum-flux magnitude
    tau0 = 1.0 / omega
    tau_model = 0.5 * (tau0 + np.sqrt(tau0 ** 2 + 2.0 * np.sqrt(2.0) * cs ** 2 * qbar / (rho / 9.0)))
    np.testing.assert_allclose(tau_read, tau_model, rtol=1e-12)
    assert tau_model > tau0 * 1.002  # the model is active at this strain


@pytest.mark.parametrize("q", [19, 27])
def test_les_collision_conserves_mass_and_adds_the_force(q):
    c, w, _ = lattice(q)
    rng = np.random.default_rng(4)
    g = np.array([1e-4, -2e-4, 5e-5])
    for coll in (0, 1):
        fin = w * rng.uniform(0.9, 1.1, q)
        out, rho, _ = collide(q, coll, 1.9, 3.0 / 16.0, g, fin, cs=0.1)
        assert abs(out.sum() - fin.sum()) < 1e-15
        dj = c.T.astype(np.float64) @ (out - fin)
        np.testing.assert_allclose(dj, rho * g, rtol=1e-10, atol=1e-18)
