"""Pins of the oracle's lattice algebra (Sec. 2.1) against closed forms.

* equilibrium moments (Eq. fbc-eq-moments, Appendix A);
* mass conservation and momentum gain F per collision under Guo forcing
  (Eqs. nm-lbm-collision, nm-lbm-velocity, nm-lbm-force-guo);
* TRT with omega- = omega+ reduces to SRT;
* lattice isotropy identities of the weights.
"""
import numpy as np
import pytest

from oracle import collide, feq, lattice

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("q", [9, 19, 27])
def test_lattice_isotropy(q):
    c, w, opp = lattice(q)
    c = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ c, 0.0, atol=1e-16)
    d = 2 if q == 9 else 3
    M2 = np.einsum("i,ia,ib->ab", w, c, c)[:d, :d]
    np.testing.assert_allclose(M2, CS2 * np.eye(d), atol=1e-15)
    # fourth-order isotropy: sum w c_a c_b c_g c_d = cs^4 (d_ab d_gd + d_ag d_bd + d_ad d_bg)
    M4 = np.einsum("i,ia,ib,ig,id->abgd", w, c, c, c, c)[:d, :d, :d, :d]
    I = np.eye(d)
    ref = CS2 ** 2 * (np.einsum("ab,gd->abgd", I, I) + np.einsum("ag,bd->abgd", I, I)
                      + np.einsum("ad,bg->abgd", I, I))
    np.testing.assert_allclose(M4, ref, atol=1e-15)
    for i in range(q):
        np.testing.assert_array_equal(c[opp[i]], -c[i])


@pytest.mark.parametrize("q", [9, 19, 27])
def test_equilibrium_moments(q):
    """Eq. fbc-eq-moments: sum f^eq = rho, sum f^eq c = rho u,
    sum f^eq c c = rho cs^2 delta + rho u u."""
    rng = np.random.default_rng(1)
    c, _, _ = lattice(q)
    c = c.astype(np.float64)
    d = 2 if q == 9 else 3
    for _ in range(50):
        rho = rng.uniform(0.5, 1.5)
        u = np.zeros(3)
        u[:d] = rng.uniform(-0.1, 0.1, d)
        f = feq(q, rho, u)
        assert abs(f.sum() - rho) < 1e-14
        np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f, c, c)[:d, :d]
        np.testing.assert_allclose(P, rho * CS2 * np.eye(d) + rho * np.outer(u[:d], u[:d]), atol=1e-14)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("collision", [0, 1])
def test_collision_conserves_mass_and_adds_force(q, collision):
    """A collision conserves rho and raises the momentum by F = rho g:
    sum c f* = sum c f + F (relaxation removes F/2 through the shifted
    equilibrium velocity, the Guo source adds (1 - omega/2) F)."""
    rng = np.random.default_rng(2)
    c, w, _ = lattice(q)
    c = c.astype(np.float64)
    for _ in range(30):
        fin = w * rng.uniform(0.8, 1.2, q)
        g = rng.uniform(-1e-3, 1e-3, 3)
        omega = rng.uniform(0.6, 1.95)
        fout, rho, u = collide(q, collision, omega, 3.0 / 16.0, g, fin)
        assert abs(rho - fin.sum()) < 1e-15
        assert abs(fout.sum() - fin.sum()) < 1e-14
        np.testing.assert_allclose(fout @ c, fin @ c + rho * g, atol=1e-15)
        # velocity with the force shift (Eq. nm-lbm-velocity)
        np.testing.assert_allclose(u, (fin @ c) / rho + 0.5 * g, atol=1e-16)


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_is_fixed_point_without_force(q):
    rng = np.random.default_rng(3)
    for collision in (0, 1):
        rho = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.05, 0.05, 3)
        f = feq(q, rho, u)
        fout, _, _ = collide(q, collision, 1.3, 3.0 / 16.0, np.zeros(3), f)
        np.testing.assert_allclose(fout, f, atol=2e-16)


@pytest.mark.parametrize("q", [19, 27])
def test_trt_reduces_to_srt(q):
    """TRT with Lambda = (1/omega - 1/2)^2 has omega- = omega+ and equals SRT."""
    rng = np.random.default_rng(4)
    _, w, _ = lattice(q)
    for _ in range(20):
        omega = rng.uniform(0.6, 1.9)
        lam = (1.0 / omega - 0.5) ** 2
        fin = w * rng.uniform(0.8, 1.2, q)
        g = rng.uniform(-1e-3, 1e-3, 3)
        a, _, _ = collide(q, 0, omega, lam, g, fin)
        b, _, _ = collide(q, 1, omega, lam, g, fin)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def test_srt_relaxation_rate_on_nonequilibrium():
    """Without force the non-equilibrium part decays by (1 - omega) per
    collision (SRT, Eq. nm-lbm-collision-operator with the sign of R1)."""
    q = 19
    rng = np.random.default_rng(5)
    _, w, _ = lattice(q)
    fin = w * rng.uniform(0.9, 1.1, q)
    omega = 1.4
    fout, rho, u = collide(q, 0, omega, 0.0, np.zeros(3), fin)
    fe = feq(q, rho, u)
    np.testing.assert_allclose(fout - fe, (1.0 - omega) * (fin - fe), atol=1e-16)
