"""Mass drift of the reduced-precision storage formats, attributed and closed.

The liquid mass (Eq. nm-fslbm-mass) is the sum of the stored PDFs of the
liquid cells plus the interface masses.  Streaming and bounce-back move
stored values unchanged and the mass exchange (Eq. nm-fslbm-mass-flux) is
summed in FP64 from stored values, so in exact arithmetic only the
collision could change it, and it conserves each cell's density.  With
rounding, every collision of a liquid cell stores q values whose sum
differs from the density it received.

Attribution (printed):
* bulk: a periodic all-liquid box with random velocities and gravity (no
  interface cells), where only the collision and its stores act;
* whole step: the standing gravity wave, which adds the interface band
  (exchange, conversion, excess mass);
for FP32 and FP16S deviation storage and for their mass-conserving forms
FP32MC / FP16SMC, whose rest PDF takes up the rounding of the others.

Bar: relative drift |M(t) - M(0)| / M(0) <= 1e-10 for the mass-conserving
formats on both cases (1000 steps) and on a batch of uneven cylindrical dam
breaks (D3Q27).  The gravity-wave amplitude of FP32MC stays within 1e-3 of
a(0) of the FP64 oracle's, the observable bar; that of FP16SMC is measured
and reported (at the size of FP16 rounding the observable itself moves by
0.15 a(0), test_oracle_physics.py::test_gravity_wave_observable_conditioning).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

STEPS = 1000
A0 = 0.32


def _box():
    n = 24
    N = n ** 3
    rng = np.random.default_rng(17)
    vel = rng.uniform(-0.03, 0.03, 3 * N)
    rho = 1.0 + rng.uniform(-5e-3, 5e-3, N)
    return S.Scenario("liquid_box", (n, n, n), (True, True, True), np.ones(N), np.full(N, S.LIQ, np.uint8),
                      vel, rho, q=19, omega=1.7, g=(1e-5, -2e-5, 0.0))


def _drift(sc, precision, steps=STEPS):
    from paper_2207_13962_gb300 import fslbm
    g = fslbm.context_for(sc, precision=precision)
    M0 = g.observables()["total_mass"]
    g.step(steps)
    obs = g.observables()
    g.close()
    assert obs["status"] == 0
    return abs(obs["total_mass"] - M0) / M0


def test_drift_attribution_and_mass_conserving_formats(gpu_lib):
    box, wave = _box(), S.gravity_wave(variant="OM")
    res = {}
    for prec in ("FP32", "FP32MC", "FP16S", "FP16SMC"):
        res[prec] = (_drift(box, prec), _drift(wave, prec))
        print(f"relative mass drift over {STEPS} steps, {prec}: bulk (liquid box) {res[prec][0]:.2e}, "
              f"whole step (gravity wave) {res[prec][1]:.2e}")
    for prec in ("FP32MC", "FP16SMC"):
        assert res[prec][0] <= 1e-10 and res[prec][1] <= 1e-10, (prec, res[prec])


def _amplitude(fill):
    return fill.reshape(64, 32)[:, 0].sum() - 32.0


@pytest.mark.parametrize("precision", ["FP32MC", "FP16SMC"])
def test_mass_conserving_formats_keep_the_observable(precision, gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    sc = S.gravity_wave(variant="OM")
    o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
    o.init(sc.fill, sc.flags, sc.velocity, sc.density)
    g = fslbm.context_for(sc, precision=precision)
    err = 0.0
    for _ in range(STEPS // 10):
        o.step(10)
        g.step(10)
        err = max(err, abs(_amplitude(g.read(pdf=False)["fill"]) - _amplitude(o.read()["fill"])) / A0)
    print(f"gravity wave OM {precision}: amplitude error {err:.3e} of a(0)")
    g.close()
    if precision == "FP32MC":
        assert err <= 1e-3, err
    elif err > 1e-3:
        pytest.xfail(f"{precision} amplitude error {err:.3e} of a(0): above the 1e-3 bar at FP16 rounding")


@pytest.mark.parametrize("precision", ["FP32MC", "FP16SMC"])
def test_batched_cylinders_conserve_mass(precision, gpu_lib):
    from paper_2207_13962_gb300 import fslbm
    Ls = [24, 31, 40, 17, 33]
    scs = [S.cylinder_dam_break(L=L, r_frac=0.2 + 0.04 * k, h_frac=0.35 - 0.03 * k, q=27, g=1e-4)
           for k, L in enumerate(Ls)]
    members = [fslbm.context_for(sc, precision=precision) for sc in scs]
    M0 = [m.observables()["total_mass"] for m in members]
    batch = fslbm.Batch(members)
    batch.step(300)
    st, _ = batch.sync()
    assert st == 0
    drift = [abs(m.observables()["total_mass"] - a) / a for m, a in zip(members, M0)]
    print(f"batched cylinders {precision}: max relative mass drift {max(drift):.2e} over 300 steps")
    assert max(drift) <= 1e-10, drift
    batch.close()
