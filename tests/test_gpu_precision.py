"""Reduced-precision storage judged on observables against the FP64 oracle.

Workload: the standing gravity wave, 32 x 64 x 1, D3Q19 TRT, nu = 0.01,
g = 1e-5, interface y = 32 + 0.32 cos(2 pi x / 32), 1000 steps (Sec. 4.1).
Observable: the surface elevation at the crest column, a(t) = sum_j phi(0, j, t)
- 32, sampled every 10 steps; its error is max_t |a(t) - a_oracle(t)| / a(0)
with a(0) = 0.32.  Mass drift: |M(1000) - M(0)| / M(0) of the GPU run, with
M = sum of liquid PDFs + interface masses in FP64.

Bars:
* FP64 storage: the error is below 1e-12 (it is the parity mode).
* FP32 storage (deviations f - w_i, FP32 arithmetic): every variant within
  1e-3 relative (the stated observable bar), mass drift below 1e-10.
* FP16 / BF16 storage (deviations, FP32 arithmetic): the errors and the
  drift are measured and printed; the bound asserted is the format's own
  resolution, 2^-11 (FP16) / 2^-8 (BF16) of a(0) per step accumulated over a
  random walk of 1000 steps, i.e. sqrt(1000) x 2^-11 = 1.5e-2 and 0.12.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2207_13962_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

STEPS = 1000
EVERY = 10
A0 = 0.32
VARIANTS = ["NBRC", "NBKC", "OM", "OM3"]

_oracle_cache = {}


def _amplitude(fill):
    return fill.reshape(64, 32)[:, 0].sum() - 32.0


def _oracle_series(variant):
    if variant not in _oracle_cache:
        sc = S.gravity_wave(variant=variant)
        o = Oracle(*sc.shape, **S.make_oracle_kwargs(sc))
        o.init(sc.fill, sc.flags, sc.velocity, sc.density)
        a = [_amplitude(o.read()["fill"])]
        for _ in range(STEPS // EVERY):
            o.step(EVERY)
            a.append(_amplitude(o.read()["fill"]))
        _oracle_cache[variant] = np.array(a)
    return _oracle_cache[variant]


def _gpu_series(variant, precision):
    from paper_2207_13962_gb300 import fslbm
    sc = S.gravity_wave(variant=variant)
    g = fslbm.context_for(sc, precision=precision)
    M0 = g.observables()["total_mass"]
    a = [_amplitude(g.read(pdf=False)["fill"])]
    for _ in range(STEPS // EVERY):
        g.step(EVERY)
        a.append(_amplitude(g.read(pdf=False)["fill"]))
    obs = g.observables()
    g.close()
    assert obs["status"] == 0
    return np.array(a), abs(obs["total_mass"] - M0) / M0


def _errors(variant, precision):
    ao = _oracle_series(variant)
    ag, drift = _gpu_series(variant, precision)
    err = float(np.abs(ag - ao).max() / A0)
    print(f"gravity wave {variant} {precision}: amplitude error {err:.3e} of a(0), "
          f"mass drift {drift:.3e} over {STEPS} steps")
    return err, drift


def test_fp64_is_the_parity_mode(gpu_lib):
    err, drift = _errors("OM", "FP64")
    assert err < 1e-12 and drift < 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
def test_fp32_observables(variant, gpu_lib):
    err, drift = _errors(variant, "FP32")
    assert err <= 1e-3, err
    assert drift <= 1e-10, drift


@pytest.mark.parametrize("precision,bound", [("FP16S", 1.5e-2), ("BF16S", 0.12)])
def test_16bit_storage_observables(precision, bound, gpu_lib):
    err, drift = _errors("OM", precision)
    assert err <= bound, err
