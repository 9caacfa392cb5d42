"""What FP32 can reach on the parity cases, from the oracle itself (no GPU).

The FP32 bound of the parity tests is a relative L2 error of 1e-5 on rho, u
and T against the FP64 oracle.  These tests evaluate the oracle's own step
with FP32 rounding and measure how far that lands from the FP64 oracle:

* FP32 storage with exact arithmetic (the populations rounded to float32
  after every step) stays near 1e-6 on the D2Q9 Riemann problem (1000 steps)
  and a Ma 1.2 D2Q9 shock tube (300 steps): storing the state in FP32 is not
  what limits FP32 runs.
* The whole step in float32 arithmetic (the oracle run with float32 state
  and constants) misses 1e-5 in u on the shock tube for one of three noise
  seeds: plain FP32 arithmetic does not meet the bar on shock cases, whatever
  the implementation, so their GPU parity tests use 5e-5.
* The temperature of Eq. lbm_temp, T = (E - |u|^2/2 + a rho)/c_v, evaluated in
  FP64 from the float32 moments (the mixed-precision form of the FP32 kernels,
  lbm_set_temperature_fp64) is no systematic gain: it lowers the shock tube's
  error in T about threefold, and raises rho's about twofold on a drifting
  Taylor-Green box (1000 steps).  The error of an FP32 trajectory is set by
  rounding throughout the step, not by the inversion alone.
"""
import numpy as np
import pytest

import inputs
from fp32_eval import errors, run, shock_case, tgv_drift_case
from oracle import thermo


def t_fp64(rho, E, u_sq, a, cv):
    """Eq. lbm_temp in FP64 from float32 inputs, rounded once to float32."""
    d = np.float64
    return ((np.asarray(E, d) - 0.5 * np.asarray(u_sq, d) + float(a) * np.asarray(rho, d)) / float(cv)).astype(
        np.asarray(rho).dtype)


@pytest.fixture(scope="module")
def shock_refs():
    return {seed: run(shock_case(seed), 300) for seed in (3, 4, 5)}


def test_fp32_storage_alone_is_not_the_limit(shock_refs):
    want = run(inputs.riemann(), 1000)
    e = errors(run(inputs.riemann(), 1000, "store32"), want)
    assert max(e.values()) < 2e-6, e
    e = errors(run(shock_case(3), 300, "store32"), shock_refs[3])
    assert max(e.values()) < 2e-6, e


def test_plain_fp32_arithmetic_misses_the_bar_on_shocks(shock_refs):
    eu = [errors(run(shock_case(s), 300, "fp32"), shock_refs[s])["u"] for s in (3, 4, 5)]
    assert max(eu) >= 1e-5, eu              # one seed misses 1e-5 with plain FP32 arithmetic
    assert max(eu) < 2e-5, eu


def test_fp64_temperature_inversion_is_no_systematic_gain(shock_refs, monkeypatch):
    plain = {s: errors(run(shock_case(s), 300, "fp32"), shock_refs[s]) for s in (3, 4, 5)}
    tgv_ref = run(tgv_drift_case(), 1000)
    tgv_plain = errors(run(tgv_drift_case(), 1000, "fp32"), tgv_ref)
    monkeypatch.setattr(thermo, "temperature_from_energy", t_fp64)
    mixed = {s: errors(run(shock_case(s), 300, "fp32"), shock_refs[s]) for s in (3, 4, 5)}
    tgv_mixed = errors(run(tgv_drift_case(), 1000, "fp32"), tgv_ref)
    mean = lambda d, k: np.mean([d[s][k] for s in d])
    assert mean(mixed, "T") < 0.5 * mean(plain, "T"), (plain, mixed)        # shock tubes: better
    assert tgv_mixed["rho"] > 1.5 * tgv_plain["rho"], (tgv_plain, tgv_mixed)  # drifting vortex: worse
