"""Pins of the oracle's shock-capturing numerical transport (Sec. 4.4).

Each building block against an exact value (linear and polynomial fields,
rigid rotation, an isentrope), the whole step against the step without it,
and what it is for: planar shocks stay stable and keep the Rankine-Hugoniot
jump.
"""
import math

import numpy as np
import pytest

import inputs
import physics_cases as pc
from oracle import lbm, thermo


def grid2(nx=24, ny=20):
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    return x, y


def test_strain_rate_of_shear_and_rotation():
    x, y = grid2()
    gam = 0.013
    per = [False, False]
    S = lbm.strain_rate_magnitude([gam * y, 0 * x], 2, per)
    assert np.allclose(S[1:-1, 1:-1], gam / math.sqrt(2.0), rtol=1e-14)
    w = 0.021
    S = lbm.strain_rate_magnitude([-w * y, w * x], 2, per)          # rigid rotation: no strain
    assert np.abs(S[1:-1, 1:-1]).max() < 1e-16


def test_entropy_gradient_of_isothermal_ramp_and_isentrope():
    a, b, R, cv = 0.25, 1 / 3, 8 / 3, 8.0
    x, y = grid2()
    per = [False, True]
    T = 0.1 + 1e-4 * x
    rho = 0.4 + 0 * x
    G = lbm.entropy_gradient_magnitude(rho, T, b, R, cv, 2, per)
    assert np.allclose(G[:, 1:-1], cv * 1e-4 / T[:, 1:-1], rtol=1e-12)
    # along an isentrope of the vdW fluid, T (1/rho - b)^(R/c_v) = const: |grad s| is O(h^2)
    rho = 0.4 + 1e-3 * np.sin(2 * np.pi * x / 24)
    T = 0.1 * ((1 / 0.4 - b) / (1 / rho - b)) ** (R / cv)
    G = lbm.entropy_gradient_magnitude(rho, T, b, R, cv, 2, [True, True])
    G_ramp = R / (0.4 * (1 - b * 0.4)) * 1e-3 * 2 * np.pi / 24            # size of one term alone
    assert G.max() < 1e-3 * G_ramp


def test_fourth_difference_and_binomial_filter():
    x, y = grid2()
    per = [False, False]
    d = lbm.fourth_difference_norm(x ** 4 + 2 * y ** 4, 2, per)
    assert np.allclose(d[2:-2, 2:-2], math.hypot(24.0, 48.0), rtol=1e-12)
    assert np.abs(lbm.fourth_difference_norm(3 * x ** 3 - x * y + y ** 2, 2, per)[2:-2, 2:-2]).max() < 1e-9
    lin = 0.3 + 0.01 * x - 0.02 * y
    assert np.allclose(lbm.binomial_filter(lin, 2, per)[2:-2, 2:-2], lin[2:-2, 2:-2], rtol=1e-14)
    rng = inputs.uniform(4, 24 * 20).reshape(20, 24)
    f = lbm.binomial_filter(rng, 2, [True, True])
    assert abs(f.sum() - rng.sum()) < 1e-12                               # a normalised filter on a torus
    delta = np.zeros((20, 24))
    delta[10, 12] = 1.0
    w = np.array([1, 4, 6, 4, 1]) / 16.0
    assert np.allclose(lbm.binomial_filter(delta, 2, [True, True])[8:13, 10:15], np.outer(w, w), rtol=1e-14)


def coefficient_errors(transport):
    """Largest relative errors of (mu, eta, k)^num from `transport` against closed forms.

    The two fields have filtered fourth-difference norms that are known exactly.
    - u_x = c y^5/120, u_y = 0. The central-difference strain magnitude is
      S = c (y^4/24 + y^2/12 + 1/120) / sqrt2, a quartic in y. Its five-point fourth
      difference is c/sqrt2, a constant that the normalised filter keeps.
    - b = 0, uniform T, rho = exp(lam x^2 / 2). Then |grad s| = R e^(lam/2) sinh(lam x).
      The fourth difference multiplies sinh(lam x) by 16 sinh^4(lam/2), and the
      (1, 4, 6, 4, 1)/16 filter multiplies it by cosh^4(lam/2). Together that is
      R e^(lam/2) sinh^4(lam) sinh(lam x).
    c_s^2 is a given non-uniform field. Compared on the nodes at least six away from
    the clamped faces.
    """
    nx, ny = 24, 20
    x, y = grid2(nx, ny)
    c, lam, R, cv = 1e-3, 0.2, 8.0 / 3.0, 8.0
    rho = np.exp(lam * x * x / 2.0)
    u = [c * y ** 5 / 120.0, 0.0 * x]
    T = 0.1 + 0.0 * x
    cs2 = 0.2 + 0.05 * np.cos(0.3 * x + 0.2 * y)
    coef = (0.3, 0.7, 0.11)
    got = transport(rho, u, T, cs2, coef, 0.0, R, cv, 2, [False, False])
    s4 = c / math.sqrt(2.0)
    g4 = R * math.exp(lam / 2.0) * math.sinh(lam) ** 4 * np.sinh(lam * x)
    want = (rho * coef[0] * s4, rho * coef[1] * s4, rho * np.sqrt(cs2) * coef[2] * g4)
    inner = (slice(6, -6), slice(6, -6))
    return [float(np.abs(g[inner] / w[inner] - 1.0).max()) for g, w in zip(got, want)]


def test_coefficients_of_fields_with_known_filtered_norms():
    assert max(coefficient_errors(lbm.numerical_transport)) < 1e-9


def test_uniform_state_and_zero_coefficients_give_zero():
    sh = (6, 8)
    rho, T = 0.4 + np.zeros(sh), 0.1 + np.zeros(sh)
    u = [0.05 + np.zeros(sh), np.zeros(sh)]
    for coef in ((0.1, 0.5, 0.1), (0.0, 0.0, 0.0)):
        out = lbm.numerical_transport(rho, u, T, 0.3 + np.zeros(sh), coef, 1 / 3, 8 / 3, 8.0, 2, [True, True])
        assert all(np.abs(o).max() == 0.0 for o in out)


def _tube(sc_on, steps=60):
    c = inputs.add_noise(inputs.shock_drop(2, (96, 4), shock_x=30, with_drop=False, sc=_post_sc(1.2)), 2)
    m = lbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
    m.shock_capturing = sc_on
    s = lbm.Sim(m, c.rho, c.u, c.T).step(steps)
    return s.fields()


def test_zero_coefficients_reproduce_the_plain_step():
    a, b = _tube(None), _tube((0.0, 0.0, 0.0))
    for k in ("rho", "T"):
        assert np.allclose(a[k], b[k], rtol=1e-13, atol=0)


def test_first_step_uses_no_numerical_transport():
    """Coefficients of step t come from step t-1: the first collision is the plain one."""
    a, b = _tube(None, 1), _tube((0.5, 0.0, 0.5), 1)
    for k in ("rho", "T"):
        assert np.allclose(a[k], b[k], rtol=1e-13, atol=0)
    a, b = _tube(None, 3), _tube((0.5, 0.0, 0.5), 3)
    assert not np.allclose(a["T"], b["T"], rtol=1e-10, atol=0)


def test_shock_keeps_rankine_hugoniot_jump_with_shock_capturing():
    """P7 with the numerical transport on: it acts only in the shock, the plateau and speed stay."""
    speed, us, plateau, post = pc.shock_tube(Ma=1.3, shock_capturing=(0.1, 0.0, 0.1))
    assert abs(speed / us - 1) < 0.02
    for got, want in zip(plateau, post):
        assert abs(got / want - 1) < 0.01


def test_wide_strong_shock_is_stable_only_with_shock_capturing():
    """A Ma 1.3 planar shock 40 nodes wide: a transverse instability of the front blows
    the plain scheme up; with the numerical transport the run stays finite."""
    c = inputs.add_noise(inputs.shock_drop(2, (384, 40), shock_x=48, with_drop=False,
                                           sc=_post_sc(1.3)), 5)

    def run(coef, steps):
        m = lbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
        m.shock_capturing = coef
        s = lbm.Sim(m, c.rho, c.u, c.T)
        with np.errstate(all="ignore"):
            for _ in range(steps // 50):
                s.step(50)
                if not np.isfinite(s.fields()["rho"]).all():
                    return False
        return True
    assert run((0.1, 0.0, 0.1), 700)
    assert not run(None, 700)


def _post_sc(Ma):
    sc = dict(inputs.scenario("shock_drop_d2q9"))
    vap = sc["vapour"]
    e = sc["eos"]
    r2, T2, u2, us = thermo.rankine_hugoniot(vap["rho"], vap["T"], 0.0, Ma, e["a"], e["b"], e["R"], sc["cv"])
    sc["post"] = dict(rho=r2, T=T2, u=u2)
    return sc


@pytest.mark.parametrize("coef", [None, (0.3, 0.0, 0.3)])
def test_ma147_shock_at_the_larger_velocity_scale(coef):
    """The shock-drop workloads' Ma 1.47 shock on the U^2 = 16 velocity scale keeps the
    Rankine-Hugoniot plateau and speed, with and without the numerical transport."""
    speed, us, plateau, post = pc.shock_tube(Ma=1.47, Nx=600, steps=(100, 300), shock_capturing=coef,
                                             scenario="strong_shock_d2q9")
    assert abs(speed / us - 1) < 0.02
    for got, want in zip(plateau, post):
        assert abs(got / want - 1) < 0.01
