"""Pins of the Peng-Robinson oracle (oracle/eos.py) and of the lattice step with it
(the general equation of state of Sec. 2, temperature from a non-linear caloric
relation).  What fixes them, independently of the module's closed forms:
  - the textbook Peng-Robinson critical constants: Z_c = 0.3074, Omega_a = 0.45724,
    Omega_b = 0.07780, and dP/drho = d2P/drho2 = 0 at the critical point (finite
    differences of P);
  - the caloric relation against a quadrature of the identity
    e = c_v T + int_0^rho (P - T dP/dT)/rho'^2 drho' with dP/dT by differences;
  - c_v(rho, T), (dP/dT)_rho, (dP/drho)_T, c_s^2, c_p against finite differences
    and the generic numerical routines of thermo;
  - the ideal-gas limit rho -> 0;
  - the Newton inversion: T(rho, e(rho, T)) = T;
  - the lattice step: a uniform moving state is a fixed point, mass, momentum and
    energy are conserved on a periodic box (kappa = 0), and a weak pressure step
    moves at the Peng-Robinson sound speed.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import inputs
from oracle import eos, lbm, thermo

A, B, R = eos.reduced_constants()
CV = 2.5 * R
M = eos.m_of_omega(0.0372)
PR = eos.PengRobinson(A, B, R, CV, 1.0, M)
STATES = [(0.3, 0.8), (0.6, 1.05), (1.0, 1.0), (1.7, 0.9), (2.2, 1.3)]


def test_critical_constants_match_textbook():
    assert abs(1.0 / R - 0.3074) < 1e-4                  # Z_c
    assert abs(A / R ** 2 - 0.45724) < 1e-5               # Omega_a
    assert abs(B / R - 0.07780) < 1e-5                    # Omega_b
    h = 1e-4
    p0, pp, pm = PR.pressure(1.0, 1.0), PR.pressure(1.0 + h, 1.0), PR.pressure(1.0 - h, 1.0)
    assert abs(p0 - 1.0) < 1e-12
    assert abs((pp - pm) / (2 * h)) < 1e-7
    assert abs((pp - 2 * p0 + pm) / h ** 2) < 1e-5
    assert PR.dPdrho(1.0, 0.95) < 0 < PR.dPdrho(1.0, 1.05)   # subcritical spinodal, supercritical stable


@pytest.mark.parametrize("rho,T", STATES)
def test_caloric_relation_against_quadrature(rho, T):
    h = 1e-6

    def integrand(r):
        dPdT = (PR.pressure(r, T + h) - PR.pressure(r, T - h)) / (2 * h)
        return (PR.pressure(r, T) - T * dPdT) / (r * r)
    dep, _ = quad(integrand, 1e-12, rho, epsabs=1e-12, epsrel=1e-10, limit=200)
    assert abs(PR.energy(rho, T) - (CV * T + dep)) < 1e-8


@pytest.mark.parametrize("rho,T", STATES)
def test_derivatives_against_differences(rho, T):
    h = 1e-6
    assert abs(PR.cv_real(rho, T) - (PR.energy(rho, T + h) - PR.energy(rho, T - h)) / (2 * h)) < 1e-6
    assert abs(PR.dPdT(rho, T) - (PR.pressure(rho, T + h) - PR.pressure(rho, T - h)) / (2 * h)) < 1e-6
    assert abs(PR.dPdrho(rho, T) - (PR.pressure(rho + h, T) - PR.pressure(rho - h, T)) / (2 * h)) < 1e-6
    cv = PR.cv_real(rho, T)
    assert abs(PR.sound_speed_sq(rho, T) - thermo.sound_speed_sq_general(PR.pressure, rho, T, cv)) < 1e-6
    if PR.dPdrho(rho, T) > 0.1:
        assert abs(PR.cp(rho, T) / thermo.cp_general(PR.pressure, rho, T, cv) - 1) < 1e-6


def test_ideal_gas_limit():
    rho, T = 1e-7, 1.3
    assert abs(PR.pressure(rho, T) / (rho * R * T) - 1) < 1e-6
    assert abs(PR.energy(rho, T) - CV * T) < 1e-6
    assert abs(PR.sound_speed_sq(rho, T) / (R * T * (1 + R / CV)) - 1) < 1e-6


def test_newton_inverts_the_caloric_relation():
    rho = np.array([s[0] for s in STATES] + [0.05, 2.5])
    T = np.array([s[1] for s in STATES] + [3.0, 0.7])
    assert np.abs(PR.temperature(rho, PR.energy(rho, T)) / T - 1).max() < 1e-14


def pr_model(shape, kappa=0.0, eta=1.0, nu=0.02):
    sc = inputs.scenario("tgv_pr_d3q27")
    e = dict(sc["eos"])
    e["kappa"], e["eta_over_mu"] = kappa, eta
    tau = nu * sc["rho0"] / lbm.eos_pr.PengRobinson(e["a"], e["b"], e["R"], sc["cv"], e["Tc"], e["m"]).pressure(
        sc["rho0"], sc["T0"])
    return lbm.Model(2, shape, e, tau, 0.71, sc["cv"]), sc


def test_lattice_uniform_moving_state_is_a_fixed_point():
    m, sc = pr_model((8, 5))
    shp = (5, 8)
    s = lbm.Sim(m, np.full(shp, sc["rho0"]), [np.full(shp, 0.1), np.full(shp, -0.05)], np.full(shp, sc["T0"]))
    F0 = s.fields()
    s.step(20)
    F = s.fields()
    assert np.abs(F["rho"] - F0["rho"]).max() < 1e-14
    assert np.abs(F["T"] - sc["T0"]).max() < 1e-13
    assert np.abs(F["u"][0] - 0.1).max() < 1e-14


def test_lattice_conserves_on_periodic_box():
    m, sc = pr_model((12, 9))
    shp = (9, 12)
    rng = inputs.uniform(3, 9 * 12).reshape(shp)
    s = lbm.Sim(m, sc["rho0"] * (1 + 0.01 * rng), [0.02 * rng, -0.01 * rng], sc["T0"] * (1 - 0.005 * rng))
    t0 = s.totals()
    s.step(30)
    t1 = s.totals()
    assert np.abs(np.asarray(t1) - np.asarray(t0)).max() < 1e-12 * abs(t0[0])


def test_lattice_sound_speed_is_peng_robinson():
    """A weak pressure box splits at each edge into an outgoing and an incoming wave of
    half the jump; the 3/4 level of the left edge rides the incoming one.  Its speed
    against the Peng-Robinson c_s (0.5%)."""
    Nx = 600
    m, sc = pr_model((Nx, 1), eta=1.0)
    rho0, T0 = sc["rho0"], sc["T0"]
    x = np.arange(Nx)[None, :]
    rho = np.where((x >= 150) & (x < 450), rho0 * (1 + 1e-3), rho0)
    s = lbm.Sim(m, rho, [np.zeros((1, Nx)), np.zeros((1, Nx))], np.full((1, Nx), T0))
    P0 = m.fluid.pressure(rho0, T0)
    lev = P0 + 0.75 * (m.fluid.pressure(rho0 * (1 + 1e-3), T0) - P0)

    def front():
        p = s.fields()["P"][0]
        for i in range(155, 445):
            if p[i - 1] < lev <= p[i]:
                return i - 1 + (lev - p[i - 1]) / (p[i] - p[i - 1])
        raise AssertionError("front not found")
    s.step(50)
    x1, t1 = front(), s.t
    s.step(80)
    x2, t2 = front(), s.t
    cs = np.sqrt(m.fluid.sound_speed_sq(rho0, T0))
    assert abs((x2 - x1) / (t2 - t1) / cs - 1) < 0.005
