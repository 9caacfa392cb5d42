"""Pins of the oracle's discrete attractors (oracle/lbm.py, Eqs. LBMeq..LBMgstar).

Checked against Table moments_fg / moments_fgstar of Appendix A, the exact
lattice defect of the diagonal third moment, and the textbook lattice weights
at rest with theta = 1/3.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import lbm

RNG = np.random.default_rng(7)


def rand_state(D):
    rho = RNG.uniform(0.3, 1.8)
    u = RNG.uniform(-0.2, 0.2, D)
    theta = RNG.uniform(0.1, 0.3)
    e = RNG.uniform(-0.5, 2.0)
    return rho, u, theta, e


def moment(p, c, *axes):
    w = np.ones(len(c))
    for a in axes:
        w = w * c[:, a]
    return float(np.dot(w, p))


@pytest.mark.parametrize("D", [2, 3])
def test_weights_at_rest(D):
    """u = 0, theta = 1/3: f^eq/rho are the D2Q9 / D3Q27 weights (2/3)^n0 (1/6)^(D-n0)."""
    c = lbm.velocities(D)
    f = lbm.f_equilibrium(1.0, [0.0] * D, [1.0 / 3.0] * D, c)
    for i, ci in enumerate(c):
        n0 = int(np.sum(ci == 0))
        w = Fraction(2, 3) ** n0 * Fraction(1, 6) ** (D - n0)
        assert abs(f[i] - float(w)) < 4e-16
    if D == 3:
        assert sorted(set(np.round(f, 15))) == sorted({round(8 / 27, 15), round(2 / 27, 15), round(1 / 54, 15), round(1 / 216, 15)})


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("trial", range(4))
def test_feq_moments(D, trial):
    """Table moments_fg, f^eq column, up to the off-diagonal third moments."""
    c = lbm.velocities(D)
    rho, u, theta, e = rand_state(D)
    P = rho * theta
    f = lbm.f_equilibrium(rho, list(u), [theta + ua * ua for ua in u], c)
    tol = 1e-14
    assert abs(f.sum() - rho) < tol
    for a in range(D):
        assert abs(moment(f, c, a) - rho * u[a]) < tol
        for b in range(D):
            want = rho * u[a] * u[b] + (P if a == b else 0.0)
            assert abs(moment(f, c, a, b) - want) < tol
            if a != b:
                # v_a^2 v_b: rho u_a^2 u_b + P u_b (Table moments_fg, third moments)
                assert abs(moment(f, c, a, a, b) - (rho * u[a] ** 2 * u[b] + P * u[b])) < tol
        # diagonal third moment: c^3 = c on the lattice, defect is -Lambda (Eq. correction)
        Lam = rho * u[a] ** 3 + 3 * rho * u[a] * (theta - 1.0 / 3.0)
        assert abs(moment(f, c, a, a, a) - (rho * u[a] ** 3 + 3 * P * u[a]) + Lam) < tol


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("trial", range(4))
def test_geq_moments(D, trial):
    """Table moments_fg, g^eq column: rho E, rho(E+P/rho)u, rho u u (E+2P/rho) + P(E+P/rho) delta."""
    c = lbm.velocities(D)
    rho, u, theta, e = rand_state(D)
    P = rho * theta
    E = e + 0.5 * float(np.dot(u, u))
    g = lbm.g_equilibrium(rho, list(u), theta, e, c)
    tol = 1e-13
    assert abs(g.sum() - rho * E) < tol
    for a in range(D):
        assert abs(moment(g, c, a) - rho * (E + P / rho) * u[a]) < tol
        for b in range(D):
            want = rho * u[a] * u[b] * (E + 2 * P / rho) + (P * (E + P / rho) if a == b else 0.0)
            assert abs(moment(g, c, a, b) - want) < tol


@pytest.mark.parametrize("D", [2, 3])
def test_star_moments(D):
    """f*: sum = rho, first = rho u*, diagonal second = rho(theta* + u*^2 + Phi).

    g*: sum = rho E + u.F when T* follows Eq. sh_T_1 (energy compensation,
    comment 5 of Sec. 3.1), first moment = that of g^eq at the star state + q^c.
    """
    c = lbm.velocities(D)
    rho, u, theta, e = rand_state(D)
    a_vdw, cv = 0.3, 8.0
    T = (e + a_vdw * rho) / cv
    F = RNG.uniform(-0.01, 0.01, D)
    Phi = RNG.uniform(-0.01, 0.01, D)
    qc = RNG.uniform(-0.01, 0.01, D)
    theta_s = theta * (1 + RNG.uniform(-0.05, 0.05))
    us = u + F / rho
    f = lbm.f_equilibrium(rho, list(us), [theta_s + us[a] ** 2 + Phi[a] for a in range(D)], c)
    assert abs(f.sum() - rho) < 1e-14
    for a in range(D):
        assert abs(moment(f, c, a) - rho * us[a]) < 1e-14
        assert abs(moment(f, c, a, a) - rho * (theta_s + us[a] ** 2 + Phi[a])) < 1e-14
    T_s = T - float(np.dot(F, F)) / (2 * rho * rho * cv)
    e_s = cv * T_s - a_vdw * rho
    g = lbm.g_equilibrium(rho, list(us), theta_s, e_s, c)
    for i, ci in enumerate(c):
        if int(np.sum(ci * ci)) == 1:
            g[i] += 0.5 * float(np.dot(ci, qc))
    E = e + 0.5 * float(np.dot(u, u))
    assert abs(g.sum() - (rho * E + float(np.dot(u, F)))) < 1e-13
    E_s = e_s + 0.5 * float(np.dot(us, us))
    for a in range(D):
        assert abs(moment(g, c, a) - (rho * us[a] * (E_s + theta_s) + qc[a])) < 1e-13


def test_velocity_order():
    """Lexicographic order over (c_x, c_y, c_z) with c_z fastest; rest node in the middle."""
    c = lbm.velocities(3)
    assert c.shape == (27, 3)
    assert list(c[0]) == [-1, -1, -1] and list(c[13]) == [0, 0, 0] and list(c[26]) == [1, 1, 1]
    assert list(c[1]) == [-1, -1, 0]
    assert [tuple(x) for x in c] == list(itertools.product((-1, 0, 1), repeat=3))
