"""Pins of the oracle's van der Waals thermodynamics (oracle/thermo.py).

Each closed form is checked against something other than itself: the general
definitions evaluated by finite differences of the EOS, numbers printed in the
paper, or textbook ideal-gas shock relations.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import thermo

GOLD = os.path.join(os.path.dirname(__file__), "golden")
A, B, R, CV = 3.0, 1.0 / 3.0, 8.0 / 3.0, 8.0     # reduced vdW, c_v/R = 3


def P_of(a, b, r):
    return lambda rho, T: thermo.pressure(rho, T, a, b, r)


@pytest.mark.parametrize("rho,T", [(0.3, 1.1), (0.6, 1.05), (1.0, 1.2), (1.8, 0.869), (0.54, 1.40)])
def test_sound_speed_closed_form_matches_definition(rho, T):
    """Eq. vdW_speed_of_sound against Eq. speed_of_sound by finite differences."""
    closed = thermo.sound_speed_sq(rho, T, A, B, R, CV)
    general = thermo.sound_speed_sq_general(P_of(A, B, R), rho, T, CV)
    assert abs(closed - general) <= 1e-8 * max(1.0, abs(closed))


@pytest.mark.parametrize("rho,T", [(0.3, 1.1), (0.6, 1.05), (1.0, 1.2), (1.8, 0.869)])
def test_cp_closed_form_matches_definition(rho, T):
    """Eq. cpvdW against c_v + T (dP/dT)_v (dv/dT)_P by finite differences."""
    closed = thermo.cp(rho, T, A, B, R, CV)
    general = thermo.cp_general(P_of(A, B, R), rho, T, CV)
    assert abs(closed - general) <= 1e-7 * abs(closed)


def test_ideal_gas_limits():
    """a = b = 0: c_s^2 = gamma R T and c_p = c_v + R (Sec. 4.1, ideal-gas limit)."""
    g = 1.0 + R / CV
    assert math.isclose(thermo.sound_speed_sq(0.7, 1.3, 0, 0, R, CV), g * R * 1.3, rel_tol=1e-15)
    assert math.isclose(thermo.cp(0.7, 1.3, 0, 0, R, CV), CV + R, rel_tol=1e-15)


def test_caloric_inversion_roundtrip():
    """Eq. lbm_temp inverts e = c_v T - a rho (Eq. de_vdW) with the kinetic part."""
    rng = np.random.default_rng(1)
    rho, T, u2 = rng.uniform(0.2, 2.0, 50), rng.uniform(0.5, 2.0, 50), rng.uniform(0, 0.3, 50)
    E = thermo.internal_energy(rho, T, A, CV) + 0.5 * u2
    assert np.allclose(thermo.temperature_from_energy(rho, E, u2, A, CV), T, rtol=1e-14)


def test_reduced_critical_point():
    """With R = 8/3, a = 3, b = 1/3 the critical point is rho = T = P = 1 (Sec. 2, a and b from critical data)."""
    crit = json.load(open(os.path.join(GOLD, "n2_critical.json")))
    Pc, Tc, rc = crit["P_c"], crit["T_c"], crit["rho_c"]
    Rg = Pc / (rc * Tc) * 8.0 / 3.0          # vdW critical compressibility 3/8 fixes R
    a = 27 * Rg ** 2 * Tc ** 2 / (64 * Pc)
    b = Rg * Tc / (8 * Pc)
    # reduced: a rho_c^2 / P_c = 3, b rho_c = 1/3
    assert math.isclose(a * rc * rc / Pc, 3.0, rel_tol=1e-12)
    assert math.isclose(b * rc, 1.0 / 3.0, rel_tol=1e-12)
    assert math.isclose(thermo.pressure(1.0, 1.0, A, B, R), 1.0, rel_tol=1e-14)
    h = 1e-4
    d1 = (thermo.pressure(1 + h, 1.0, A, B, R) - thermo.pressure(1 - h, 1.0, A, B, R)) / (2 * h)
    assert abs(d1) < 1e-7


def test_maxwell_matches_printed_coexistence():
    """Maxwell construction at T_r = 0.9 against the densities printed in Sec. 4.2.2."""
    gold = json.load(open(os.path.join(GOLD, "n2_coexistence.json")))
    rl, rv = thermo.maxwell_coexistence(gold["T_r"], A, B, R)
    tol = gold["printed_rounding_rel"]
    assert abs(rl / (gold["rho_l"] / gold["rho_c"]) - 1) < tol
    assert abs(rv / (gold["rho_v"] / gold["rho_c"]) - 1) < tol
    # equal pressure at the two densities
    assert math.isclose(thermo.pressure(rl, 0.9, A, B, R), thermo.pressure(rv, 0.9, A, B, R), rel_tol=1e-11)


def test_maxwell_equal_area():
    """Equal-area rule checked by quadrature of the isotherm P(v) between v_l and v_v."""
    T = 0.85
    rl, rv = thermo.maxwell_coexistence(T, A, B, R)
    Ps = thermo.pressure(rv, T, A, B, R)
    v = np.linspace(1 / rl, 1 / rv, 400001)
    area = np.trapezoid(thermo.pressure(1 / v, T, A, B, R) - Ps, v)
    assert abs(area) < 1e-8


@pytest.mark.parametrize("Ma", [1.2, 1.47, 2.0])
def test_rankine_hugoniot_ideal_gas_textbook(Ma):
    """a = b = 0: normal-shock density and pressure ratios of a perfect gas."""
    g = 1.0 + R / CV
    r2, T2, u2, us = thermo.rankine_hugoniot(1.0, 1.0, 0.0, Ma, 0.0, 0.0, R, CV)
    ratio_rho = (g + 1) * Ma ** 2 / ((g - 1) * Ma ** 2 + 2)
    ratio_P = 1 + 2 * g / (g + 1) * (Ma ** 2 - 1)
    assert math.isclose(r2, ratio_rho, rel_tol=1e-10)
    assert math.isclose(thermo.pressure(r2, T2, 0, 0, R, ) / thermo.pressure(1.0, 1.0, 0, 0, R), ratio_P, rel_tol=1e-10)
    assert math.isclose(us, Ma * math.sqrt(g * R), rel_tol=1e-14)


@pytest.mark.parametrize("Ma", [1.1, 1.3, 1.47])
def test_rankine_hugoniot_vdw_residuals(Ma):
    """vdW post-shock state satisfies the three jump conditions to round-off."""
    r2, T2, u2, us = thermo.rankine_hugoniot(0.3, 1.1, 0.0, Ma, A, B, R, CV)
    for res in thermo.rh_residuals(0.3, 1.1, 0.0, r2, T2, u2, us, A, B, R, CV):
        assert abs(res) < 1e-12
    assert r2 > 0.3 and u2 > 0.0
