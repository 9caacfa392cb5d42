"""van der Waals thermodynamics for the FP64 CPU oracle.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package (and ``oracle/write_scenarios.py``, which writes stored scalar
constants).  The CUDA product path never imports it and shares no code with it.

Every function cites the passage of Hosseini, Feinberg & Karlin,
"Lattice Boltzmann model for non-ideal compressible fluid dynamics"
(arXiv 2510.14712) that it writes out.  All arithmetic is float64.

Pins (tests/test_oracle_thermo.py): the closed-form sound speed and c_p are
checked against finite differences of the equation of state; the Maxwell
construction against the coexistence densities printed in Sec. 4.2.2; the
Rankine-Hugoniot solver against the textbook ideal-gas normal-shock ratios
and its own jump residuals.
"""
import math

import numpy as np


# ---------------------------------------------------------------------------
# Equation of state and caloric relation (Sec. 2)
# ---------------------------------------------------------------------------

def pressure(rho, T, a, b, R):
    """van der Waals pressure P = rho R T / (1 - b rho) - a rho^2 (Eq. Pvdw)."""
    return rho * R * T / (1.0 - b * rho) - a * rho * rho


def internal_energy(rho, T, a, cv):
    """Specific internal energy e = c_v T - a rho.

    Integral of de = c_v dT - a drho (Eq. de_vdW) with e = 0 at rho = T = 0.
    """
    return cv * T - a * rho


def temperature_from_energy(rho, E, u_sq, a, cv):
    """T = (E - |u|^2/2 + a rho) / c_v  (Eq. lbm_temp)."""
    return (E - 0.5 * u_sq + a * rho) / cv


def sound_speed_sq(rho, T, a, b, R, cv):
    """Adiabatic sound speed squared of the vdW fluid (Eq. vdW_speed_of_sound).

    c_s^2 = R T (1 + R/c_v) / (1 - b rho)^2 - 2 a rho.  Negative inside the
    spinodal, so callers use c_s^2, never c_s.
    """
    return R * T * (1.0 + R / cv) / (1.0 - b * rho) ** 2 - 2.0 * a * rho


def sound_speed_sq_general(P, rho, T, cv, h=1e-6):
    """Eq. speed_of_sound from numerical derivatives of a callable P(rho, T).

    c_s^2 = (dP/drho)_T + T/(rho^2 c_v) (dP/dT)_rho^2, with second-order
    central differences.  Used only to pin the closed form above.
    """
    dPdr = (P(rho + h, T) - P(rho - h, T)) / (2 * h)
    dPdT = (P(rho, T + h) - P(rho, T - h)) / (2 * h)
    return dPdr + T / (rho * rho * cv) * dPdT * dPdT


def cp(rho, T, a, b, R, cv):
    """Specific heat at constant pressure of the vdW fluid (Eq. cpvdW)."""
    return cv + R * R * T / (R * T - 2.0 * a * rho * (1.0 - b * rho) ** 2)


def cp_general(P, rho, T, cv, h=1e-6):
    """c_p = c_v + T (dP/dT)_v (dv/dT)_P from numerical derivatives (Sec. 4.1).

    (dv/dT)_P = -(dP/dT)_v / (dP/dv)_T and dP/dv = -rho^2 dP/drho.  Used only
    to pin the closed form above.
    """
    dPdr = (P(rho + h, T) - P(rho - h, T)) / (2 * h)
    dPdT = (P(rho, T + h) - P(rho, T - h)) / (2 * h)
    dPdv = -rho * rho * dPdr
    dvdT_P = -dPdT / dPdv
    return cv + T * dPdT * dvdT_P


def enthalpy(rho, T, a, b, R, cv):
    """Specific enthalpy h = e + P/rho (Eq. enthalpy)."""
    return internal_energy(rho, T, a, cv) + pressure(rho, T, a, b, R) / rho


def temperature_from_pressure(rho, P, a, b, R):
    """Invert Eq. Pvdw for T at given (rho, P); explicit because P is linear in T."""
    return (P + a * rho * rho) * (1.0 - b * rho) / (rho * R)


# ---------------------------------------------------------------------------
# Maxwell equal-area construction (Sec. 4.1 and 4.2.1)
# ---------------------------------------------------------------------------

def maxwell_coexistence(T, a, b, R, tol=1e-13):
    """Saturated liquid and vapour densities (rho_l, rho_v) at temperature T.

    Equal pressure and equal Gibbs free energy (equal area) on the vdW
    isotherm; solved by Newton's method on (ln rho_l, ln rho_v).  The
    chemical potential of the vdW fluid up to a T-only function is
    mu = R T [ln(rho/(1 - b rho)) + 1/(1 - b rho)] - 2 a rho.
    """
    def P(r):
        return pressure(r, T, a, b, R)

    def mu(r):
        return R * T * (math.log(r / (1.0 - b * r)) + 1.0 / (1.0 - b * r)) - 2.0 * a * r

    def dP(r):
        return R * T / (1.0 - b * r) ** 2 - 2.0 * a * r

    def dmu(r):
        return dP(r) / r

    # spinodal bracket: dP/drho = 0 gives the two spinodal densities
    grid = np.linspace(1e-6, 1.0 / b - 1e-6, 200001)
    dp = dP(grid)
    neg = np.nonzero(dp < 0)[0]
    if len(neg) == 0:
        raise ValueError("temperature is supercritical: no coexistence")
    r_sl, r_sh = grid[neg[0]], grid[neg[-1]]
    rl, rv = 0.5 * (r_sh + 1.0 / b), 0.5 * r_sl
    for _ in range(200):
        F1 = P(rl) - P(rv)
        F2 = mu(rl) - mu(rv)
        J = np.array([[dP(rl), -dP(rv)], [dmu(rl), -dmu(rv)]])
        d = np.linalg.solve(J, [-F1, -F2])
        lam = 1.0
        while True:
            nl, nv = rl + lam * d[0], rv + lam * d[1]
            if 0 < nv < r_sl and r_sh < nl < 1.0 / b:
                break
            lam *= 0.5
        rl, rv = nl, nv
        if abs(d[0]) < tol * rl and abs(d[1]) < tol * rv:
            break
    return rl, rv


# ---------------------------------------------------------------------------
# Rankine-Hugoniot post-shock state (Sec. 4.4)
# ---------------------------------------------------------------------------

def rankine_hugoniot(rho1, T1, u1, Ma, a, b, R, cv, tol=1e-14):
    """Post-shock state behind a right-running normal shock.

    The pre-shock state (rho1, T1, u1) lies on the right; the shock speed is
    u_s = u1 + Ma c_s(rho1, T1) (shock Mach number as in Sec. 4.4).  With
    w = u_s - u the velocity relative to the shock, the jump conditions are
        rho1 w1 = rho2 w2,
        P1 + rho1 w1^2 = P2 + rho2 w2^2,
        h1 + w1^2/2 = h2 + w2^2/2,
    solved for (rho2, T2) by Newton's method.  Returns (rho2, T2, u2, u_s).
    """
    cs1 = math.sqrt(sound_speed_sq(rho1, T1, a, b, R, cv))
    us = u1 + Ma * cs1
    w1 = us - u1
    m = rho1 * w1
    P1 = pressure(rho1, T1, a, b, R)
    h1 = enthalpy(rho1, T1, a, b, R, cv)

    def resid(x):
        r2, t2 = x
        w2 = m / r2
        return np.array([
            P1 + m * w1 - pressure(r2, t2, a, b, R) - m * w2,
            h1 + 0.5 * w1 * w1 - enthalpy(r2, t2, a, b, R, cv) - 0.5 * w2 * w2,
        ])

    # initial guess from the ideal-gas ratios with gamma = 1 + R/cv
    g = 1.0 + R / cv
    r2 = rho1 * (g + 1) * Ma * Ma / ((g - 1) * Ma * Ma + 2)
    t2 = T1 * (1.0 + 2 * g / (g + 1) * (Ma * Ma - 1)) * rho1 / r2
    x = np.array([r2, t2])
    for _ in range(100):
        F = resid(x)
        J = np.empty((2, 2))
        for k in range(2):
            hk = 1e-7 * max(1.0, abs(x[k]))
            xp = x.copy(); xp[k] += hk
            xm = x.copy(); xm[k] -= hk
            J[:, k] = (resid(xp) - resid(xm)) / (2 * hk)
        dx = np.linalg.solve(J, -F)
        x = x + dx
        if np.all(np.abs(dx) < tol * np.abs(x)):
            break
    r2, t2 = x
    u2 = us - m / r2
    return float(r2), float(t2), float(u2), float(us)


def rh_residuals(rho1, T1, u1, rho2, T2, u2, us, a, b, R, cv):
    """Relative residuals of the three jump conditions (mass, momentum, energy)."""
    w1, w2 = us - u1, us - u2
    P1, P2 = pressure(rho1, T1, a, b, R), pressure(rho2, T2, a, b, R)
    h1, h2 = enthalpy(rho1, T1, a, b, R, cv), enthalpy(rho2, T2, a, b, R, cv)
    r_mass = (rho1 * w1 - rho2 * w2) / (rho1 * w1)
    r_mom = (P1 + rho1 * w1 ** 2 - P2 - rho2 * w2 ** 2) / (P1 + rho1 * w1 ** 2)
    r_en = (h1 + 0.5 * w1 ** 2 - h2 - 0.5 * w2 ** 2) / (abs(h1) + 0.5 * w1 ** 2)
    return r_mass, r_mom, r_en
