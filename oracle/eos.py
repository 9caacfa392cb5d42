"""Peng-Robinson thermodynamics for the FP64 CPU oracle (a general equation of state
with a non-linear caloric relation: Sec. 2, the closing remark on Eq. lbm_temp).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package (and ``oracle/write_scenarios.py``).  The CUDA product path never imports
it and shares no code with it.

The paper names Peng-Robinson as the example of an equation of state whose
temperature must be recovered at each node from a non-linear caloric relation;
it gives no formulas.  This module writes out the textbook Peng-Robinson fluid
(Peng & Robinson 1976) in the paper's variables (mass density rho, specific gas
constant R, ideal-gas c_v constant):

  P = rho R T / (1 - b rho) - a alpha(T) rho^2 / (1 + 2 b rho - b^2 rho^2)
  alpha(T) = (1 + m (1 - sqrt(T / T_c)))^2

and derives everything else from it with the thermodynamic identities of Sec. 2:
  e = c_v T + int_0^rho (P - T dP/dT)/rho'^2 drho'    (caloric relation)
  c_s^2 = (dP/drho)_T + T (dP/dT)_rho^2 / (rho^2 c_v(rho, T))   (Eq. speed_of_sound)
  c_p - c_v = T (dP/dT)_rho^2 / (rho^2 (dP/drho)_T)
The departure integral has the closed form -(a alpha - T a alpha') L(rho) / (2 sqrt2 b),
L = ln((1 + (1 + sqrt2) b rho) / (1 + (1 - sqrt2) b rho)).  T(rho, e) solves
c_v T + e_dep(rho, T) = e by Newton's method: the left side increases with T
(its derivative is c_v(rho, T) > 0) and is concave in T (alpha'' > 0 and
(T alpha'')' < 0), so the iteration converges from any start.

Pins (tests/test_oracle_pr.py): the critical point of the reduced constants
(dP/drho = d2P/drho2 = 0, Z_c = 0.3074 of the textbook); e against a quadrature of
the identity; c_v, dP/dT, dP/drho, c_s^2, c_p against finite differences; the
ideal-gas limit; T(rho, e(rho, T)) = T.  All arithmetic is float64.
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def m_of_omega(omega):
    """Peng-Robinson slope of sqrt(alpha) in sqrt(T_r) from the acentric factor."""
    return 0.37464 + 1.54226 * omega - 0.26992 * omega * omega


class PengRobinson:
    """Peng-Robinson fluid with constants a, b, R, c_v (ideal part), T_c, m."""

    def __init__(self, a, b, R, cv, Tc, m):
        self.a, self.b, self.R, self.cv, self.Tc, self.m = a, b, R, cv, Tc, m

    # alpha(T) and its derivatives
    def _s(self, T):
        return 1.0 + self.m * (1.0 - np.sqrt(T / self.Tc))

    def alpha(self, T):
        return self._s(T) ** 2

    def dalpha(self, T):
        return -self.m * self._s(T) / np.sqrt(T * self.Tc)

    def d2alpha(self, T):
        return 0.5 * self.m / T * (self.m / self.Tc + self._s(T) / np.sqrt(T * self.Tc))

    def _D(self, rho):
        b = self.b
        return 1.0 + 2.0 * b * rho - b * b * rho * rho

    def _L(self, rho):
        b = self.b
        return np.log((1.0 + (1.0 + SQRT2) * b * rho) / (1.0 + (1.0 - SQRT2) * b * rho))

    def pressure(self, rho, T):
        return rho * self.R * T / (1.0 - self.b * rho) - self.a * self.alpha(T) * rho * rho / self._D(rho)

    def dPdT(self, rho, T):
        """(dP/dT) at fixed rho."""
        return rho * self.R / (1.0 - self.b * rho) - self.a * self.dalpha(T) * rho * rho / self._D(rho)

    def dPdrho(self, rho, T):
        """(dP/drho) at fixed T."""
        b = self.b
        D = self._D(rho)
        return self.R * T / (1.0 - b * rho) ** 2 - self.a * self.alpha(T) * 2.0 * rho * (1.0 + b * rho) / (D * D)

    def energy_departure(self, rho, T):
        """e - c_v T = int_0^rho (P - T dP/dT)/rho'^2 drho' (closed form)."""
        return (T * self.a * self.dalpha(T) - self.a * self.alpha(T)) * self._L(rho) / (2.0 * SQRT2 * self.b)

    def energy(self, rho, T):
        """Specific internal energy, zero for the ideal gas at T = 0."""
        return self.cv * T + self.energy_departure(rho, T)

    def cv_real(self, rho, T):
        """c_v(rho, T) = de/dT at fixed rho."""
        return self.cv + T * self.a * self.d2alpha(T) * self._L(rho) / (2.0 * SQRT2 * self.b)

    def sound_speed_sq(self, rho, T):
        """Eq. speed_of_sound for this fluid."""
        return self.dPdrho(rho, T) + T * self.dPdT(rho, T) ** 2 / (rho * rho * self.cv_real(rho, T))

    def cp(self, rho, T):
        return self.cv_real(rho, T) + T * self.dPdT(rho, T) ** 2 / (rho * rho * self.dPdrho(rho, T))

    def temperature(self, rho, e, tol=1e-15, itmax=60):
        """T with energy(rho, T) = e, by Newton's method from the temperature the
        departure at T_c would give (elementwise on arrays)."""
        rho = np.asarray(rho, dtype=np.float64)
        e = np.asarray(e, dtype=np.float64)
        T = (e - self.energy_departure(rho, self.Tc)) / self.cv
        T = np.maximum(T, 1e-3 * self.Tc)
        for _ in range(itmax):
            dT = (self.energy(rho, T) - e) / self.cv_real(rho, T)
            T = np.maximum(T - dT, 1e-3 * self.Tc)
            if np.all(np.abs(dT) <= tol * np.abs(T)):
                break
        return T

    def closure(self, rho, e):
        """(T, P, c_s^2) from (rho, e): the exact closure of the lattice step."""
        T = self.temperature(rho, e)
        return T, self.pressure(rho, T), self.sound_speed_sq(rho, T)


def reduced_constants(Zc_guess=0.3074):
    """(a, b, R) of the Peng-Robinson fluid with its critical point at rho = T = P = 1
    (T_c = 1, alpha(T_c) = 1): the roots of dP/drho = d2P/drho2 = 0 and P = 1 there,
    from the textbook constants as the starting point."""
    import warnings
    from scipy.optimize import fsolve
    R0 = 1.0 / Zc_guess
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)      # converged to rounding before xtol
        a, b, R = fsolve(_exact_critical, [0.45724 * R0 * R0, 0.0778 * R0, R0], xtol=1e-14)
    return float(a), float(b), float(R)


def _exact_critical(x):
    """Residuals of dP/drho = 0, d2P/drho2 = 0 and P = 1 at rho = T = 1 (alpha = 1)."""
    a, b, R = x
    rho = 1.0
    D = 1.0 + 2.0 * b * rho - b * b * rho * rho
    dP = R / (1.0 - b * rho) ** 2 - a * 2.0 * rho * (1.0 + b * rho) / (D * D)
    # d/drho [2 rho (1 + b rho) / D^2] = (2 + 4 b rho) / D^2 - 2 rho (1 + b rho) 2 D' / D^3, D' = 2b - 2b^2 rho
    Dp = 2.0 * b - 2.0 * b * b * rho
    d2P = 2.0 * b * R / (1.0 - b * rho) ** 3 - a * ((2.0 + 4.0 * b * rho) / (D * D)
                                                    - 4.0 * rho * (1.0 + b * rho) * Dp / D ** 3)
    P = R / (1.0 - b) - a / D
    return [dP, d2P, P - 1.0]
