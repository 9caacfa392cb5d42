"""Small oracle experiments whose outcome the paper fixes in closed form.

Used by tests/test_oracle_physics.py (pins P3-P7) and by
tests/test_oracle_planted.py (each planted mistake must break one of them).
All runs are D2Q9 pseudo-one-dimensional (Nx x 1, periodic unless stated)
in the dense-vapour state of the Taylor-Green workload (rho0 = 0.6,
T0 = 1.05 reduced), lattice units.
"""
import math

import numpy as np

from oracle import lbm, thermo
import inputs

SC = inputs.scenario("tgv_d3q27")
EOS = dict(SC["eos"])
CV = SC["cv"]
RHO0, T0 = SC["rho0"], SC["T0"]
A, B, R = EOS["a"], EOS["b"], EOS["R"]
P0 = thermo.pressure(RHO0, T0, A, B, R)
CS = math.sqrt(thermo.sound_speed_sq(RHO0, T0, A, B, R, CV))


def model(Nx, nu, Pr=0.71, eta=1.0, kappa=0.0):
    e = dict(EOS, kappa=kappa, eta_over_mu=eta, rho_ref=RHO0, T_ref=T0)
    return lbm.Model(2, (Nx, 1), e, tau=nu * RHO0 / P0, Pr=Pr, cv=CV)


def fourier_amp(q, L):
    x = np.arange(L)
    return math.hypot(2 * np.mean(q * np.sin(2 * np.pi * x / L)),
                      2 * np.mean(q * np.cos(2 * np.pi * x / L)))


def shear_decay(May, L=64, nu=0.02):
    """Measured kinematic viscosity from u_y = Ma_y c_s + 0.01 c_s sin(2 pi x/L) (Sec. 4.1)."""
    m = model(L, nu)
    x = np.arange(L)[None, :]
    uy = May * CS + 0.01 * CS * np.sin(2 * np.pi * x / L)
    s = lbm.Sim(m, np.full((1, L), RHO0), [np.zeros((1, L)), uy], np.full((1, L), T0))
    ts, amps = [], []
    for _ in range(24):
        uy_now = s.fields()["u"][1][0]
        ts.append(s.t)
        amps.append(fourier_amp(uy_now - uy_now.mean(), L))
        s.step(20)
    slope = np.polyfit(ts[3:], np.log(amps[3:]), 1)[0]
    return -slope * L * L / (4 * np.pi ** 2), m.mu / RHO0


def sound_speed(Nx=800, nu=0.02, u0=0.0):
    """Front speed of a weak pressure step (Sec. 4.1), returns (measured, c_s + u0)."""
    m = model(Nx, nu)
    x = np.arange(Nx)[None, :]
    rho = np.where((x >= 200) & (x < 600), RHO0 * (1 + 1e-3), RHO0)
    dP = thermo.pressure(RHO0 * (1 + 1e-3), T0, A, B, R) - P0
    s = lbm.Sim(m, rho, [np.full((1, Nx), u0), np.zeros((1, Nx))], np.full((1, Nx), T0))
    lev = P0 + 0.75 * dP

    def front():
        p = s.fields()["P"][0]
        for i in range(205, 595):
            if p[i - 1] < lev <= p[i]:
                return i - 1 + (lev - p[i - 1]) / (p[i] - p[i - 1])
        raise AssertionError("front not found")

    s.step(60)
    x1, t1 = front(), s.t
    s.step(100)
    x2, t2 = front(), s.t
    return (x2 - x1) / (t2 - t1), CS + u0


def thermal_decay(L=64, nu=0.02, Pr=0.71):
    """Entropic-mode decay at constant pressure (Sec. 4.1): returns (measured, k/(rho0 c_p))."""
    m = model(L, nu, Pr=Pr)
    x = np.arange(L)[None, :]
    rho = RHO0 * (1 + 1e-3 * np.sin(2 * np.pi * x / L))
    T = thermo.temperature_from_pressure(rho, P0, A, B, R)
    s = lbm.Sim(m, rho, [np.zeros((1, L))] * 2, T)
    ts, amps = [], []
    for _ in range(50):
        Tn = s.fields()["T"][0]
        ts.append(s.t)
        amps.append(fourier_amp(Tn - Tn.mean(), L))
        s.step(10)
    chi = -np.polyfit(ts[10:], np.log(amps[10:]), 1)[0] * L * L / (4 * np.pi ** 2)
    cp0 = thermo.cp(RHO0, T0, A, B, R, CV)
    return chi, m.mu * m.k_over_mu / (RHO0 * cp0)


def acoustic_decay(L=64, nu=0.02, eta=1.0, Max=0.0):
    """Acoustic-energy decay rate sigma of a standing wave (Sec. 4.1).

    Initial isentropic perturbation dP sin(2 pi x/L) with drho = dP/c_s^2 and
    dT = T R/(c_v rho (1 - b rho)) drho (ds = 0 in Eq. ds_vdW).  Returns
    (measured, 2(D-1)/D mu/rho + eta/rho + k/(rho c_p)(c_p/c_v - 1)) with D = 2.
    A background flow u_x = Max c_s (as in the paper's runs) leaves sigma unchanged.
    """
    m = model(L, nu, eta=eta)
    x = np.arange(L)[None, :]
    dP = 1e-4 * P0 * np.sin(2 * np.pi * x / L)
    drho = dP / CS ** 2
    dT = T0 * R / (CV * RHO0 * (1 - B * RHO0)) * drho
    u0 = Max * CS
    s = lbm.Sim(m, RHO0 + drho, [np.full((1, L), u0), np.zeros((1, L))], T0 + dT)
    ts, Es = [], []
    for _ in range(80):
        F = s.fields()
        u = F["u"][0][0] - u0
        r = F["rho"][0] - RHO0
        ts.append(s.t)
        Es.append(0.5 * np.sum(RHO0 * u * u + r * r * CS * CS / RHO0))
        s.step(5)
    sig = -np.polyfit(ts[10:], np.log(Es[10:]), 1)[0] * L * L / (4 * np.pi ** 2)
    cp0 = thermo.cp(RHO0, T0, A, B, R, CV)
    k = m.mu * m.k_over_mu
    theory = (2 * (2 - 1) / 2) * m.mu / RHO0 + eta * m.mu / RHO0 + k / (RHO0 * cp0) * (cp0 / CV - 1)
    return sig, theory


def shock_tube(Ma=1.2, Nx=400, steps=(100, 250), shock_capturing=None, scenario="shock_drop_d2q9"):
    """Planar shock from the Rankine-Hugoniot post-state into vapour at rest (Sec. 4.4 states).

    Returns (speed measured, speed RH, plateau (rho, u, T) measured, RH post-state).
    """
    sc = inputs.scenario(scenario)
    eos = dict(sc["eos"])
    vap = sc["vapour"]
    r2, T2, u2, us = thermo.rankine_hugoniot(vap["rho"], vap["T"], 0.0, Ma,
                                             eos["a"], eos["b"], eos["R"], sc["cv"])
    m = lbm.Model(2, (Nx, 1), eos, sc["tau"], sc["Pr"], sc["cv"],
                  x_low=("inflow", (r2, [u2, 0.0], T2)), x_high="outflow")
    m.shock_capturing = shock_capturing
    x = np.arange(Nx)[None, :]
    behind = x < 50
    rho = np.where(behind, r2, vap["rho"])
    T = np.where(behind, T2, vap["T"])
    u = [np.where(behind, u2, 0.0), np.zeros((1, Nx))]
    s = lbm.Sim(m, rho, u, T)
    mid = 0.5 * (r2 + vap["rho"])

    def pos():
        r = s.fields()["rho"][0]
        for i in range(Nx - 1, 0, -1):
            if r[i - 1] >= mid > r[i]:
                return i - 1 + (r[i - 1] - mid) / (r[i - 1] - r[i])
        raise AssertionError("shock not found")

    s.step(steps[0])
    x1 = pos()
    s.step(steps[1] - steps[0])
    x2 = pos()
    F = s.fields()
    lo, hi = 20, int(x2) - 40
    plateau = (F["rho"][0, lo:hi].mean(), F["u"][0][0, lo:hi].mean(), F["T"][0, lo:hi].mean())
    return (x2 - x1) / (steps[1] - steps[0]), us, plateau, (r2, u2, T2)


def wall_channel(Nx=24, Ma=0.0, Pr=0.71, nu=0.2, perturb=0.0, moving="high"):
    """D2Q9 channel between two walls at T_w (the riemann_d2q9 fluid at rho_ref, T_w =
    T_ref), one node in y, the `moving` wall ("high" or "low") sliding along y at
    U_w = Ma c_s.  Initial state at rest at T_w with rho = rho_ref (1 + perturb sin x).
    Returns (Sim, U_w, rho_ref, T_w)."""
    sc = inputs.scenario("riemann_d2q9")
    eos = dict(sc["eos"])
    rho0, T_w = eos["rho_ref"], eos["T_ref"]
    cs = math.sqrt(thermo.sound_speed_sq(rho0, T_w, eos["a"], eos["b"], eos["R"], sc["cv"]))
    U_w = Ma * cs
    tau = nu * rho0 / thermo.pressure(rho0, T_w, eos["a"], eos["b"], eos["R"])
    lo = ("wall", ([0.0, U_w if moving == "low" else 0.0], T_w))
    hi = ("wall", ([0.0, U_w if moving == "high" else 0.0], T_w))
    m = lbm.Model(2, (Nx, 1), eos, tau, Pr, sc["cv"], x_low=lo, x_high=hi)
    rho = rho0 * (1.0 + perturb * np.sin(np.arange(Nx, dtype=float)))[None, :]
    s = lbm.Sim(m, rho, [np.zeros((1, Nx)), np.zeros((1, Nx))], np.full((1, Nx), T_w))
    return s, U_w, rho0, T_w


def wall_channel(Nx=24, Ma=0.0, Pr=0.71, nu=0.2, perturb=0.0, moving="high"):
    """D2Q9 channel between two walls at T_w (the couette_d2q9 fluid at rho_ref, T_w =
    T_ref), one node in y, the `moving` wall ("high" or "low") sliding along y at
    U_w = Ma c_s.  Initial state at rest at T_w with rho = rho_ref (1 + perturb sin x).
    Returns (Sim, U_w, rho_ref, T_w)."""
    sc = inputs.scenario("couette_d2q9")
    eos = dict(sc["eos"])
    rho0, T_w = eos["rho_ref"], eos["T_ref"]
    cs = math.sqrt(thermo.sound_speed_sq(rho0, T_w, eos["a"], eos["b"], eos["R"], sc["cv"]))
    U_w = Ma * cs
    tau = nu * rho0 / thermo.pressure(rho0, T_w, eos["a"], eos["b"], eos["R"])
    lo = ("wall", ([0.0, U_w if moving == "low" else 0.0], T_w))
    hi = ("wall", ([0.0, U_w if moving == "high" else 0.0], T_w))
    m = lbm.Model(2, (Nx, 1), eos, tau, Pr, sc["cv"], x_low=lo, x_high=hi)
    rho = rho0 * (1.0 + perturb * np.sin(np.arange(Nx, dtype=float)))[None, :]
    s = lbm.Sim(m, rho, [np.zeros((1, Nx)), np.zeros((1, Nx))], np.full((1, Nx), T_w))
    return s, U_w, rho0, T_w


def thermal_couette(Nx=24, Ma=0.5, Pr=0.71, nu=0.2, steps=6000):
    """Thermal Couette flow (Sec. 4.1): walls at both x faces at T_w, the upper one moving
    with U_w = Ma c_s along y; D2Q9, one node in y.  Returns (x, u_y, T, rho, U_w, T_w, mu, k)
    of the final state."""
    s, U_w, _, T_w = wall_channel(Nx, Ma, Pr, nu)
    s.step(steps)
    F = s.fields()
    m = s.m
    return np.arange(Nx, dtype=float), F["u"][1][0], F["T"][0], F["rho"][0], U_w, T_w, m.mu, m.k_over_mu * m.mu
