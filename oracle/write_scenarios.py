"""Write inputs/scenarios.json: the scalar constants of every benchmark workload.

Run as ``python -m oracle.write_scenarios`` from the repository root.  It calls
only the oracle's thermodynamics (vdW EOS, sound speed, Rankine-Hugoniot), so
every stored number is an oracle output, never a CUDA-path output.  The field
builders in ``inputs/`` read these scalars and add geometry only.

Units.  The workloads are stated in reduced van der Waals units (rho_c = T_c =
P_c = 1, so R = 8/3, a = 3, b = 1/3; c_v/R = 3).  The lattice scheme is stable
only for theta = P/rho < 1/3 (Sec. 5), so velocities are rescaled by U: lattice
u = u_r / U, T = T_r / U^2, a = a_r / U^2, with rho, b, R, c_v unchanged.  U^2 is
the smallest integer with max(theta_r)/U^2 <= 1/4 over the states of the
workload.  Viscosities of the D2Q9 workloads are lattice values (their boxes
fix no reduced length); the Taylor-Green viscosity is a reduced value on the
[0, 2 pi)^3 box (see tgv).  mu = nu rho_ref and the stored relaxation time is
tau = mu / P(rho_ref, T_ref) (Sec. 3.1, tau = mu/P).
"""
import json
import math
import os

from . import thermo

A_R, B, R_GAS = 3.0, 1.0 / 3.0, 8.0 / 3.0
CV = 3.0 * R_GAS


def _theta_r(rho, T):
    return thermo.pressure(rho, T, A_R, B, R_GAS) / rho


def _u2_for(states):
    return float(math.ceil(max(_theta_r(r, t) for r, t in states) / 0.25))


def _lattice_eos(U2, kappa, eta_over_mu, rho_ref, T_ref_r):
    return dict(a=A_R / U2, b=B, R=R_GAS, kappa=kappa, eta_over_mu=eta_over_mu,
                rho_ref=rho_ref, T_ref=T_ref_r / U2)


def _tau(eos, nu):
    P = thermo.pressure(eos["rho_ref"], eos["T_ref"], eos["a"], eos["b"], eos["R"])
    return nu * eos["rho_ref"] / P


def _cs_lattice(rho, T_lat, eos):
    return math.sqrt(thermo.sound_speed_sq(rho, T_lat, eos["a"], eos["b"], eos["R"], CV))


def riemann():
    """D2Q9 non-ideal Riemann problem (left rho=1.0 T=1.2 | right rho=0.3 T=1.1)."""
    left, right = (1.0, 1.2), (0.3, 1.1)
    U2 = _u2_for([left, right])
    eos = _lattice_eos(U2, kappa=0.01, eta_over_mu=1.0, rho_ref=0.65, T_ref_r=1.15)
    return dict(D=2, U2=U2, cv=CV, Pr=0.71, nu=0.01, eos=eos, tau=_tau(eos, 0.01),
                left=dict(rho=left[0], T=left[1] / U2), right=dict(rho=right[0], T=right[1] / U2))


def couette(D, nu=0.2, rho=0.65, T_r=1.15, Ma=(0.8, 1.2, 1.6), Ma_transverse=0.5):
    """Thermal Couette flow (Sec. 4.1): a supercritical fluid at rest at (rho, T_w)
    between two isothermal walls, one sliding at U_w = Ma c_s.  The paper's runs:
    100 nodes, Pr in {0.6, 1.2, 4.9} at Ma 0.8 and Ma in {0.8, 1.2, 1.6} at Pr
    1.2, pseudo-one-dimensional.  Lattice viscosity nu (the channel width fixes
    the units).

    Velocity scale: the rule of strong_shock, U^2 the smallest integer with
    (theta_r + U_w,r^2) / U^2 <= 0.27, here for a wall at Ma_transverse.  The
    fluid next to a sliding wall moves with it, and with transverse structure
    (seeded noise, several nodes along y) a flow with theta + u^2 above about
    1/3 is unstable in this scheme (a seeded periodic box: stable at 0.28 and
    0.32, unstable at 0.34 and 0.35).  No integer scale brings the paper's
    Ma 1.6 wall below that with theta >= 0.1, so its runs stay
    pseudo-one-dimensional (one node along y), as the paper's case is: there
    the transverse populations stay on their node and no transverse mode
    exists."""
    cs_r = math.sqrt(thermo.sound_speed_sq(rho, T_r, A_R, B, R_GAS, CV))
    uw_r = Ma_transverse * cs_r
    U2 = float(math.ceil((_theta_r(rho, T_r) + uw_r * uw_r) / 0.27))
    eos = _lattice_eos(U2, kappa=0.01, eta_over_mu=1.0, rho_ref=rho, T_ref_r=T_r)
    cs = _cs_lattice(eos["rho_ref"], eos["T_ref"], eos)
    return dict(D=D, U2=U2, cv=CV, Pr=1.2, nu=nu, eos=eos, tau=_tau(eos, nu), cs=cs,
                rho=eos["rho_ref"], T_w=eos["T_ref"], Nx=100,
                Ma=list(Ma), Pr_runs=[0.6, 1.2, 4.9], Ma_transverse=Ma_transverse)


def _shock_drop(D, Ma, nu):
    vap = (0.3, 1.1)
    rho_d = 1.8
    P_v = thermo.pressure(vap[0], vap[1], A_R, B, R_GAS)
    T_d = thermo.temperature_from_pressure(rho_d, P_v, A_R, B, R_GAS)   # pressure match
    r2, T2, u2, us = thermo.rankine_hugoniot(vap[0], vap[1], 0.0, Ma, A_R, B, R_GAS, CV)
    U2 = _u2_for([vap, (rho_d, T_d), (r2, T2)])
    U = math.sqrt(U2)
    eos = _lattice_eos(U2, kappa=0.01, eta_over_mu=1.0, rho_ref=vap[0], T_ref_r=vap[1])
    return dict(D=D, U2=U2, cv=CV, Pr=0.71, nu=nu, eos=eos, tau=_tau(eos, nu), Ma=Ma,
                vapour=dict(rho=vap[0], T=vap[1] / U2),
                drop=dict(rho=rho_d, T=T_d / U2),
                post=dict(rho=r2, T=T2 / U2, u=u2 / U),
                shock_speed=us / U)


def shock_column(D, Tr=0.9, Ma=1.47, nu=0.01, kappa=0.01):
    """The paper's shock-liquid column (Sec. "Shock-liquid-column interaction"):
    saturated vapour and a saturated liquid column (or sphere) at T_r (Maxwell
    densities, one temperature), a Ma_s planar shock into the vapour with the
    Rankine-Hugoniot post-state.  t0_per_radius: the paper's time scale t0 =
    2 R c_s^v / (u_s c_s^l) sqrt(rho_l / rho_v) per node of radius R.

    The paper gives no lattice parameters; these are measured choices.
    - U^2: the liquid's sound speed is the largest signal speed (c_s^2 = 6.05
      reduced, theta 1.5 in the vapour).  A uniform liquid is unstable once
      c_s^2 / U^2 is about 0.5; a shocked 3-D sphere needs about 0.17 (U^2 = 25,
      0.24, ends at impact; U^2 = 35, 0.17, runs).  U^2 is the smallest integer
      with c_s^2(liquid) / U^2 <= 0.175, theta / U^2 <= 1/4 and (theta + u^2)
      (post) / U^2 <= 0.27 (U^2 = 35).
    - kappa = 0.01 lattice (0.35 reduced): a 2-D column at U^2 = 25 holds with
      0.02 and ends at impact with 0.05.
    - nu = 0.01 lattice (tau 0.23): in the liquid the explicit bulk shift
      (alpha about -15) enters with weight 2 tau / (2 tau + 1); tau 0.45 ends a
      4096 x 2048 run before impact.
    Run with shock capturing (C_mu = C_k = 0.3); without it the column ends within
    150 steps of impact."""
    rl, rv = thermo.maxwell_coexistence(Tr, A_R, B, R_GAS)
    r2, T2, u2, us = thermo.rankine_hugoniot(rv, Tr, 0.0, Ma, A_R, B, R_GAS, CV)
    cs2_l = thermo.sound_speed_sq(rl, Tr, A_R, B, R_GAS, CV)
    cs2_v = thermo.sound_speed_sq(rv, Tr, A_R, B, R_GAS, CV)
    U2 = float(max(math.ceil(cs2_l / 0.175), math.ceil((_theta_r(r2, T2) + u2 * u2) / 0.27),
                   _u2_for([(rl, Tr), (rv, Tr), (r2, T2)])))
    U = math.sqrt(U2)
    eos = _lattice_eos(U2, kappa=kappa, eta_over_mu=1.0, rho_ref=rv, T_ref_r=Tr)
    c_l, c_v = math.sqrt(cs2_l / U2), math.sqrt(cs2_v / U2)
    return dict(D=D, U2=U2, cv=CV, Pr=0.71, nu=nu, eos=eos, tau=_tau(eos, nu), Ma=Ma, T_r=Tr,
                vapour=dict(rho=rv, T=Tr / U2), drop=dict(rho=rl, T=Tr / U2),
                post=dict(rho=r2, T=T2 / U2, u=u2 / U), shock_speed=us / U, c_l=c_l, c_v=c_v,
                t0_per_radius=2.0 * c_v / (us / U * c_l) * math.sqrt(rl / rv),
                shock_capturing=[0.3, 0.0, 0.3])


def tgv(N=256, nu_reduced=1e-3):
    """D3Q27 compressible Taylor-Green vortex in dense vapour (rho0=0.6, T0=1.05, Ma 0.5).

    nu = 1e-3 is a reduced-unit viscosity like rho0 and T0, on the classic
    Taylor-Green box [0, 2 pi)^3: one lattice spacing is 2 pi / N reduced
    lengths and one lattice velocity unit is U reduced velocities, so
    nu_lattice = nu_reduced / (U 2 pi / N); Re = U0_r / nu_r = 747.  tau is
    stored for N = 256 and scales linearly with N at fixed Re.
    """
    rho0, T0 = 0.6, 1.05
    U2 = _u2_for([(rho0, T0)])
    # Stokes hypothesis (zero bulk viscosity), the usual choice for the
    # compressible Taylor-Green vortex; with eta/mu = 1 the explicit shift of
    # Eq. sh_temp_1 (alpha = -0.65 here) lets a symmetry-breaking mode grow
    # within ~200 steps at 128^3 and 256^3.
    eos = _lattice_eos(U2, kappa=0.01, eta_over_mu=0.0, rho_ref=rho0, T_ref_r=T0)
    cs = _cs_lattice(rho0, T0 / U2, eos)
    U0 = 0.5 * cs
    # T from Eq. Pvdw at constant rho0 is affine in P:
    #   T = T0 + dP (1 - b rho0)/(rho0 R),  dP = rho0 U0^2/16 (cos2x + cos2y)(cos2z + 2)
    T_amp = U0 * U0 * (1.0 - B * rho0) / (16.0 * R_GAS)
    nu_lat = nu_reduced / (math.sqrt(U2) * 2.0 * math.pi / N)
    return dict(D=3, U2=U2, cv=CV, Pr=0.71, nu_reduced=nu_reduced, N=N, nu=nu_lat, eos=eos,
                tau=_tau(eos, nu_lat), rho0=rho0, T0=T0 / U2, U0=U0, T_amp=T_amp, cs=cs,
                Re=0.5 * math.sqrt(thermo.sound_speed_sq(rho0, T0, A_R, B, R_GAS, CV)) / nu_reduced)


def tgv_pr(N=256, nu_reduced=1e-3, omega=0.0372, rho0=0.4, T0=1.05):
    """The compressible Taylor-Green vortex of tgv() in a Peng-Robinson fluid (the
    general-EOS case of Sec. 2: temperature from a non-linear caloric relation).

    Reduced units with the critical point at rho = T = P = 1 (oracle/eos.py,
    Z_c = 0.3074); acentric factor omega (nitrogen's), c_v = 2.5 R (a diatomic
    ideal part).  Mach number 0.5, Re and T0 1.05 as tgv(), density 0.4 (at 256^3
    in FP32 the van der Waals case's 0.6 ends within 125 steps in this fluid for
    every T0 tried, 1.05 to 1.4; 0.4 and 0.3 run 400 steps); Stokes hypothesis
    (eta/mu = 0).  Velocity scale: this fluid's sound speed is
    larger against theta than the van der Waals one's, so the rule of strong_shock
    sets U^2: (theta + U0^2) / U^2 <= 0.27 and theta / U^2 <= 1/4.  The
    temperature field gives the classical TGV pressure at constant density to first
    order: T = T0 + dP / (dP/dT)_rho, T_amp = rho0 U0^2 / (16 (dP/dT)_rho)."""
    from . import eos as eos_pr
    a_r, b_r, R_r = eos_pr.reduced_constants()
    m = eos_pr.m_of_omega(omega)
    cv = 2.5 * R_r
    pr = eos_pr.PengRobinson(a_r, b_r, R_r, cv, 1.0, m)
    th_r, U0_r = pr.pressure(rho0, T0) / rho0, 0.5 * math.sqrt(pr.sound_speed_sq(rho0, T0))
    U2 = float(max(math.ceil(th_r / 0.25), math.ceil((th_r + U0_r * U0_r) / 0.27)))
    eos = dict(kind="pr", a=a_r / U2, b=b_r, R=R_r, Tc=1.0 / U2, m=m, kappa=0.01, eta_over_mu=0.0,
               rho_ref=rho0, T_ref=T0 / U2)
    prl = eos_pr.PengRobinson(eos["a"], b_r, R_r, cv, eos["Tc"], m)
    cs = math.sqrt(prl.sound_speed_sq(rho0, T0 / U2))
    U0 = 0.5 * cs
    T_amp = rho0 * U0 * U0 / (16.0 * prl.dPdT(rho0, T0 / U2))
    nu_lat = nu_reduced / (math.sqrt(U2) * 2.0 * math.pi / N)
    tau = nu_lat * rho0 / prl.pressure(rho0, T0 / U2)
    return dict(D=3, U2=U2, cv=cv, Pr=0.71, nu_reduced=nu_reduced, N=N, nu=nu_lat, eos=eos, tau=tau, rho0=rho0,
                T0=T0 / U2, U0=U0, T_amp=T_amp, cs=cs, omega=omega,
                crit=dict(a=a_r, b=b_r, R=R_r))


def strong_shock(D, Ma=1.47, nu=0.01):
    """Planar Ma 1.47 shock into the supercritical vapour (rho 0.3, T 1.1), no drop.

    The velocity scale keeps the second moment of the equilibrium away from
    the lattice limit: U^2 is the smallest integer with
    max(theta_r + u_r^2) / U^2 <= 0.27 over the states (the rule of the other
    workloads, max theta_r / U^2 <= 1/4, leaves theta + u^2 = 0.35 behind a
    Ma 1.47 shock, where the scheme is unstable).  Run with shock capturing.
    """
    vap = (0.3, 1.1)
    r2, T2, u2, us = thermo.rankine_hugoniot(vap[0], vap[1], 0.0, Ma, A_R, B, R_GAS, CV)
    U2 = float(math.ceil(max(_theta_r(*vap), _theta_r(r2, T2) + u2 * u2) / 0.27))
    U = math.sqrt(U2)
    eos = _lattice_eos(U2, kappa=0.01, eta_over_mu=1.0, rho_ref=vap[0], T_ref_r=vap[1])
    return dict(D=D, U2=U2, cv=CV, Pr=0.71, nu=nu, eos=eos, tau=_tau(eos, nu), Ma=Ma,
                vapour=dict(rho=vap[0], T=vap[1] / U2),
                drop=dict(rho=1.8, T=thermo.temperature_from_pressure(1.8, thermo.pressure(*vap, A_R, B, R_GAS),
                                                                      A_R, B, R_GAS) / U2),
                post=dict(rho=r2, T=T2 / U2, u=u2 / U), shock_speed=us / U)


def strong_posts(n=13, Ma_lo=1.1, Ma_hi=1.5):
    """RH post-states of shocks Ma_lo .. Ma_hi into the vapour, in the lattice units of
    the strong_shock scenarios (U^2 = 16): the learned closure's training runs there."""
    sc = strong_shock(2)
    vap = (0.3, 1.1)
    U = math.sqrt(sc["U2"])
    out = []
    for k in range(n):
        Ma = Ma_lo + (Ma_hi - Ma_lo) * k / (n - 1)
        r2, T2, u2, us = thermo.rankine_hugoniot(vap[0], vap[1], 0.0, Ma, A_R, B, R_GAS, CV)
        out.append(dict(Ma=Ma, post=dict(rho=r2, T=T2 / sc["U2"], u=u2 / U)))
    return dict(base="strong_shock_d2q9", instances=out)


def batch(n=256, seed=2025, Ma_lo=1.1, Ma_hi=1.3):
    """Uneven D2Q9 shock-tube instances for the batched form.

    Nx uniform over the multiples of 64 in [128, 1024], Ny = Nx/2, shock Mach
    number uniform in [Ma_lo, Ma_hi], shock at x = Nx/8, vapour at rest ahead
    of it.  Draws come from the seeded generator of inputs/ (two streams);
    each Rankine-Hugoniot post-state is computed here.  Ma is capped at 1.3
    and no drop is placed: larger Ma and liquid drops need the shock-capturing
    viscosity of Sec. 4.4, which this build does not have.
    """
    import inputs
    sd = _shock_drop(2, 1.2, 0.01)
    vap = (0.3, 1.1)
    U = math.sqrt(sd["U2"])
    kx = inputs.uniform(seed, n)
    km = inputs.uniform(seed + 1, n)
    out = []
    for k in range(n):
        nx = 64 * (2 + min(14, int((kx[k] + 1.0) * 0.5 * 15)))
        Ma = Ma_lo + (Ma_hi - Ma_lo) * (km[k] + 1.0) * 0.5
        r2, T2, u2, us = thermo.rankine_hugoniot(vap[0], vap[1], 0.0, Ma, A_R, B, R_GAS, CV)
        out.append(dict(Nx=nx, Ny=nx // 2, Ma=Ma, shock_x=nx // 8,
                        post=dict(rho=r2, T=T2 / sd["U2"], u=u2 / U)))
    return dict(base="shock_drop_d2q9", instances=out)


def coexistence_key(T_r):
    """Table key of a reduced temperature: two decimals, three where needed (0.845)."""
    return "%.2f" % T_r if abs(round(T_r, 2) - T_r) < 1e-12 else "%.3f" % T_r


def coexistence(T_r=(0.85, 0.9, 0.95, 0.99), nu=0.01, kappa=0.1):
    """Flat liquid-vapour equilibria (Sec. "Liquid-vapour co-existence"): for each
    reduced temperature the Maxwell densities (the reference the paper compares
    with) and the lattice units of a slab of saturated liquid in its saturated
    vapour.  U^2 follows the liquid rule of shock_column (c_s^2(liquid) / U^2 <=
    0.175; theta / U^2 <= 1/4); lattice viscosity nu, kappa the default lattice
    capillarity (the interface spans about 2 sqrt(kappa / a) / sqrt(1 - T_r)
    nodes).  Below T_r = 27/32 the van der Waals pressure is negative inside the
    interface (the isotherm's minimum crosses zero there), so theta = P / rho and
    tau = mu / P are negative at the first step and the slab cannot run.  At 0.845
    (minimum interface pressure 0.010) a 256-node slab's relaxation, which lowers
    its temperature by about 1e-3, still reaches P <= 0; 0.85 (0.050) runs."""
    out = {}
    for Tr in T_r:
        rl, rv = thermo.maxwell_coexistence(Tr, A_R, B, R_GAS)
        cs2_l = thermo.sound_speed_sq(rl, Tr, A_R, B, R_GAS, CV)
        U2 = float(max(math.ceil(cs2_l / 0.175), _u2_for([(rl, Tr), (rv, Tr)])))
        eos = _lattice_eos(U2, kappa=kappa, eta_over_mu=1.0, rho_ref=rv, T_ref_r=Tr)
        out[coexistence_key(Tr)] = dict(U2=U2, eos=eos, tau=_tau(eos, nu), rho_l=rl, rho_v=rv, T=Tr / U2)
    return dict(D=2, cv=CV, Pr=0.71, nu=nu, T_r=list(T_r), states=out)


def batch_columns(n=256, seed=2027, Ma_lo=1.1, Ma_hi=1.5, r_lo=8, r_hi=64):
    """Uneven D2Q9 instances mixing shock tubes and shock-liquid columns for the
    batched form with shock capturing, in the fluid and units of column_d2q9
    (saturated vapour and liquid at T_r 0.9, U^2 = 35).

    Nx uniform over the multiples of 64 in [128, 1024], Ny = Nx/2, Ma uniform in
    [Ma_lo, Ma_hi], shock at x = Nx/8.  About half the instances hold a column
    centred at (Nx/4, Ny/2) with radius uniform in [r_lo, r_hi], capped so that it
    starts 2 nodes ahead of the shock and 4 nodes inside the y extent (radius 0:
    a plain tube).  Draws come from the seeded generator of inputs/ (four
    streams); each Rankine-Hugoniot post-state is computed here."""
    import inputs
    col = shock_column(2)
    U2 = col["U2"]
    U = math.sqrt(U2)
    Tr = col["T_r"]
    rv = col["vapour"]["rho"]
    kx, km, kd, kr = (inputs.uniform(seed + j, n) for j in range(4))
    out = []
    for k in range(n):
        nx = 64 * (2 + min(14, int((kx[k] + 1.0) * 0.5 * 15)))
        ny = nx // 2
        Ma = Ma_lo + (Ma_hi - Ma_lo) * (km[k] + 1.0) * 0.5
        r2, T2, u2, us = thermo.rankine_hugoniot(rv, Tr, 0.0, Ma, A_R, B, R_GAS, CV)
        radius = 0
        if kd[k] < 0.0:
            r = int(r_lo + (r_hi - r_lo) * (kr[k] + 1.0) * 0.5)
            radius = max(r_lo, min(r, nx // 4 - nx // 8 - 2, ny // 2 - 4))
        out.append(dict(Nx=nx, Ny=ny, Ma=Ma, shock_x=nx // 8, radius=radius,
                        post=dict(rho=r2, T=T2 / U2, u=u2 / U), shock_speed=us / U))
    return dict(base="column_d2q9", instances=out)


def main():
    out = dict(
        riemann_d2q9=riemann(),
        shock_drop_d2q9=_shock_drop(2, 1.47, 0.01),
        tgv_d3q27=tgv(),
        shock_drop_d3q27=_shock_drop(3, 1.47, 0.01),
        strong_shock_d2q9=strong_shock(2),
        strong_shock_d3q27=strong_shock(3),
        tgv_pr_d3q27=tgv_pr(),
        column_d2q9=shock_column(2),
        column_d3q27=shock_column(3),
        couette_d2q9=couette(2),
        couette_d3q27=couette(3),
    )
    bt = batch()
    # parity cases: smaller noise amplitude reference sound speed per scenario
    for k, sc in out.items():
        if "vapour" in sc:
            sc["cs_ref"] = _cs_lattice(sc["vapour"]["rho"], sc["vapour"]["T"], sc["eos"])
        elif "left" in sc:
            sc["cs_ref"] = _cs_lattice(sc["right"]["rho"], sc["right"]["T"], sc["eos"])
        else:
            sc["cs_ref"] = sc["cs"]
    out["batch_d2q9"] = bt
    out["batch_columns_d2q9"] = batch_columns()
    out["coexistence_d2q9"] = coexistence()
    out["strong_posts_d2q9"] = strong_posts()
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "inputs", "scenarios.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
