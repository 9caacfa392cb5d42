"""Plain FP64 CPU oracle of the non-ideal compressible lattice Boltzmann scheme.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA product path never imports it and shares no code, table or
helper with it.  It is slow on purpose: whole-grid numpy arrays, one array
expression per formula of the paper, no blocking, fusion or reordering.

Source: Hosseini, Feinberg & Karlin, "Lattice Boltzmann model for non-ideal
compressible fluid dynamics" (arXiv 2510.14712), Sec. 3.2 and the flow chart
of Fig. FlowChart.  One step, at every node:

 1. rho, j = sum c_i f_i, S = sum g_i                   (Eqs. def_h, def_u, def_E)
 2. Korteweg force F = kappa rho grad(lap rho)          (Eq. FK; central differences)
 3. u, E, T, P, theta, e, h, c_s^2, alpha, tau, beta    (Eqs. def_u, def_E, lbm_temp,
                                                         Pvdw, theta, corr_bulk, beta_main)
 4. div u, grad T, grad h (central); Phi (upwind)       (Sec. 3.2, Eq. correction)
 5. u*, theta*, T*, q^c                                 (Eqs. sh_vel_1, sh_temp_1,
                                                         sh_T_1, qc_1)
 6. f^eq, f*, g^eq, g*                                  (Eqs. LBMeq, LBMstar, LBMeqG,
                                                         LBMgstar)
 7. collide                                             (Eqs. fLBGK, gLBGK)
 8. boundary fill of the post-collision ghost nodes, then stream.

Readings of the paper taken here (each also listed in the design notes):
 * Phi keeps the -1/rho prefactor of Eq. correction; the upwind stencil of
   Sec. 3.2 gives the derivative only.  sgn(0) = 0 (central difference).
 * Lambda_a = rho u_a^3 + 3 rho u_a (theta - 1/3) (main text, not Appendix C).
 * g* carries no Phi term: g^eq at (u*, T*, theta*) plus (1/2) c_i.q^c on the
   |c_i|^2 = 1 directions only.
 * The Laplacian is the compact 2D+1-point stencil, then a central gradient.
 * mu = tau P(rho_ref, T_ref) and k/mu = c_p(rho_ref, T_ref)/Pr are constants;
   the local relaxation time is mu/P and beta = 1/(2 mu/P + 1).
 * Boundaries: y and z are periodic.  x is periodic, or closed by G = 4 ghost
   layers per face whose post-collision populations are refilled after every
   collision: an inflow face with the equilibrium of a prescribed state, an
   outflow face with a copy of the nearest interior layer (zero gradient).
   At start the primitive fields are extended to the ghosts by the same rule
   and every node, ghosts included, starts at equilibrium (Fig. FlowChart,
   "Initialize").
 * D2Q9 is the two-dimensional product form (D = 2 in alpha).

All quantities are lattice units (delta x = delta t = 1, lattice sound speed
squared 1/3).
"""
import itertools

import numpy as np

from . import eos as eos_pr
from . import thermo

CS2 = 1.0 / 3.0          # lattice speed of sound squared (Eq. cs)
GHOST = 4                # ghost layers per non-periodic x face


def velocities(D):
    """Discrete velocities c_i with components in {-1, 0, 1} (Eq. D3Q27c).

    Order: lexicographic over (c_x, c_y[, c_z]), the last component fastest.
    """
    return np.array(list(itertools.product((-1, 0, 1), repeat=D)), dtype=np.int64)


def psi(c, xi, zeta):
    """Product-form factor Psi(c; xi, zeta) of Eq. phi.

    1 - zeta for c = 0 and (zeta + c xi)/2 for c = +-1.
    """
    if c == 0:
        return 1.0 - zeta
    return 0.5 * (zeta + c * xi)


def chi(c, u, theta):
    """Psi(O, O^2) of Eq. phi applied to u^2/2 with O = theta d/du + u (Eq. Oa).

    O(u^2/2) = theta u + u^3/2 =: A and O^2(u^2/2) = theta^2 + (5/2) theta u^2
    + u^4/2 =: B, so the factor is u^2/2 - B for c = 0 and (B + c A)/2 for
    c = +-1.  Together with Psi(c; u, theta + u^2) acting on the constant e this
    spells out the generating-function construction of Eq. LBMeqG.
    """
    u2 = u * u
    A = theta * u + 0.5 * u2 * u
    B = theta * theta + 2.5 * theta * u2 + 0.5 * u2 * u2
    if c == 0:
        return 0.5 * u2 - B
    return 0.5 * (B + c * A)


def f_equilibrium(rho, u, zeta, c):
    """rho prod_a Psi(c_ia; u_a, zeta_a) for every i.

    With zeta_a = theta + u_a^2 this is f^eq (Eq. LBMeq); with the shifted
    arguments of Eqs. xistar/zetastar it is f* (Eq. LBMstar).
    """
    D = c.shape[1]
    tab = [{k: psi(k, u[a], zeta[a]) for k in (-1, 0, 1)} for a in range(D)]
    out = []
    for ci in c:
        p = rho * tab[0][ci[0]]
        for a in range(1, D):
            p = p * tab[a][ci[a]]
        out.append(p)
    return np.array(out)


def g_equilibrium(rho, u, theta, e, c):
    """g^eq(rho, u, T, theta) of Eq. LBMeqG, with e = e(rho, T).

    g_i = rho [ e prod_a psi_a + sum_b chi_b prod_{a != b} psi_a ] with
    psi_a = Psi(c_ia; u_a, theta + u_a^2) and chi_b = chi(c_ib; u_b, theta).
    """
    D = c.shape[1]
    ptab = [{k: psi(k, u[a], theta + u[a] * u[a]) for k in (-1, 0, 1)} for a in range(D)]
    ctab = [{k: chi(k, u[a], theta) for k in (-1, 0, 1)} for a in range(D)]
    out = []
    for ci in c:
        ps = [ptab[a][ci[a]] for a in range(D)]
        ch = [ctab[a][ci[a]] for a in range(D)]
        prod_all = ps[0]
        for a in range(1, D):
            prod_all = prod_all * ps[a]
        acc = e * prod_all
        for b in range(D):
            term = ch[b]
            for a in range(D):
                if a != b:
                    term = term * ps[a]
            acc = acc + term
        out.append(rho * acc)
    return np.array(out)


def first_moment(f, c, a):
    """sum_i c_ia f_i (Eqs. def_u, transform_u), summed over mirror pairs.

    Each direction with c_ia = +1 is paired with its mirror image in axis a
    (c_ia = -1, other components equal) and the sum runs over the differences
    f_i - f_mirror.  This is the same sum reassociated; it is exactly zero
    whenever the populations are mirror-symmetric, so that a state at rest
    has u = 0 exactly and the upwind stencil of Sec. 3.2 takes its sgn(0)
    (central) branch, as it does in exact arithmetic.
    """
    acc = np.zeros_like(f[0])
    for i, ci in enumerate(c):
        if ci[a] == 1:
            mirror = list(ci)
            mirror[a] = -1
            k = int(np.nonzero(np.all(c == np.array(mirror), axis=1))[0][0])
            acc = acc + (f[i] - f[k])
    return acc


def velocity(j, F, rho):
    """u = (sum c_i f_i + F/2) / rho (Eq. def_u with delta t = 1)."""
    return [(j[a] + 0.5 * F[a]) / rho for a in range(len(j))]


def bulk_shift(D, rho, cs2, P, eta_over_mu):
    """alpha = (D+2)/D - rho c_s^2 / P - eta/mu (Eq. corr_bulk)."""
    return (D + 2.0) / D - rho * cs2 / P - eta_over_mu


def shifted_temperature(T, F, rho, cv):
    """T* = T - F.F / (2 rho^2 c_v) (Eq. sh_T_1 with delta t = 1)."""
    FF = sum(Fa * Fa for Fa in F)
    return T - FF / (2.0 * rho * rho * cv)


def heat_flux_correction(P, gradh, gradT, k_over_mu):
    """q^c = P (grad h - (k/mu) grad T) (Eq. qc_1 with delta t = 1)."""
    return [P * (gh - k_over_mu * gT) for gh, gT in zip(gradh, gradT)]


def galilean_correction(m, rho, u, theta):
    """Phi_aa = -(1/rho) d_a Lambda_a with the upwind-biased stencil of Sec. 3.2.

    Lambda_a = rho u_a^3 + 3 rho u_a (theta - 1/3) (Eq. correction).  The
    stencil is the backward difference where u_a > 0, the forward difference
    where u_a < 0 and their mean (central) where u_a = 0.
    """
    Phi = []
    for a in range(m.D):
        Lam = rho * u[a] * u[a] * u[a] + 3.0 * rho * u[a] * (theta - CS2)
        back = Lam - m.nb(Lam, a, -1)
        fwd = m.nb(Lam, a, 1) - Lam
        sgn = np.sign(u[a])
        dLam = 0.5 * (1.0 + sgn) * back + 0.5 * (1.0 - sgn) * fwd
        Phi.append(-dLam / rho)
    return Phi


# ---------------------------------------------------------------------------
# Shock-capturing numerical transport coefficients (Sec. 4.4, Eqs. shock_cap,
# shock_cap_k), on interior fields.  Readings: r = 5, so the derivative in
# |grad^(r-1) .| is the fourth; it is the Euclidean norm of the per-axis
# five-point fourth differences; delta x^(r+1) = 1 in lattice units; the
# Gaussian filter is the separable binomial (1, 4, 6, 4, 1)/16 per axis (the
# paper gives no width); neighbours wrap on periodic axes and are clamped to
# the nearest interior node on non-periodic x faces.
# ---------------------------------------------------------------------------
def _shift(f, a, s, D, periodic):
    """Interior field f at x + s e_a (wrapped, or clamped on a non-periodic axis)."""
    ax = D - 1 - a
    if periodic:
        return np.roll(f, -s, axis=ax)
    n = f.shape[ax]
    idx = np.clip(np.arange(n) + s, 0, n - 1)
    return np.take(f, idx, axis=ax)


def strain_rate_magnitude(u, D, per):
    """S = |grad u + grad u^T| / 2 (Frobenius norm), central differences."""
    g = [[0.5 * (_shift(u[b], a, 1, D, per[a]) - _shift(u[b], a, -1, D, per[a])) for b in range(D)]
         for a in range(D)]
    return 0.5 * np.sqrt(sum((g[a][b] + g[b][a]) ** 2 for a in range(D) for b in range(D)))


def entropy_gradient_magnitude(rho, T, b, R, cv, D, per, fluid=None):
    """|grad s| with grad s = (c_v/T) grad T - R/(rho (1 - b rho)) grad rho (van der Waals);
    for another fluid (an object with cv_real and dPdT) the general form of the same
    identity, grad s = (c_v(rho, T)/T) grad T - (dP/dT)_rho / rho^2 grad rho."""
    gs = []
    for a in range(D):
        gT = 0.5 * (_shift(T, a, 1, D, per[a]) - _shift(T, a, -1, D, per[a]))
        gr = 0.5 * (_shift(rho, a, 1, D, per[a]) - _shift(rho, a, -1, D, per[a]))
        if fluid is None:
            gs.append(cv / T * gT - R / (rho * (1.0 - b * rho)) * gr)
        else:
            gs.append(fluid.cv_real(rho, T) / T * gT - fluid.dPdT(rho, T) / (rho * rho) * gr)
    return np.sqrt(sum(x * x for x in gs))


def fourth_difference_norm(f, D, per):
    """sqrt(sum_a (d_a^4 f)^2), d_a^4 the five-point fourth difference (1, -4, 6, -4, 1)."""
    acc = 0.0
    for a in range(D):
        d4 = (_shift(f, a, 2, D, per[a]) - 4.0 * _shift(f, a, 1, D, per[a]) + 6.0 * f
              - 4.0 * _shift(f, a, -1, D, per[a]) + _shift(f, a, -2, D, per[a]))
        acc = acc + d4 * d4
    return np.sqrt(acc)


def binomial_filter(f, D, per):
    """Separable (1, 4, 6, 4, 1)/16 filter along every axis."""
    for a in range(D):
        f = (_shift(f, a, -2, D, per[a]) + 4.0 * _shift(f, a, -1, D, per[a]) + 6.0 * f
             + 4.0 * _shift(f, a, 1, D, per[a]) + _shift(f, a, 2, D, per[a])) / 16.0
    return f


def numerical_transport(rho, u, T, cs2, coef, b, R, cv, D, per, fluid=None):
    """(mu, eta, k)^num = (rho C_mu F4(S), rho C_eta F4(S), rho c_s C_k F4(|grad s|)),
    F4 = filtered fourth-difference norm; c_s = sqrt(max(c_s^2, 0))."""
    C_mu, C_eta, C_k = coef
    s4 = binomial_filter(fourth_difference_norm(strain_rate_magnitude(u, D, per), D, per), D, per)
    g4 = binomial_filter(fourth_difference_norm(entropy_gradient_magnitude(rho, T, b, R, cv, D, per, fluid), D, per),
                         D, per)
    return rho * C_mu * s4, rho * C_eta * s4, rho * np.sqrt(np.maximum(cs2, 0.0)) * C_k * g4


class Model:
    """Constants of one run: lattice, vdW parameters, transport and boundaries.

    eos: dict with a, b, R (lattice units), kappa, eta_over_mu, rho_ref, T_ref, and
    optionally kind = "pr" with Tc and m: the Peng-Robinson fluid of oracle/eos.py
    (T_c and the slope m of sqrt(alpha)), whose temperature comes from its
    non-linear caloric relation (Sec. 2, closing remark on Eq. lbm_temp).  Its exact
    closure runs through the closure hook, and its sound speed and entropy
    gradient enter the shock capturing.
    x_low / x_high: "periodic", "outflow", ("inflow", (rho, u_vector, T)) or
    ("wall", (u_vector, T)): a wall moving with velocity u at temperature T
    (the thermal Couette flow of Sec. 4.1; the paper gives no wall scheme).
    Reading: diffuse reflection.  The wall re-emits the mass that reaches it
    from the first fluid layer with the equilibrium at (u_wall, T_wall): the
    ghost layers of a wall face hold s f^eq, s g^eq at (rho_e, u_wall, T_wall),
    rho_e the density of the first fluid node and s = (sum of its
    post-collision f that stream into the wall) / (sum of those f^eq that
    stream out of it).  f^eq is not linear in rho (theta = P/rho), so the
    shape is taken at rho_e and scaled: a wall at rest at the fluid's own
    state re-emits that state's equilibrium, and no mass crosses the wall.
    The Laplacian of the Korteweg force sees the wall as a symmetry plane
    (capillary_density): with the ghost layers' own density s rho_e in it, the
    flux-balance factor s feeds the capillary stencil and an odd-even mode
    grows from the wall.
    """

    def __init__(self, D, shape, eos, tau, Pr, cv, x_low="periodic", x_high="periodic"):
        self.D = D
        self.c = velocities(D)
        self.Q = len(self.c)
        self.shape = tuple(shape)             # interior (Nx, Ny[, Nz])
        self.a, self.b, self.R = float(eos["a"]), float(eos["b"]), float(eos["R"])
        self.cv = float(cv)
        self.kappa = float(eos["kappa"])
        self.eta_over_mu = float(eos["eta_over_mu"])
        rho_ref, T_ref = float(eos["rho_ref"]), float(eos["T_ref"])
        self.fluid = None
        if eos.get("kind", "vdw") == "pr":
            self.fluid = eos_pr.PengRobinson(self.a, self.b, self.R, self.cv, float(eos["Tc"]), float(eos["m"]))
            P_ref, cp_ref = self.fluid.pressure(rho_ref, T_ref), self.fluid.cp(rho_ref, T_ref)
        else:
            P_ref = thermo.pressure(rho_ref, T_ref, self.a, self.b, self.R)
            cp_ref = thermo.cp(rho_ref, T_ref, self.a, self.b, self.R, self.cv)
        # tau = mu/P (Sec. 3.1): the given tau fixes the constant mu at the reference state
        self.mu = float(tau) * P_ref
        # Eq. qc: k/mu from the Prandtl number Pr = mu c_p / k at the reference state
        self.k_over_mu = cp_ref / float(Pr)
        self.x_low, self.x_high = x_low, x_high
        # Optional thermodynamic closure (rho, e) -> (T, P, c_s^2) standing in
        # for Eqs. lbm_temp, Pvdw and vdW_speed_of_sound (a learned closure);
        # None: the exact van der Waals relations.  A Peng-Robinson fluid starts
        # with its exact closure (the Newton inversion of its caloric relation).
        self.closure = None if self.fluid is None else self.fluid.closure
        # Optional shock capturing (C_mu, C_eta, C_k) of Sec. 4.4: numerical
        # transport coefficients added to mu, eta, k; those of step t come from
        # the primitive fields of step t-1 (zero at the first step).  None: off.
        self.shock_capturing = None
        self.periodic_x = (x_low == "periodic")
        if (x_high == "periodic") != self.periodic_x:
            raise ValueError("x is periodic on both faces or on neither")
        self.G = 0 if self.periodic_x else GHOST

    # array axis of dimension alpha (x is the last array axis)
    def ax(self, alpha):
        return self.D - 1 - alpha

    def nb(self, q, alpha, s):
        """Value of field q at x + s e_alpha (periodic wrap of the padded array)."""
        return np.roll(q, -s, axis=self.ax(alpha))

    def padded_shape(self):
        nx = self.shape[0] + 2 * self.G
        return tuple(reversed((nx,) + self.shape[1:]))

    def interior(self):
        sl = [slice(None)] * self.D
        sl[self.ax(0)] = slice(self.G, self.G + self.shape[0])
        return tuple(sl)

    def state_eq(self, rho, u, T):
        """(f^eq, g^eq) at a primitive state (Fig. FlowChart, Initialize)."""
        if self.fluid is None:
            P = thermo.pressure(rho, T, self.a, self.b, self.R)
            e = thermo.internal_energy(rho, T, self.a, self.cv)
        else:
            P, e = self.fluid.pressure(rho, T), self.fluid.energy(rho, T)
        theta = P / rho                                   # Eq. theta
        zeta = [theta + ua * ua for ua in u]              # Eq. def_zeta_eq
        return (f_equilibrium(rho, u, zeta, self.c),
                g_equilibrium(rho, u, theta, e, self.c))


class Sim:
    """FP64 state of one run on the padded grid (pre-collision populations)."""

    def __init__(self, model, rho, u, T):
        """rho, T: arrays of the interior shape in array order ([z,] y, x);
        u: D arrays of that shape (u_x, u_y[, u_z])."""
        m = self.m = model
        rho = np.asarray(rho, dtype=np.float64)
        T = np.asarray(T, dtype=np.float64)
        u = [np.asarray(ua, dtype=np.float64) for ua in u]
        rho, u, T = self._extend(rho, u, T)
        self.f, self.g = m.state_eq(rho, u, T)
        self.t = 0
        self.visc = None           # numerical (mu, eta, k) on the interior for the next collision

    def _extend(self, rho, u, T):
        """Extend the initial primitive fields into the x ghost layers."""
        m = self.m
        if m.periodic_x:
            return rho, u, T
        ax, G = m.ax(0), m.G
        fields = [rho] + list(u) + [T]
        out = []
        for k, q in enumerate(fields):
            lo = self._ghost_prim(m.x_low, q, k, first=True)
            hi = self._ghost_prim(m.x_high, q, k, first=False)
            out.append(np.concatenate([lo] * G + [q] + [hi] * G, axis=ax))
        return out[0], out[1:-1], out[-1]

    def _ghost_prim(self, spec, q, k, first):
        m = self.m
        ax = m.ax(0)
        edge = np.take(q, [0 if first else -1], axis=ax)
        if spec == "outflow":
            return edge
        kind, state = spec
        if kind == "wall":
            u_w, T_w = state
            if k == 0:
                return edge                          # density: nearest interior node
            return np.full_like(edge, float((list(u_w) + [T_w])[k - 1]))
        rho_b, u_b, T_b = state
        val = ([rho_b] + list(u_b) + [T_b])[k]
        return np.full_like(edge, float(val))

    def capillary_density(self, rho):
        """Density seen by the Laplacian of the Korteweg force (Eq. FK): rho itself,
        except in the ghost layers of a wall face, which hold the mirror image of the
        fluid across the wall (ghost x = G - 1 - k takes fluid x = G + k): the wall
        is a symmetry plane of the capillary terms (neutral wetting)."""
        m = self.m
        walls = [(spec, lo) for spec, lo in ((m.x_low, True), (m.x_high, False))
                 if spec not in ("periodic", "outflow") and spec[0] == "wall"]
        if not walls:
            return rho
        ax, G, Nx = m.ax(0), m.G, m.shape[0]
        out = rho.copy()
        for spec, lo in walls:
            for k in range(G):
                xg, xs = (G - 1 - k, G + k) if lo else (G + Nx + k, G + Nx - 1 - k)
                dst = [slice(None)] * m.D
                src = [slice(None)] * m.D
                dst[ax], src[ax] = xg, xs
                out[tuple(dst)] = rho[tuple(src)]
        return out

    # -- flow chart steps 1-3 ------------------------------------------------
    def macroscopic(self, f=None, g=None):
        """rho, j, S (Eqs. def_h..def_E), F (Eq. FK), u, E, T (Eq. lbm_temp), P."""
        m = self.m
        f = self.f if f is None else f
        g = self.g if g is None else g
        D = m.D
        rho = f.sum(axis=0)                                           # Eq. def_h
        j = [first_moment(f, m.c, a) for a in range(D)]
        S = g.sum(axis=0)
        rk = self.capillary_density(rho)
        lap = sum(m.nb(rk, a, 1) - 2.0 * rk + m.nb(rk, a, -1) for a in range(D))
        F = [m.kappa * rho * 0.5 * (m.nb(lap, a, 1) - m.nb(lap, a, -1)) for a in range(D)]
        u = velocity(j, F, rho)                                        # Eq. def_u
        uF = sum(u[a] * F[a] for a in range(D))
        E = (S + 0.5 * uF) / rho                                       # Eq. def_E
        usq = sum(ua * ua for ua in u)
        if m.closure is None:
            T = thermo.temperature_from_energy(rho, E, usq, m.a, m.cv)    # Eq. lbm_temp
            P = thermo.pressure(rho, T, m.a, m.b, m.R)                    # Eq. Pvdw
            return dict(rho=rho, j=j, S=S, F=F, u=u, E=E, T=T, P=P, usq=usq, uF=uF)
        e = E - 0.5 * usq                                              # specific internal energy
        T, P, cs2 = m.closure(rho, e)
        return dict(rho=rho, j=j, S=S, F=F, u=u, E=E, T=T, P=P, usq=usq, uF=uF, e=e, cs2=cs2)

    # -- one time step -------------------------------------------------------
    def collide(self):
        """Steps 1-7: post-collision populations on the padded grid."""
        m = self.m
        D, c = m.D, m.c
        q = self.macroscopic()
        rho, u, F, T, P = q["rho"], q["u"], q["F"], q["T"], q["P"]
        theta = P / rho                                                # Eq. theta
        if m.closure is None:
            e = thermo.internal_energy(rho, T, m.a, m.cv)
            cs2 = thermo.sound_speed_sq(rho, T, m.a, m.b, m.R, m.cv)  # Eq. vdW_speed_of_sound
        else:
            e, cs2 = q["e"], q["cs2"]
        h = e + P / rho                                                # Eq. enthalpy
        if m.shock_capturing is None:
            alpha = bulk_shift(D, rho, cs2, P, m.eta_over_mu)          # Eq. corr_bulk
            tau = m.mu / P                                             # tau = mu / P
            k_over_mu = m.k_over_mu
        else:
            # effective coefficients {mu, eta, k} + {mu, eta, k}^num (Sec. 4.4)
            I = m.interior()
            num = [np.zeros_like(rho) for _ in range(3)]
            if self.visc is not None:
                for k in range(3):
                    num[k][I] = self.visc[k]
            mu_e = m.mu + num[0]
            eta_e = m.eta_over_mu * m.mu + num[1]
            k_e = m.k_over_mu * m.mu + num[2]
            alpha = bulk_shift(D, rho, cs2, P, eta_e / mu_e)           # Eq. corr_bulk
            tau = mu_e / P
            k_over_mu = k_e / mu_e
            per = [m.periodic_x] + [True] * (D - 1)
            # c_s of k^num: the van der Waals sound speed at (rho, T), whatever the closure
            if m.fluid is None:
                cs2_vdw = thermo.sound_speed_sq(rho[I], T[I], m.a, m.b, m.R, m.cv)
            else:
                cs2_vdw = m.fluid.sound_speed_sq(rho[I], T[I])
            self.visc = numerical_transport(rho[I], [ua[I] for ua in u], T[I], cs2_vdw, m.shock_capturing,
                                            m.b, m.R, m.cv, D, per, m.fluid)
        beta = 1.0 / (2.0 * tau + 1.0)                                 # Eq. beta_main

        # step 4: derivatives (central; upwind for Phi)
        div_u = sum(0.5 * (m.nb(u[a], a, 1) - m.nb(u[a], a, -1)) for a in range(D))
        gradT = [0.5 * (m.nb(T, a, 1) - m.nb(T, a, -1)) for a in range(D)]
        gradh = [0.5 * (m.nb(h, a, 1) - m.nb(h, a, -1)) for a in range(D)]
        Phi = galilean_correction(m, rho, u, theta)                    # Eq. correction

        # step 5: shifted state
        ustar = [u[a] + F[a] / rho for a in range(D)]                  # Eq. sh_vel_1
        theta_s = theta + alpha * theta * div_u                        # Eq. sh_temp_1
        if m.closure is None:
            T_s = shifted_temperature(T, F, rho, m.cv)                 # Eq. sh_T_1
            e_s = thermo.internal_energy(rho, T_s, m.a, m.cv)
        else:
            # Eq. sh_T_1 in energy form (e linear in T at fixed rho): e* = e - |F|^2/(2 rho^2)
            e_s = e - 0.5 * sum(F[a] * F[a] for a in range(D)) / (rho * rho)
        qc = heat_flux_correction(P, gradh, gradT, k_over_mu)          # Eq. qc_1

        # step 6: attractors
        feq = f_equilibrium(rho, u, [theta + u[a] * u[a] for a in range(D)], c)          # Eq. LBMeq
        fst = f_equilibrium(rho, ustar,
                            [theta_s + ustar[a] * ustar[a] + Phi[a] for a in range(D)], c)  # Eq. LBMstar
        geq = g_equilibrium(rho, u, theta, e, c)                                       # Eq. LBMeqG
        gst = g_equilibrium(rho, ustar, theta_s, e_s, c)                               # Eq. LBMgstar
        for i, ci in enumerate(c):
            if int(np.sum(ci * ci)) == 1:
                gst[i] = gst[i] + 0.5 * sum(ci[a] * qc[a] for a in range(D))

        # step 7: collision (Eqs. fLBGK, gLBGK)
        fpost = self.f + 2.0 * beta * (feq - self.f) + (1.0 - beta) * (fst - feq)
        gpost = self.g + 2.0 * beta * (geq - self.g) + (1.0 - beta) * (gst - geq)
        return fpost, gpost

    def wall_emission(self, fpost, src, sign, u_w, T_w):
        """Ghost (f, g) of a diffuse-reflection wall next to fluid layer src: the
        equilibrium at (rho_e, u_w, T_w) of that layer's density rho_e, scaled so
        that the f it streams out of the wall (c_x = -sign) carry the mass of the
        layer's post-collision f that stream into it (c_x = sign)."""
        m = self.m
        ax = m.ax(0) + 1
        layer = np.take(fpost, src, axis=ax)                     # [Q, transverse...]
        rho_e = layer.sum(axis=0)
        fb, gb = m.state_eq(rho_e, [np.full_like(rho_e, float(x)) for x in u_w],
                            np.full_like(rho_e, float(T_w)))
        into = sum(layer[i] for i, ci in enumerate(m.c) if ci[0] == sign)
        out = sum(fb[i] for i, ci in enumerate(m.c) if ci[0] == -sign)
        s = into / out
        return fb * s, gb * s

    def fill_ghosts(self, p, which, fpost=None):
        """Refill the x ghost layers of post-collision populations p (f or g); wall faces
        take their density from the post-collision f (fpost, or p itself for f)."""
        m = self.m
        if m.periodic_x:
            return
        G, Nx = m.G, m.shape[0]
        ax = m.ax(0) + 1                       # +1: leading population axis
        for spec, ghosts, src, sign in ((m.x_low, range(0, G), G, -1),
                                        (m.x_high, range(G + Nx, 2 * G + Nx), G + Nx - 1, 1)):
            if spec != "outflow" and spec[0] == "wall":
                u_w, T_w = spec[1]
                fb, gb = self.wall_emission(p if fpost is None else fpost, src, sign, u_w, T_w)
                val = fb if which == "f" else gb
                for xg in ghosts:
                    dst = [slice(None)] * (m.D + 1)
                    dst[ax] = xg
                    p[tuple(dst)] = val
                continue
            for xg in ghosts:
                dst = [slice(None)] * (m.D + 1)
                dst[ax] = xg
                if spec == "outflow":
                    srcs = [slice(None)] * (m.D + 1)
                    srcs[ax] = src
                    p[tuple(dst)] = p[tuple(srcs)]
                else:
                    _, (rho_b, u_b, T_b) = spec
                    fb, gb = m.state_eq(np.float64(rho_b), [np.float64(x) for x in u_b],
                                        np.float64(T_b))
                    val = fb if which == "f" else gb
                    shape = [m.Q] + [1] * (m.D - 1)
                    p[tuple(dst)] = val.reshape(shape)

    def stream(self, p):
        """p_i(x) <- p_i(x - c_i) on the padded grid (left-hand sides of Eq. fLBGK)."""
        m = self.m
        axes = tuple(m.ax(a) for a in range(m.D))
        out = np.empty_like(p)
        for i, ci in enumerate(m.c):
            out[i] = np.roll(p[i], shift=tuple(int(s) for s in ci), axis=axes)
        return out

    def step(self, n=1):
        for _ in range(n):
            fpost, gpost = self.collide()
            self.fill_ghosts(gpost, "g", fpost)      # before f: a wall's density comes from fpost
            self.fill_ghosts(fpost, "f")
            self.f = self.stream(fpost)
            self.g = self.stream(gpost)
            self.t += 1
        return self

    # -- outputs ---------------------------------------------------------------
    def fields(self):
        """Interior rho, u (list of D arrays), T, P, E from the current state."""
        q = self.macroscopic()
        I = self.m.interior()
        return dict(rho=q["rho"][I], u=[ua[I] for ua in q["u"]], T=q["T"][I],
                    P=q["P"][I], E=q["E"][I])

    def totals(self):
        """Interior sums of rho, rho u (= j + F/2) and rho E (= S + u.F/2)."""
        q = self.macroscopic()
        I = self.m.interior()
        mass = q["rho"][I].sum()
        mom = [(q["rho"] * q["u"][a])[I].sum() for a in range(self.m.D)]
        energy = (q["rho"] * q["E"])[I].sum()
        return np.array([mass] + mom + [energy])
