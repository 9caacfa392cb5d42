"""Planted mistakes: each plausible slip in the oracle must break at least one pin.

The mistake is planted in the oracle (monkeypatched on the CPU) and the pin
that should catch it is asserted to fail.
"""
import numpy as np
import pytest

from oracle import lbm
import physics_cases as pc  # noqa: E402
import test_oracle_step as st


def test_dropping_phi_breaks_galilean_invariance(monkeypatch):
    monkeypatch.setattr(lbm, "galilean_correction", lambda m, rho, u, theta: [0.0 * rho] * m.D)
    sig, want = pc.acoustic_decay(Max=0.4)
    assert abs(sig / want - 1) > 0.03


def upwind_dependence(galilean_correction):
    """Phi at x with u_x > 0 (< 0) must not see Lambda at x + 1 (x - 1) (Sec. 3.2 upwinding)."""
    m = lbm.Model(2, (9, 1), pc.EOS, tau=0.05, Pr=0.71, cv=pc.CV)
    rho = np.full((1, 9), pc.RHO0)
    theta = np.full((1, 9), 0.2)
    for sign in (1.0, -1.0):
        u = [np.full((1, 9), 0.1 * sign), np.zeros((1, 9))]
        base = galilean_correction(m, rho, u, theta)[0][0, 4]
        u2 = [u[0].copy(), u[1]]
        u2[0][0, 4 + int(sign)] *= 1.5          # changes Lambda downstream only
        assert galilean_correction(m, rho, u2, theta)[0][0, 4] == base


def test_upwind_pin_holds():
    upwind_dependence(lbm.galilean_correction)


def test_flipping_upwind_direction_is_caught(monkeypatch):
    def downwind(m, rho, u, theta):
        Phi = []
        for a in range(m.D):
            Lam = rho * u[a] ** 3 + 3.0 * rho * u[a] * (theta - lbm.CS2)
            back, fwd = Lam - m.nb(Lam, a, -1), m.nb(Lam, a, 1) - Lam
            sgn = -np.sign(u[a])
            Phi.append(-(0.5 * (1 + sgn) * back + 0.5 * (1 - sgn) * fwd) / rho)
        return Phi
    with pytest.raises(AssertionError):
        upwind_dependence(downwind)


def test_dropping_heat_flux_correction_breaks_thermal_pin(monkeypatch):
    monkeypatch.setattr(lbm, "heat_flux_correction", lambda P, gh, gT, k: [0.0 * P for _ in gh])
    chi, want = pc.thermal_decay()
    assert abs(chi / want - 1) > 0.03


def test_alpha_zero_breaks_acoustic_pin(monkeypatch):
    monkeypatch.setattr(lbm, "bulk_shift", lambda D, rho, cs2, P, e: 0.0 * rho)
    sig, want = pc.acoustic_decay()
    assert abs(sig / want - 1) > 0.03


def test_sign_of_eta_term_breaks_acoustic_pin(monkeypatch):
    monkeypatch.setattr(lbm, "bulk_shift", lambda D, rho, cs2, P, e: (D + 2.0) / D - rho * cs2 / P + e)
    sig, want = pc.acoustic_decay()
    assert abs(sig / want - 1) > 0.03


def test_dropping_energy_compensation_breaks_identity(monkeypatch):
    monkeypatch.setattr(lbm, "shifted_temperature", lambda T, F, rho, cv: T)
    with pytest.raises(AssertionError):
        st.test_moment_identities_with_korteweg(2, (12, 9))


def test_dropping_half_force_in_velocity_breaks_identity(monkeypatch):
    monkeypatch.setattr(lbm, "velocity", lambda j, F, rho: [j[a] / rho for a in range(len(j))])
    with pytest.raises(AssertionError):
        st.test_moment_identities_with_korteweg(2, (12, 9))


def test_transposed_chi_breaks_geq_moments(monkeypatch):
    orig = lbm.chi
    monkeypatch.setattr(lbm, "chi", lambda c, u, theta: orig(-c, u, theta))
    import test_oracle_equilibria as te
    with pytest.raises(AssertionError):
        te.test_geq_moments(3, 0)


def test_wrong_psi_rest_factor_breaks_weights(monkeypatch):
    orig = lbm.psi
    monkeypatch.setattr(lbm, "psi", lambda c, xi, zeta: 1.0 - 0.5 * zeta if c == 0 else orig(c, xi, zeta))
    import test_oracle_equilibria as te
    with pytest.raises(AssertionError):
        te.test_weights_at_rest(3)


def unit_density_emission(self, fpost, src, sign, u_w, T_w):
    """Wall re-emitting at rho_w = into / (outgoing f^eq at unit density): f^eq is not
    linear in rho (theta = P / rho), so this does not balance the mass flux."""
    m = self.m
    layer = np.take(fpost, src, axis=m.ax(0) + 1)
    f1, _ = m.state_eq(np.float64(1.0), [np.float64(x) for x in u_w], np.float64(T_w))
    into = sum(layer[i] for i, ci in enumerate(m.c) if ci[0] == sign)
    out = sum(f1[i] for i, ci in enumerate(m.c) if ci[0] == -sign)
    rw = into / out
    return m.state_eq(rw, [np.full_like(rw, float(x)) for x in u_w], np.full_like(rw, float(T_w)))


def test_unit_density_wall_emission_breaks_mass_pin(monkeypatch):
    import test_oracle_walls as tw
    monkeypatch.setattr(lbm.Sim, "wall_emission", unit_density_emission)
    with pytest.raises(AssertionError):
        tw.test_walls_conserve_mass()


def test_swapped_wall_direction_breaks_mass_pin(monkeypatch):
    import test_oracle_walls as tw
    orig = lbm.Sim.wall_emission
    monkeypatch.setattr(lbm.Sim, "wall_emission",
                        lambda self, fpost, src, sign, u_w, T_w: orig(self, fpost, src, -sign, u_w, T_w))
    with pytest.raises(AssertionError):
        tw.test_walls_conserve_mass()


def test_wrong_ghost_source_layer_breaks_mirror_pin(monkeypatch):
    import test_oracle_walls as tw
    orig = lbm.Sim.wall_emission
    monkeypatch.setattr(lbm.Sim, "wall_emission",
                        lambda self, fpost, src, sign, u_w, T_w: orig(self, fpost, src + (1 if sign < 0 else 0),
                                                                     sign, u_w, T_w))
    with pytest.raises(AssertionError):
        tw.test_faces_are_mirror_images()


def test_ghost_density_in_capillary_stencil_breaks_odd_even_pin(monkeypatch):
    import test_oracle_walls as tw
    monkeypatch.setattr(lbm.Sim, "capillary_density", lambda self, rho: rho)
    with pytest.raises(AssertionError):
        tw.test_odd_even_disturbance_decays_next_to_walls()


def test_korteweg_force_without_density_breaks_coexistence_pin(monkeypatch):
    import test_oracle_coexistence as tc
    orig = lbm.Sim.macroscopic

    def without_rho(self, f=None, g=None):
        m = self.m
        kappa = m.kappa
        m.kappa = kappa / (self.f if f is None else f).sum(axis=0)     # kappa rho grad lap rho -> kappa grad lap rho
        try:
            return orig(self, f, g)
        finally:
            m.kappa = kappa
    monkeypatch.setattr(lbm.Sim, "macroscopic", without_rho)
    import pytest as _pytest
    with _pytest.raises(AssertionError):
        tc.test_slab_plateaus_reach_maxwell_coexistence()


def test_departure_energy_without_alpha_slope_breaks_caloric_pin(monkeypatch):
    """e - c_v T = -(a alpha - T a alpha') L / (2 sqrt2 b): dropping T a alpha' is caught."""
    import test_oracle_pr as tp
    from oracle import eos as oeos
    monkeypatch.setattr(oeos.PengRobinson, "energy_departure",
                        lambda self, rho, T: -self.a * self.alpha(T) * self._L(rho) / (2.0 * oeos.SQRT2 * self.b))
    with pytest.raises(AssertionError):
        tp.test_caloric_relation_against_quadrature(0.6, 1.05)


# ---- shock capturing (Sec. 4.4): the coefficient assembly and its building blocks ----

def _n1_pin_fails():
    import test_oracle_n1 as n1
    return max(n1.coefficient_errors(lbm.numerical_transport)) > 1e-6


def test_swapped_shear_and_conduction_constants_break_coefficient_pin(monkeypatch):
    orig = lbm.numerical_transport

    def swapped(rho, u, T, cs2, coef, *rest, **kw):
        return orig(rho, u, T, cs2, (coef[2], coef[1], coef[0]), *rest, **kw)
    monkeypatch.setattr(lbm, "numerical_transport", swapped)
    assert _n1_pin_fails()


def test_conductivity_without_sound_speed_breaks_coefficient_pin(monkeypatch):
    orig = lbm.numerical_transport

    def no_cs(rho, u, T, cs2, coef, *rest, **kw):
        return orig(rho, u, T, np.ones_like(cs2), coef, *rest, **kw)
    monkeypatch.setattr(lbm, "numerical_transport", no_cs)
    assert _n1_pin_fails()


def test_three_point_filter_breaks_coefficient_pin(monkeypatch):
    def filter121(f, D, per):
        for a in range(D):
            f = (lbm._shift(f, a, -1, D, per[a]) + 2.0 * f + lbm._shift(f, a, 1, D, per[a])) / 4.0
        return f
    monkeypatch.setattr(lbm, "binomial_filter", filter121)
    assert _n1_pin_fails()


def test_unsymmetrised_velocity_gradient_breaks_coefficient_pin(monkeypatch):
    def grad_norm(u, D, per):
        g = [[0.5 * (lbm._shift(u[b], a, 1, D, per[a]) - lbm._shift(u[b], a, -1, D, per[a])) for b in range(D)]
             for a in range(D)]
        return np.sqrt(sum(g[a][b] ** 2 for a in range(D) for b in range(D)))
    monkeypatch.setattr(lbm, "strain_rate_magnitude", grad_norm)
    assert _n1_pin_fails()


def test_flipped_density_term_of_entropy_gradient_breaks_isentrope_pin(monkeypatch):
    import test_oracle_n1 as n1

    def flipped(rho, T, b, R, cv, D, per, fluid=None):
        gs = []
        for a in range(D):
            gT = 0.5 * (lbm._shift(T, a, 1, D, per[a]) - lbm._shift(T, a, -1, D, per[a]))
            gr = 0.5 * (lbm._shift(rho, a, 1, D, per[a]) - lbm._shift(rho, a, -1, D, per[a]))
            gs.append(cv / T * gT + R / (rho * (1.0 - b * rho)) * gr)
        return np.sqrt(sum(x * x for x in gs))
    monkeypatch.setattr(lbm, "entropy_gradient_magnitude", flipped)
    with pytest.raises(AssertionError):
        n1.test_entropy_gradient_of_isothermal_ramp_and_isentrope()


# ---- learned closure oracle (oracle/mlp.py) ----

def test_transposed_hidden_weights_break_wiring_pin(monkeypatch):
    import test_oracle_mlp as tm
    from oracle import mlp
    orig_unpack = mlp.unpack

    def unpack_t(theta):
        p = orig_unpack(theta)
        p["W2"] = p["W2"].T.copy()
        return p
    monkeypatch.setattr(mlp, "unpack", unpack_t)
    assert tm.forward_wiring_error() > 0.05


def test_hidden_bias_dropped_breaks_wiring_pin(monkeypatch):
    import test_oracle_mlp as tm
    from oracle import mlp
    orig_unpack = mlp.unpack

    def unpack_nob(theta):
        p = orig_unpack(theta)
        p["b2"] = 0.0 * p["b2"]
        return p
    monkeypatch.setattr(mlp, "unpack", unpack_nob)
    assert tm.forward_wiring_error() > 0.05


def test_loss_summed_over_outputs_breaks_normalisation_pin(monkeypatch):
    import test_oracle_mlp as tm
    from oracle import mlp
    orig = mlp.loss_and_grad

    def summed(theta, X, Y):
        loss, g = orig(theta, X, Y)
        return 3.0 * loss, 3.0 * g
    monkeypatch.setattr(mlp, "loss_and_grad", summed)
    assert tm.loss_normalisation_error() > 0.5


def test_adamw_without_second_moment_correction_breaks_constant_gradient_pin(monkeypatch):
    import test_oracle_mlp as tm
    from oracle import mlp

    def adamw_nov(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
        m = beta1 * m + (1 - beta1) * grad
        v = beta2 * v + (1 - beta2) * grad * grad
        mhat = m / (1 - beta1 ** t)
        theta = theta - lr * (mhat / (np.sqrt(v) + eps) + wd * theta)
        return theta, m, v
    monkeypatch.setattr(mlp, "adamw_step", adamw_nov)
    assert tm.adamw_constant_gradient_error() > 0.1
