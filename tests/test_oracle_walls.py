"""Pins of the oracle's wall faces (the thermal Couette flow of Sec. 4.1).

The paper prescribes the wall values u = (0, 0), T_w at x = 0 and u = (0, U_w),
T_w at x = L_x but no wall scheme; the oracle reads it as diffuse reflection
with a mass-balancing factor and a symmetry plane for the capillary terms.
What fixes it, independently of the oracle's own arithmetic:
  - a wall at rest at the fluid's own state leaves that uniform state exactly
    unchanged (it re-emits the fluid's own equilibrium);
  - no mass crosses a wall: the interior mass is constant to rounding;
  - the two faces are mirror images of each other: reflecting the channel
    (x -> Nx - 1 - x, u_x -> -u_x) and moving the other wall gives the
    reflected run;
  - the steady Couette flow has the closed form of Sec. 4.1: u_y linear in x
    and k T'' = -mu (du_y/dx)^2 (constant mu and k), which the fitted profiles
    obey to the discretisation error;
  - an odd-even disturbance next to the walls decays.
"""
import numpy as np
import pytest

import physics_cases as pc


def interior_mass(s):
    return float(s.fields()["rho"].sum())


def test_wall_at_rest_keeps_uniform_state():
    s, _, rho0, T_w = pc.wall_channel(Nx=12, Ma=0.0)
    s.step(200)
    F = s.fields()
    assert np.abs(F["rho"] - rho0).max() < 1e-13
    assert max(np.abs(ua).max() for ua in F["u"]) < 1e-13
    assert np.abs(F["T"] - T_w).max() < 1e-13


def test_walls_conserve_mass():
    s, _, _, _ = pc.wall_channel(Nx=16, Ma=1.0, perturb=0.01)
    m0 = interior_mass(s)
    s.step(300)
    assert abs(interior_mass(s) / m0 - 1) < 1e-13


def test_faces_are_mirror_images():
    a, _, rho0, T_w = pc.wall_channel(Nx=14, Ma=0.8, perturb=0.01, moving="high")
    b, _, _, _ = pc.wall_channel(Nx=14, Ma=0.8, moving="low")
    # b restarted from the reflection of a's initial primitive state
    rho = rho0 * (1.0 + 0.01 * np.sin(np.arange(14, dtype=float)))[None, :]
    b = type(b)(b.m, rho[:, ::-1], [np.zeros((1, 14)), np.zeros((1, 14))], np.full((1, 14), T_w))
    a.step(150)
    b.step(150)
    Fa, Fb = a.fields(), b.fields()
    assert np.abs(Fb["rho"] - Fa["rho"][:, ::-1]).max() < 1e-13
    assert np.abs(Fb["u"][0] + Fa["u"][0][:, ::-1]).max() < 1e-13
    assert np.abs(Fb["u"][1] - Fa["u"][1][:, ::-1]).max() < 1e-13
    assert np.abs(Fb["T"] - Fa["T"][:, ::-1]).max() < 1e-13
    assert np.abs(Fa["u"][1]).max() > 1e-3            # the moving wall has driven a flow


@pytest.mark.parametrize("Ma", [0.5, 1.0])
def test_couette_profile_and_viscous_heating(Ma):
    x, uy, T, rho, U_w, T_w, mu, k = pc.thermal_couette(Nx=24, Ma=Ma, steps=8000)
    a = np.polyfit(x, uy, 1)
    c = np.polyfit(x, T, 2)
    assert np.abs(np.polyval(a, x) - uy).max() < 1e-5 * U_w     # u_y linear (Sec. 4.1)
    ratio = 2.0 * c[0] / (-mu * a[0] ** 2 / k)                    # k T'' = -mu u_y'^2
    assert abs(ratio - 1) < 0.01, ratio
    assert T.max() > T_w                                          # heated by viscous dissipation
    # the effective walls lie symmetrically about the channel centre
    x0, x1 = -a[1] / a[0], (U_w - a[1]) / a[0]
    assert abs((x0 + x1) / 2 - (len(x) - 1) / 2) < 0.01


def test_odd_even_disturbance_decays_next_to_walls():
    s, _, _, _ = pc.wall_channel(Nx=24, Ma=0.0, perturb=0.01)
    s.step(2000)
    assert np.abs(s.fields()["u"][0]).max() < 1e-6
