"""Physics pins of the oracle (P3-P7): closed-form rates and speeds of Sec. 4.1 and 4.4."""
import pytest

import physics_cases as pc


def test_sound_speed():
    """P3: a weak pressure front travels at the vdW adiabatic c_s (Eq. vdW_speed_of_sound)."""
    c, want = pc.sound_speed()
    assert abs(c / want - 1) < 0.01


def test_sound_speed_moving_frame():
    """P3 with a background flow u0: the front travels at c_s + u0."""
    c, want = pc.sound_speed(u0=0.1)
    assert abs(c / want - 1) < 0.01


@pytest.mark.parametrize("May", [0.0, 0.25, 0.5])
def test_shear_viscosity_galilean(May):
    """P4: shear-wave decay gives nu = mu/rho, independent of the background Mach number."""
    nu, want = pc.shear_decay(May)
    assert abs(nu / want - 1) < 0.02


def test_thermal_diffusivity():
    """P5: entropic-mode decay at rate k/(rho0 c_p) (Sec. 4.1, thermal conductivity test)."""
    chi, want = pc.thermal_decay()
    assert abs(chi / want - 1) < 0.03


def test_acoustic_attenuation():
    """P6: acoustic energy decays with sigma = 2(D-1)/D mu/rho + eta/rho + k/(rho c_p)(c_p/c_v - 1)."""
    sig, want = pc.acoustic_decay()
    assert abs(sig / want - 1) < 0.03


def test_acoustic_attenuation_bulk_viscosity():
    """P6 with a different eta/mu: alpha (Eq. corr_bulk) makes eta a free parameter."""
    sig, want = pc.acoustic_decay(eta=3.0)
    assert abs(sig / want - 1) < 0.03


@pytest.mark.parametrize("Max", [0.2, 0.4])
def test_acoustic_attenuation_moving_frame(Max):
    """P6 in a moving frame: sigma unchanged with u_x = Ma_x c_s (Galilean invariance, needs Phi)."""
    sig, want = pc.acoustic_decay(Max=Max)
    assert abs(sig / want - 1) < 0.03


def test_rankine_hugoniot_shock():
    """P7: a Ma 1.2 shock keeps the RH post-state plateau and moves at the RH shock speed."""
    speed, us, plateau, post = pc.shock_tube(Ma=1.2)
    assert abs(speed / us - 1) < 0.02
    for got, want in zip(plateau, post):
        assert abs(got / want - 1) < 0.01
