"""GPU tests of the two-phase equilibrium (Sec. "Liquid-vapour co-existence" and
"Interface consistency and convergence"): periodic slabs of saturated liquid in its
saturated vapour against the oracle, and their converged plateaus against Maxwell's
equal-area construction at the equilibrium temperature.

Measured range of this scheme: T_r 0.85 to 0.99.  Below T_r = 27/32 the van der
Waals pressure is negative for densities inside the interface, so theta = P / rho and
tau = mu / P are negative at the first step; the paper reports down to 0.3.  Under refinement (lattice
capillarity kappa up at a fixed velocity scale: the interface spans more nodes,
kappa_lat ~ 1/dx^2) the vapour density approaches Maxwell's about as 1/kappa, i.e.
second order in dx, the order the paper reports.
"""
import numpy as np
import pytest

import inputs
from oracle import lbm as olbm, thermo
from parity_util import assert_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2510_14712_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()
    return P


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_slab_matches_oracle(P, precision, tol):
    """The slab drifting along its interfaces at u_y = 0.1: without the drift u is the
    decaying residual of the interfaces' relaxation (|u| ~ 1e-5), and a relative L2
    error of u would measure rounding against nothing; the drift changes nothing else
    (Galilean invariance) and exercises the Galilean terms."""
    c = inputs.slab(0.9, 72)
    c.u[1] = c.u[1] + 0.1
    m = olbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
    Fo = olbm.Sim(m, c.rho, c.u, c.T).step(400).fields()
    want = dict(rho=Fo["rho"], u=np.stack(Fo["u"]), T=Fo["T"])
    s = P.Solver(c, precision=precision)
    try:
        s.init().step(400)
        got = s.fields()
    finally:
        s.close()
    assert_parity(got, want, tol, "slab %s" % precision)


def converged_plateaus(P, T_r, kappa=None, Nx=256, steps=400000, chunk=20000):
    """FP64 slab stepped until the plateaus and the mean temperature change by less than
    1e-10 over a chunk: (liquid, vapour) relative deviation from Maxwell at T_eq."""
    c = inputs.slab(T_r, Nx, kappa=kappa)
    U2 = inputs.coexistence_state(T_r)["U2"]
    s = P.Solver(c, precision="fp64")
    try:
        P.lbm_set_graphs(s.h, True)
        s.init()
        prev, done = None, 0
        while done < steps:
            s.step(chunk)
            done += chunk
            F = s.fields()
            r = F["rho"][0]
            cur = np.array([r[Nx // 2 - 10:Nx // 2 + 10].mean(), np.r_[r[:10], r[-10:]].mean(), F["T"][0].mean()])
            if prev is not None and np.abs(cur - prev).max() < 1e-10:
                break
            prev = cur
    finally:
        s.close()
    rl, rv = thermo.maxwell_coexistence(cur[2] * U2, 3.0, 1.0 / 3.0, 8.0 / 3.0)
    return cur[0] / rl - 1, cur[1] / rv - 1


# (T_r, liquid bound, vapour bound): measured 1.27e-2 / 2.49e-2, 9e-4 / 5.5e-3, 3e-5 / 9.5e-4,
# 7e-5 / 7e-6 (the deviation grows towards the 27/32 limit at a fixed lattice kappa)
COEX = [(0.85, 2e-2, 4e-2), (0.9, 2e-3, 1e-2), (0.95, 2e-4, 2e-3), (0.99, 2e-4, 1e-4)]


@pytest.mark.parametrize("T_r,tol_l,tol_v", COEX, ids=["Tr%.2f" % c[0] for c in COEX])
def test_coexistence_densities_match_maxwell(P, T_r, tol_l, tol_v):
    dl, dv = converged_plateaus(P, T_r)
    print("T_r %.2f: liquid %.2e, vapour %.2e from Maxwell" % (T_r, dl, dv))
    assert abs(dl) < tol_l and abs(dv) < tol_v, (dl, dv)


def test_vapour_density_converges_at_second_order(P):
    """T_r 0.95, kappa_lat = 0.0125 .. 0.1 (the interface 1 .. 2.8 times wider in nodes):
    the vapour's deviation from Maxwell falls about as 1/kappa (dx^2)."""
    ks = [0.0125, 0.025, 0.05, 0.1]
    dv = [abs(converged_plateaus(P, 0.95, kappa=k)[1]) for k in ks]
    slope = -np.polyfit(np.log(ks), np.log(dv), 1)[0]
    print("vapour deviation", ["%.2e" % d for d in dv], "slope in kappa %.2f" % slope)
    assert all(a > b for a, b in zip(dv, dv[1:]))
    assert slope > 0.8


def test_slab_below_27_over_32_raises_the_pressure_flag(P):
    """T_r 0.84, below the 27/32 at which the van der Waals isotherm's minimum crosses zero:
    the first step leaves interface nodes with P <= 0 (theta = P / rho and tau = mu / P
    negative), which the step reports as LBM_FLAG_PRESSURE; the slab at T_r 0.85 does not."""
    from oracle import write_scenarios as ws
    for T_r, want in ((0.84, True), (0.85, False)):
        st = ws.coexistence(T_r=(T_r,))["states"][ws.coexistence_key(T_r)]
        s = P.Solver(inputs.slab(T_r, 256, state=st), precision="fp64")
        try:
            s.init().step(1)
            flags = P.lbm_get_flags(s.h)
        finally:
            s.close()
        assert bool(flags & P.LBM_FLAG_PRESSURE) == want, (T_r, flags)
