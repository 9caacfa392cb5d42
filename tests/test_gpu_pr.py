"""GPU tests of the Peng-Robinson fluid (lbm_eos.kind LBM_EOS_PR: the general equation
of state of Sec. 2, temperature from its non-linear caloric relation) against the
oracle (oracle/eos.py, Newton's method for the temperature).

Parity: relative L2 over the interior, 1e-12 (FP64) and 1e-5 (FP32; 5e-5 for the
Riemann problem, the shock-carrying bound).  The kernels invert the caloric
relation in closed form (a quadratic in sqrt(T), in a form without cancellation),
the oracle by Newton's method: both find the same unique root.
"""
import numpy as np
import pytest

import inputs
from oracle import lbm as olbm
from oracle import eos as oeos
from parity_util import assert_parity, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2510_14712_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()
    return P


def pr_tgv(shape=(24, 20, 12), drift=(0.08, -0.05, 0.06), seed=2, nu=0.02):
    c = inputs.add_noise(inputs.tgv(shape=shape, scenario_name="tgv_pr_d3q27"), seed)
    sc = inputs.scenario("tgv_pr_d3q27")
    c.tau = sc["tau"] * nu / sc["nu"]
    c.u = [ua + d for ua, d in zip(c.u, drift)]
    c.eos = dict(c.eos, eta_over_mu=1.0)
    return c


def pr_box2d(shape=(57, 23), seed=5):
    sc = inputs.scenario("tgv_pr_d3q27")
    c = inputs.Case(name="tgv_pr_d3q27", D=2, shape=shape, eos=dict(sc["eos"], eta_over_mu=1.0), tau=0.2,
                    Pr=sc["Pr"], cv=sc["cv"])
    n, arr = shape[0] * shape[1], (shape[1], shape[0])
    c.rho = sc["rho0"] * (1 + 0.02 * inputs.uniform(seed, n).reshape(arr))
    c.T = sc["T0"] * (1 + 0.02 * inputs.uniform(seed + 1, n).reshape(arr))
    c.u = [0.1 + 0.03 * inputs.uniform(seed + 2, n).reshape(arr), -0.07 + 0.03 * inputs.uniform(seed + 3, n).reshape(arr)]
    return c


def pr_riemann(Nx=400, Ny=3):
    """Riemann problem in the Peng-Robinson fluid: left rho 0.9 T 1.3 | right rho 0.3 T 1.2
    (reduced, supercritical on both sides and through the rarefaction), outflow faces,
    split at Nx/2."""
    sc = inputs.scenario("tgv_pr_d3q27")
    U2 = 16.0                                   # theta / U^2 <= 0.2 over both states
    cr = sc["crit"]
    eos = dict(sc["eos"], a=cr["a"] / U2, Tc=1.0 / U2, eta_over_mu=1.0, rho_ref=0.3, T_ref=1.2 / U2)
    c = inputs.Case(name="tgv_pr_d3q27", D=2, shape=(Nx, Ny), eos=eos, tau=0.05,
                    Pr=sc["Pr"], cv=sc["cv"], x_low="outflow", x_high="outflow")
    x = c.grid()[0]
    left = x < Nx // 2
    c.rho = np.where(left, 0.9, 0.3)
    c.T = np.where(left, 1.3, 1.2) / U2
    c.u = [np.zeros_like(c.rho), np.zeros_like(c.rho)]
    return inputs.add_noise(c, 7)


def oracle_run(c, steps):
    m = olbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
    F = olbm.Sim(m, c.rho, c.u, c.T).step(steps).fields()
    return dict(rho=F["rho"], u=np.stack(F["u"]), T=F["T"])


def gpu_run(P, c, steps, precision, step_kernel=0):
    s = P.Solver(c, precision=precision, step_kernel=step_kernel)
    try:
        s.init().step(steps)
        return s.fields()
    finally:
        s.close()


CASES = [("d3 tgv 24x20x12", pr_tgv, 30, 1e-5), ("d2 box 57x23", pr_box2d, 80, 1e-5),
         ("d2 riemann 400x3", pr_riemann, 300, 5e-5)]


@pytest.fixture(scope="module")
def refs():
    return {name: oracle_run(make(), steps) for name, make, steps, _ in CASES}


@pytest.mark.parametrize("name,make,steps,tol32", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pr_matches_oracle(P, refs, name, make, steps, tol32, precision):
    got = gpu_run(P, make(), steps, precision)
    assert_parity(got, refs[name], 1e-12 if precision == "fp64" else tol32, "%s %s" % (name, precision))


def test_pr_multipass_matches_fused(P):
    c = pr_riemann()
    a = gpu_run(P, c, 200, "fp64")
    b = gpu_run(P, c, 200, "fp64", step_kernel=P.LBM_STEP_MULTIPASS)
    for k in ("rho", "u", "T"):
        assert rel_l2(b[k], a[k]) < 1e-13, k


def test_pr_temperature_is_the_caloric_root(P):
    """lbm_moments' T of a uniform state at rest equals the initial T (the inversion of
    e(rho, T) returns T) over a range of states, FP64."""
    sc = inputs.scenario("tgv_pr_d3q27")
    e = sc["eos"]
    fl = oeos.PengRobinson(e["a"], e["b"], e["R"], sc["cv"], e["Tc"], e["m"])
    for rho, Tr in ((0.2, 0.9), (0.6, 1.05), (1.4, 1.2), (2.0, 1.5)):
        c = pr_box2d((5, 4))
        c.rho = np.full((4, 5), rho)
        c.T = np.full((4, 5), Tr * e["Tc"])
        c.u = [np.zeros((4, 5)), np.zeros((4, 5))]
        F = gpu_run(P, c, 0, "fp64")
        assert np.abs(F["T"] / (Tr * e["Tc"]) - 1).max() < 1e-13
        assert abs(fl.temperature(rho, fl.energy(rho, Tr * e["Tc"])) / (Tr * e["Tc"]) - 1) < 1e-13


def test_pr_rejected_where_unsupported(P):
    c = pr_box2d((16, 8))
    with pytest.raises(P.LbmError):                 # FP16-deviation storage
        P.Solver(c, precision="fp16dev")
    with pytest.raises(P.LbmError):                 # batches are van der Waals only
        P.Batch([c, pr_box2d((12, 8))], precision="fp32")
    net = P.Closure(c.eos["a"], c.eos["b"], c.eos["R"], c.cv, seed=1)
    s = P.Solver(c, precision="fp32")
    try:
        net.scaling = [0.5, 0.5, 0.5, 0.5, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1]
        with pytest.raises(P.LbmError):             # the learned closure is trained on van der Waals
            net.attach(s)
    finally:
        s.close()
        net.close()
