"""GPU tests of the paper's shock-liquid column (column_d2q9 / column_d3q27: saturated
liquid and vapour at T_r 0.9, Ma 1.47 shock, U^2 = 35, shock capturing C_mu = C_k =
0.3) against the oracle, and at full size.

Parity: relative L2 over the interior.  FP64: 1e-12 through the impact on the
column.  FP32: 5e-5 (the bound of the shock-carrying cases) up to the impact.
From the impact on, the flow has a stagnation point on the column's front where
u_x crosses zero with a steep gradient, and the side of the upwind difference of
Phi (Sec. 3.2) follows sgn(u_x).  In the oracle a 1e-10 perturbation of the
initial density moves the fields by 1e-11 after 150 steps, one of 1e-7 by 2e-3:
FP32 rounding flips the side there, so FP32 runs are checked against the
oracle before the impact and by their physics after it.
"""
import math

import numpy as np
import pytest

import inputs
from oracle import lbm as olbm
from parity_util import assert_parity, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32_SHOCK_TOL = 5e-5


@pytest.fixture(scope="module")
def P():
    import paper_2510_14712_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()
    return P


def coef(D):
    return tuple(inputs.scenario("column_d2q9" if D == 2 else "column_d3q27")["shock_capturing"])


def d2_column(seed=4):
    return inputs.shock_column(2, (160, 96), radius=14, center=(45, 48), shock_x=20, seed=seed)


def d3_column(seed=4):
    return inputs.shock_column(3, (64, 24, 20), radius=6, center=(18, 12, 10), shock_x=8, seed=seed)


def impact_step(c, center_x, radius, shock_x):
    return (center_x - radius - shock_x) / inputs.scenario(c.name)["shock_speed"]


def oracle_run(c, steps):
    m = olbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
    m.shock_capturing = coef(c.D)
    s = olbm.Sim(m, c.rho, c.u, c.T).step(steps)
    F = s.fields()
    return dict(rho=F["rho"], u=np.stack(F["u"]), T=F["T"])


def gpu_run(P, c, steps, precision, sc=None, step_kernel=0, graphs=False):
    s = P.Solver(c, precision=precision, step_kernel=step_kernel)
    try:
        P.lbm_set_shock_capturing(s.h, *(coef(c.D) if sc is None else sc))
        P.lbm_set_graphs(s.h, graphs)
        s.init().step(steps)
        return s.fields()
    finally:
        s.close()


# (name, builder, FP64 steps past the impact, FP32 steps before it)
CASES = [("d2 column 160x96", d2_column, 120, 25), ("d3 column 64x24x20", d3_column, 40, 10)]


def test_parity_cases_straddle_the_impact():
    assert impact_step(d2_column(), 45, 14, 20) < 120 and impact_step(d2_column(), 45, 14, 20) > 25
    assert impact_step(d3_column(), 18, 6, 8) < 40 and impact_step(d3_column(), 18, 6, 8) > 10


@pytest.mark.parametrize("name,make,steps64,steps32", CASES, ids=[c[0] for c in CASES])
def test_column_fp64_matches_oracle_through_impact(P, name, make, steps64, steps32):
    assert_parity(gpu_run(P, make(), steps64, "fp64"), oracle_run(make(), steps64), 1e-12, name + " fp64")


# Per-node bound of the FP32 column runs: the liquid column is at rest before
# the impact, so u vanishes to rounding at every liquid node and FP32 rounding
# picks the side of Phi's upwind difference there (Sec. 3.2; reading 21 of the
# design notes: in the oracle a 1e-7 perturbation moves the fields by 2e-3
# after the impact).  Single nodes move by up to about 1e-2 x rms(u) (measured
# 4.1e-3 in 3-D, 1.0e-3 in 2-D) while the norm stays inside the bound.
COLUMN_NODE_MULT = 200.0


@pytest.mark.parametrize("name,make,steps64,steps32", CASES, ids=[c[0] for c in CASES])
def test_column_fp32_matches_oracle_before_impact(P, name, make, steps64, steps32):
    assert_parity(gpu_run(P, make(), steps32, "fp32"), oracle_run(make(), steps32), FP32_SHOCK_TOL, name + " fp32",
                  node_mult=COLUMN_NODE_MULT)


def test_column_multipass_and_graphs_match_fused(P):
    c = d2_column()
    a = gpu_run(P, c, 101, "fp64")
    b = gpu_run(P, c, 101, "fp64", step_kernel=P.LBM_STEP_MULTIPASS)
    g = gpu_run(P, c, 101, "fp64", graphs=True)
    for k in ("rho", "u", "T"):
        assert rel_l2(b[k], a[k]) < 1e-13, k
        assert np.array_equal(g[k], a[k]), k


def test_column_needs_shock_capturing(P):
    """Without the numerical transport the paper's column ends soon after the impact."""
    c = inputs.shock_column(2)
    s = P.Solver(c, precision="fp32").init()
    try:
        with pytest.raises(P.LbmError):
            s.step(400)
    finally:
        s.close()


def front(r_row, rho_mid):
    """Last node (from the outflow side) whose density is above rho_mid."""
    return len(r_row) - 1 - int(np.argmax(r_row[::-1] > rho_mid))


def run_to(P, c, t_over_t0, radius, center_x, shock_x, marks=2):
    """FP32 run to t / t0 after the impact; density fields at `marks` equal steps."""
    sc = inputs.scenario(c.name)
    n = int(impact_step(c, center_x, radius, shock_x) + t_over_t0 * sc["t0_per_radius"] * radius)
    s = P.Solver(c, precision="fp32")
    out = []
    try:
        P.lbm_set_shock_capturing(s.h, *coef(c.D))
        s.init()
        for k in range(marks):
            s.step(n // marks)
            out.append(s.fields())
    finally:
        s.close()
    return out, n // marks


def check_physics(out, dn, sc, row):
    F0, F1 = out[0], out[-1]
    assert np.isfinite(F1["rho"]).all()
    mid = 0.5 * (sc["post"]["rho"] + sc["vapour"]["rho"])
    x0, x1 = front(row(F0["rho"]), mid), front(row(F1["rho"]), mid)
    speed = (x1 - x0) / float(dn * (len(out) - 1))
    print("front speed %.4f vs RH %.4f, liquid max rho %.3f" % (speed, sc["shock_speed"], F1["rho"].max()))
    assert abs(speed / sc["shock_speed"] - 1) < 0.03      # Rankine-Hugoniot, far from the column
    assert F1["rho"].max() > 0.9 * sc["drop"]["rho"]      # the column stays liquid


def test_paper_column_to_end_time(P):
    """The paper's 800 x 800 column (radius 65) to its last time, t / t0 = 0.7."""
    c = inputs.shock_column(2)
    out, dn = run_to(P, c, 0.7, 65, 200, 100)
    check_physics(out, dn, inputs.scenario("column_d2q9"), lambda r: r[0])


def test_large_2d_column_to_end_time(P):
    """The column physics on the 4096 x 2048 grid (radius 128, tanh width 3, shock at
    Nx/8): to t / t0 = 0.7.  Later the rarefaction reflected from the rear interface
    drives the liquid to negative pressure (about t / t0 = 0.85 here), where theta =
    P / rho < 0 is outside the scheme."""
    c = inputs.shock_column(2, (4096, 2048), radius=128)
    out, dn = run_to(P, c, 0.7, 128, 1024, 512)
    check_physics(out, dn, inputs.scenario("column_d2q9"), lambda r: r[0])


def test_3d_sphere_to_end_time(P):
    """The 3-D analogue on 512 x 256 x 256 (saturated sphere of radius 32): to t / t0 = 0.7."""
    c = inputs.shock_column(3, (512, 256, 256), radius=32)
    out, dn = run_to(P, c, 0.7, 32, 128, 64)
    check_physics(out, dn, inputs.scenario("column_d3q27"), lambda r: r[0, 0])
