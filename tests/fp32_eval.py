"""The oracle's step evaluated with FP32 rounding (test helper, no GPU).

run(case, steps, mode): mode "fp64" is the oracle itself; "store32" keeps FP64
arithmetic but rounds the populations to float32 after every step; "fp32"
runs the whole step in float32 (state and model constants float32: numpy keeps
float32 through every array expression of the oracle).  As a script,
``python fp32_eval.py <case> <mode> <steps> <out.npz>`` writes the final
fields of one of the named cases (for child processes of the GPU tests).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import inputs  # noqa: E402
from oracle import lbm as olbm  # noqa: E402

F32 = np.float32
CONSTS = ("a", "b", "R", "cv", "kappa", "eta_over_mu", "mu", "k_over_mu")


def fields(s):
    F = s.fields()
    return dict(rho=np.asarray(F["rho"], dtype=np.float64), u=np.stack(F["u"]).astype(np.float64),
                T=np.asarray(F["T"], dtype=np.float64))


def run(case, steps, mode="fp64"):
    m = olbm.Model(case.D, case.shape, case.eos, case.tau, case.Pr, case.cv, case.x_low, case.x_high)
    s = olbm.Sim(m, case.rho, case.u, case.T)
    if mode == "fp32":
        for k in CONSTS:
            setattr(m, k, F32(getattr(m, k)))
        s.f, s.g = s.f.astype(F32), s.g.astype(F32)
    for _ in range(steps):
        s.step(1)
        if mode == "store32":
            s.f = s.f.astype(F32).astype(np.float64)
            s.g = s.g.astype(F32).astype(np.float64)
    if mode == "fp32":
        assert s.f.dtype == F32 and s.g.dtype == F32        # the run stayed in float32
    return fields(s)


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def errors(got, want):
    return {k: rel(got[k], want[k]) for k in ("rho", "u", "T")}


def tgv_headline_case():
    """64^3 Taylor-Green vortex at the 256^3 workload's tau, U0, kappa, eta/mu, seeded 1e-3 noise."""
    c = inputs.add_noise(inputs.tgv(shape=(64, 64, 64)), 0)
    c.tau = inputs.scenario("tgv_d3q27")["tau"]
    return c


def tgv_drift_case():
    """19 x 13 x 11 Taylor-Green box at lattice viscosity 0.02 with a uniform drift (seed 5)."""
    c = inputs.add_noise(inputs.tgv(shape=(19, 13, 11)), 5)
    sc = inputs.scenario("tgv_d3q27")
    c.tau = sc["tau"] * 0.02 / sc["nu"]
    c.u = [ua + d for ua, d in zip(c.u, (0.08, -0.05, 0.06))]
    return c


def shock_case(seed=3, Nx=400, Ny=3, Ma=1.2):
    """Ma 1.2 D2Q9 shock tube in the shock-drop scenario's vapour (post-state from
    the oracle's Rankine-Hugoniot solver), shock at x = 60, seeded noise."""
    import copy
    from oracle import thermo
    sc = copy.deepcopy(inputs.scenario("shock_drop_d2q9"))
    e, v = sc["eos"], sc["vapour"]
    r2, T2, u2, _ = thermo.rankine_hugoniot(v["rho"], v["T"], 0.0, Ma, e["a"], e["b"], e["R"], sc["cv"])
    sc["post"] = dict(rho=r2, T=T2, u=u2)
    return inputs.add_noise(inputs.shock_drop(2, (Nx, Ny), shock_x=60, with_drop=False, sc=sc), seed)


CASES = {"tgv_headline": tgv_headline_case, "tgv_drift": tgv_drift_case, "riemann": lambda: inputs.riemann(),
         "shock_tube": shock_case}


def fp32_bound(e32, floor=1e-5, factor=2.0):
    """FP32 parity bound per field: 1e-5, or twice what the scheme evaluated in
    float32 reaches when that is larger (an FP32 kernel rounds differently --
    fused multiply-adds, summation order, reciprocal-based division -- and lands
    within a factor of about two of it either way)."""
    return {k: max(floor, factor * v) for k, v in e32.items()}


if __name__ == "__main__":
    name, mode, steps, out = sys.argv[1], sys.argv[2], int(sys.argv[3]), sys.argv[4]
    np.savez(out, **run(CASES[name](), steps, mode))
