"""Pin of the two-phase equilibrium (Sec. "Liquid-vapour co-existence"): a periodic slab
of saturated liquid in its saturated vapour relaxes to plateaus at the densities of
Maxwell's equal-area construction (thermo.maxwell_coexistence, itself pinned against
the paper's printed nitrogen values) at the slab's equilibrium temperature.

On the oracle's small slab (48 nodes, T_r 0.95, 12,000 steps) the plateaus are short
and not fully settled: liquid within 1% and vapour within 2% (measured -0.5% and
+0.9%).  A Korteweg force without its density factor (F = kappa grad lap rho)
changes the effective free energy and moves them to -1.5% and -4.0%.
"""
import numpy as np

import inputs
from oracle import lbm, thermo


def slab_plateaus(steps=12000, Nx=48):
    c = inputs.slab(0.95, Nx)
    m = lbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
    s = lbm.Sim(m, c.rho, c.u, c.T).step(steps)
    F = s.fields()
    r = F["rho"][0]
    U2 = inputs.scenario("coexistence_d2q9")["states"]["0.95"]["U2"]
    T_eq = F["T"][0].mean() * U2                       # reduced units
    rl, rv = thermo.maxwell_coexistence(T_eq, 3.0, 1.0 / 3.0, 8.0 / 3.0)
    return r[Nx // 2 - 4:Nx // 2 + 4].mean() / rl - 1, np.r_[r[:3], r[-3:]].mean() / rv - 1


def test_slab_plateaus_reach_maxwell_coexistence():
    dl, dv = slab_plateaus()
    assert abs(dl) < 0.01, dl
    assert abs(dv) < 0.02, dv
