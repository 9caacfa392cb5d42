"""Helpers of the learned-closure tests: an oracle-trained network and cases."""
import numpy as np

import inputs
from oracle import mlp


def shock_eos():
    sc = inputs.scenario("shock_drop_d2q9")
    e = sc["eos"]
    return e["a"], e["b"], e["R"], sc["cv"]


def oracle_network(seed=21, n=4096, steps=1500, batch=256):
    """A closure network trained by the oracle alone (FP64 AdamW on exact labels).

    Samples are uniform in the (rho, T) box that holds the shock-tube states
    of the batch table (rho 0.27..0.50, T 0.085..0.125 in the lattice units
    of the shock scenarios), e = c_v T - a rho.  Returns the FP32 master
    parameters and the 10 scaling constants (midpoints / half-ranges of the
    samples and of their labels).
    """
    a, b, R, cv = shock_eos()
    rho = 0.385 + 0.115 * inputs.uniform(seed, n)
    T = 0.105 + 0.020 * inputs.uniform(seed + 1, n)
    e = cv * T - a * rho
    lab = mlp.vdw_targets(rho, e, a, b, R, cv)
    scale = []
    for v in (rho, e) + tuple(lab):
        lo, hi = v.min(), v.max()
        scale += [0.5 * (lo + hi), 0.5 * (hi - lo)]
    scale = np.array(scale)
    X = np.stack([(rho - scale[0]) / scale[1], (e - scale[2]) / scale[3]], axis=1)
    Y = np.stack([(lab[k] - scale[4 + 2 * k]) / scale[5 + 2 * k] for k in range(3)], axis=1)
    theta0 = mlp.init_params(inputs.uniform(seed + 2, mlp.NPARAM))
    theta, losses = mlp.train(theta0, X, Y, steps, batch, 3e-3, 1e-5, seed + 3)
    return theta.astype(np.float32), scale, losses


def oracle_closure(theta, scale):
    """The gated closure of the FP32 parameters theta as an oracle Model hook."""
    a, b, R, cv = shock_eos()
    tq = mlp.quantize(theta)

    def fn(rho, e):
        T, P, c2, _ = mlp.closure(tq, scale, rho, e, a, b, R, cv)
        return T, P, c2
    return fn


def shock_tube(D, shape, Ma=1.2, seed=13):
    """Planar shock tube in the shock scenarios' units, post-state of the batch
    table entry closest to Ma, shock at Nx/8, seeded 1e-3 perturbation."""
    tab = inputs.scenario("batch_d2q9")["instances"]
    k = min(range(len(tab)), key=lambda i: abs(tab[i]["Ma"] - Ma))
    name = "shock_drop_d2q9" if D == 2 else "shock_drop_d3q27"
    sc = dict(inputs.scenario(name))
    sc["post"] = tab[k]["post"]
    c = inputs.shock_drop(D, shape, shock_x=shape[0] // 8, with_drop=False, sc=sc)
    return inputs.add_noise(c, seed)
