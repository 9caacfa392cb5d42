"""Cases of the bounds-check test (tests/test_gpu_bounds.py): small runs that
take every indexing path of the step kernels -- the small-box modulo path,
stage A by quads of x nodes (periodic and ghost-padded x), its scalar
fallback (x not a multiple of 4, wall columns), inflow/outflow and wall ghost
fills, the multi-pass step and the batched step.  Run as a script with
LBM_LIBRARY naming a library build, it writes every case's fields and the
library's out-of-buffer access count to an .npz file."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import inputs  # noqa: E402


def _tgv(shape, seed):
    c = inputs.add_noise(inputs.tgv(shape=shape), seed)
    sc = inputs.scenario("tgv_d3q27")
    c.tau = sc["tau"] * 0.05 / sc["nu"]
    return c


def _box2d(shape, seed):
    sc = inputs.scenario("tgv_d3q27")
    c = inputs.Case(name="tgv_d3q27", D=2, shape=shape, eos=dict(sc["eos"]), tau=0.1, Pr=0.71, cv=sc["cv"])
    arr = tuple(reversed(shape))
    n = int(np.prod(shape))
    c.rho = sc["rho0"] * (1 + 0.01 * inputs.uniform(seed, n).reshape(arr))
    c.T = sc["T0"] * (1 + 0.01 * inputs.uniform(seed + 1, n).reshape(arr))
    c.u = [0.02 * inputs.uniform(seed + 2 + a, n).reshape(arr) for a in range(2)]
    return c


# name: (case builder, precision, steps, step kernel)
CASES = {
    "d3_8cube_fp32": (lambda: _tgv((8, 8, 8), 1), "fp32", 12, 0),
    "d3_8cube_fp64": (lambda: _tgv((8, 8, 8), 2), "fp64", 12, 0),
    "d2_16x4_fp32": (lambda: _box2d((16, 4), 3), "fp32", 12, 0),
    "d2_16x4_fp64": (lambda: _box2d((16, 4), 4), "fp64", 12, 0),
    "d3_quads_periodic_fp32": (lambda: _tgv((40, 24, 12), 5), "fp32", 8, 0),
    "d3_quads_periodic_fp16": (lambda: _tgv((40, 24, 12), 6), "fp16dev", 8, 0),
    "d3_scalar_ragged_fp32": (lambda: _tgv((37, 21, 13), 7), "fp32", 8, 0),
    "d3_quads_multipass_fp32": (lambda: _tgv((40, 24, 12), 8), "fp32", 6, 1),
    "d3_tube_ghosts_fp32": (lambda: inputs.shock_tube_3d(shape=(97, 9, 7), Ma=1.15, seed=9), "fp32", 10, 0),
    "d2_tube_ghosts_fp16": (lambda: inputs.riemann(Nx=203, Ny=3, split=100), "fp16dev", 10, 0),
    "d2_walls_fp64": (lambda: inputs.couette(D=2, shape=(61, 3), Ma=0.5, seed=10), "fp64", 10, 0),
    "d3_walls_fp32": (lambda: inputs.couette(D=3, shape=(45, 11, 5), Ma=0.5, seed=11), "fp32", 10, 0),
}


def run_all(P):
    out = {}
    for name, (mk, prec, steps, sk) in CASES.items():
        s = P.Solver(mk(), precision=prec, step_kernel=sk)
        try:
            s.init().step(steps)
            F = s.fields()
        finally:
            s.close()
        for k in ("rho", "u", "T"):
            out["%s.%s" % (name, k)] = np.asarray(F[k])
    cases = inputs.batch(3)
    b = P.Batch(cases, precision="fp32")
    try:
        b.init()
        b.step(6)
        for k in range(len(cases)):
            F = b.fields(k)
            for key in ("rho", "u", "T"):
                out["batch%d.%s" % (k, key)] = np.asarray(F[key])
    finally:
        b.close()
    return out


def main(path):
    import paper_2510_14712_gb300 as P
    out = run_all(P)
    out["violations"] = np.array(P.lbm_debug_bounds_violations())
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
