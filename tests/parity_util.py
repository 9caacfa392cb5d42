"""Helpers of the GPU parity tests: run one case on the oracle and on the CUDA path."""
import numpy as np

from oracle import lbm as olbm


def oracle_run(case, steps):
    m = olbm.Model(case.D, case.shape, case.eos, case.tau, case.Pr, case.cv, case.x_low, case.x_high)
    s = olbm.Sim(m, case.rho, case.u, case.T)
    s.step(steps)
    F = s.fields()
    return dict(rho=F["rho"], u=np.stack(F["u"]), T=F["T"], totals=s.totals())


def gpu_run(case, steps, precision, chunk=None, step_kernel=0):
    import paper_2510_14712_gb300 as P
    s = P.Solver(case, precision=precision, step_kernel=step_kernel)
    try:
        s.init()
        if chunk:
            done = 0
            while done < steps:
                k = min(chunk, steps - done)
                s.step(k)
                done += k
        else:
            s.step(steps)
        out = s.fields()
        out["launches"] = P.lbm_launch_count(s.h)
        return out
    finally:
        s.close()


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def assert_parity(got, want, tol, what=""):
    errs = {k: rel_l2(got[k], want[k]) for k in ("rho", "u", "T")}
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, "%s relative L2 above %g: %s" % (what, tol, errs)
    return errs
