"""Batched form: many uneven D2Q9 instances stepped by one persistent launch per step.

Each instance of a batch must end bit-identical to the same case stepped on
its own handle (the per-node arithmetic does not depend on the work split),
and small batches match the FP64 oracle within the tolerances of the parity
tests.
"""
import copy

import numpy as np
import pytest

import inputs
from parity_util import gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2510_14712_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14712_gb300 import build
    build.build()
    P.load()


def small_tube(Nx, Ny, Ma, seed):
    """A shock tube of the batched workload's fluid at a chosen size and Mach number."""
    from oracle import thermo
    sc = copy.deepcopy(inputs.scenario("shock_drop_d2q9"))
    e, v = sc["eos"], sc["vapour"]
    r2, T2, u2, _ = thermo.rankine_hugoniot(v["rho"], v["T"], 0.0, Ma, e["a"], e["b"], e["R"], sc["cv"])
    sc["post"] = dict(rho=r2, T=T2, u=u2)
    return inputs.add_noise(inputs.shock_drop(2, (Nx, Ny), shock_x=Nx // 6, with_drop=False, sc=sc), seed)


def periodic_box(Nx, Ny, seed):
    """Periodic vapour box with noise (same fluid), to mix periodic and bounded instances."""
    sc = inputs.scenario("shock_drop_d2q9")
    c = inputs.Case(name="shock_drop_d2q9", D=2, shape=(Nx, Ny), eos=dict(sc["eos"]), tau=sc["tau"], Pr=sc["Pr"],
                    cv=sc["cv"])
    n, arr = Nx * Ny, (Ny, Nx)
    c.rho = sc["vapour"]["rho"] * (1 + 0.01 * inputs.uniform(seed, n).reshape(arr))
    c.T = sc["vapour"]["T"] * (1 + 0.01 * inputs.uniform(seed + 1, n).reshape(arr))
    c.u = [0.05 * inputs.uniform(seed + 2 + a, n).reshape(arr) for a in range(2)]
    return c


def mixed_cases():
    return (inputs.batch(3) + [small_tube(301, 7, 1.15, 1), small_tube(93, 40, 1.25, 2),
                                periodic_box(77, 33, 3), periodic_box(5, 300, 4)])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_bit_identical_to_single_handles(precision):
    cases = mixed_cases()
    b = P.Batch(cases, precision=precision)
    try:
        b.init().step(25)
        got = [b.fields(k) for k in range(len(cases))]
        assert b.launches() == 50
    finally:
        b.close()
    for k, c in enumerate(mixed_cases()):
        want = gpu_run(c, 25, precision)
        for f in ("rho", "u", "T"):
            assert np.array_equal(got[k][f], want[f]), (k, f, rel_l2(got[k][f], want[f]))


def test_batch_fp64_matches_oracle():
    cases = [small_tube(301, 3, 1.2, 5), periodic_box(40, 17, 6)]
    b = P.Batch(cases, precision="fp64")
    try:
        b.init().step(200)
        for k, c in enumerate(cases):
            want = oracle_run(c, 200)
            got = b.fields(k)
            for f in ("rho", "u", "T"):
                assert rel_l2(got[f], want[f]) <= 1e-12, (k, f, rel_l2(got[f], want[f]))
    finally:
        b.close()


def test_batch_autotune_keeps_state():
    cases = mixed_cases()
    b = P.Batch(cases, precision="fp32")
    try:
        b.init()
        before = b.fields(1)
        chosen, ms = b.autotune(2)
        assert ms > 0
        assert np.array_equal(before["rho"], b.fields(1)["rho"])
        b.step(10)
        got = [b.fields(k) for k in range(len(cases))]
    finally:
        b.close()
    for k, c in enumerate(mixed_cases()):
        want = gpu_run(c, 10, "fp32")
        assert np.array_equal(got[k]["rho"], want["rho"]), k


def test_batch_unstable_instance_is_reported_and_isolated():
    cases = mixed_cases()
    cases[2].rho = cases[2].rho.copy()
    cases[2].rho[5, 7] = np.nan
    b = P.Batch(cases, precision="fp32")
    try:
        b.init()
        with pytest.raises(P.LbmError) as ei:
            b.step(3)
        assert ei.value.code == P.LBM_EUNSTABLE and "instance 2" in str(ei.value)
        assert b.flags(2) & P.LBM_FLAG_NONFINITE
        assert b.flags(0) & (P.LBM_FLAG_NONFINITE | P.LBM_FLAG_NEGATIVE) == 0
        with pytest.raises(P.LbmError) as ei:
            b.step(1)
        assert ei.value.code == P.LBM_ESTATE
        ok = inputs.batch(3)[2]
        P.load()
        b.cases[2] = ok
        b.init()
        b.step(2)
    finally:
        b.close()


def column_mix():
    """Shock-liquid columns and a Ma 1.45 tube of the column fluid (the batched
    shock-drop workload's), uneven sizes."""
    from oracle import thermo
    sc = copy.deepcopy(inputs.scenario("column_d2q9"))
    e, v = sc["eos"], sc["vapour"]
    r2, T2, u2, _ = thermo.rankine_hugoniot(v["rho"], v["T"], 0.0, 1.45, e["a"], e["b"], e["R"], sc["cv"])
    sc["post"] = dict(rho=r2, T=T2, u=u2)
    tube = inputs.shock_drop(2, (200, 64), shock_x=25, with_drop=False, sc=sc)
    tube.name = "column_d2q9"
    return [inputs.shock_column(2, (160, 96), radius=14, center=(45, 48), shock_x=20, seed=1), tube,
            inputs.shock_column(2, (192, 100), radius=16, center=(50, 50), shock_x=24, seed=2),
            inputs.shock_column(2, (130, 70), radius=10, center=(36, 35), shock_x=16, seed=3)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_shock_capturing_bit_identical_to_single_handles(precision):
    """Shock capturing on instances 0-2 (not 3): the batched stencils, one block per
    row of those instances, give each instance exactly its single-handle result."""
    coef = tuple(inputs.scenario("column_d2q9")["shock_capturing"])
    cases = column_mix()
    b = P.Batch(cases, precision=precision)
    try:
        for k in range(3):
            b.set_shock_capturing(*coef, k=k)
        b.init().step(60)
        got = [b.fields(k) for k in range(len(cases))]
        assert b.launches() == 60 * (2 + 4)
    finally:
        b.close()
    for k, c in enumerate(column_mix()):
        s = P.Solver(c, precision=precision)
        try:
            if k < 3:
                P.lbm_set_shock_capturing(s.h, *coef)
            s.init().step(60)
            want = s.fields()
        finally:
            s.close()
        for f in ("rho", "u", "T"):
            assert np.array_equal(got[k][f], want[f]), (k, f, rel_l2(got[k][f], want[f]))


def test_batch_shock_capturing_bad_index():
    b = P.Batch(column_mix()[:2], precision="fp32")
    try:
        with pytest.raises(P.LbmError):
            b.set_shock_capturing(0.3, 0.0, 0.3, k=2)
    finally:
        b.close()


def test_batch_autotune_with_shock_capturing_keeps_results():
    """Timing the tile shapes must not touch the shock-capturing coefficients the next
    step reads: a tuned batch steps bit-identically to an untuned one."""
    coef = tuple(inputs.scenario("column_d2q9")["shock_capturing"])
    runs = []
    for tune in (False, True):
        b = P.Batch(column_mix(), precision="fp32")
        try:
            b.set_shock_capturing(*coef)
            b.init()
            if tune:
                b.autotune(2)
            b.step(30)
            runs.append([b.fields(k) for k in range(4)])
        finally:
            b.close()
    for k in range(4):
        for f in ("rho", "u", "T"):
            assert np.array_equal(runs[0][k][f], runs[1][k][f]), (k, f)
