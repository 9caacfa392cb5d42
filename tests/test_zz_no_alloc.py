"""lbm_totals_noalloc: conservation totals for callers that cannot allocate device memory.

Such a caller (one capturing a stream into a CUDA graph, a real-time loop
with a fixed memory budget, a framework with its own pool) cannot create a
handle, but can reduce device fields it owns.  The entry point keeps its
block partials in a fixed device array instead of allocating; this test
checks it against the totals of the handle-based lbm_moments on the same
state, on two calls in a row (the second call must not be disturbed by what
the first left in the shared array).  The file name sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import inputs

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


def device_fields(case, precision, steps):
    """Run the solver, return (device rho, u, T tensors, reference totals from lbm_moments)."""
    import torch
    s = P.Solver(case, precision=precision)
    try:
        s.init().step(steps)
        shape = tuple(reversed(case.shape))
        rho = torch.empty(shape, dtype=torch.float64, device="cuda")
        u = torch.empty((case.D,) + shape, dtype=torch.float64, device="cuda")
        T = torch.empty(shape, dtype=torch.float64, device="cuda")
        ref = np.empty(case.D + 2)
        P.lbm_moments_device(s.h, rho, u, T, ref)
        torch.cuda.synchronize()
        return rho, u, T, ref
    finally:
        s.close()


def noalloc_totals(case, rho, u, T):
    import torch
    out = torch.full((case.D + 2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P.lbm_totals_noalloc(case.lattice, case.nodes, rho, u, T, case.eos["a"], case.cv, out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def close(got, want, tol):
    scale = np.abs(want).max()
    return np.all(np.abs(got - want) <= tol * scale)


def test_noalloc_totals_match_lbm_moments_twice():
    # FP64 state: the two routes agree to round-off (tolerance of the FP64 parity tests)
    a = inputs.add_noise(inputs.tgv(shape=(37, 21, 13)), 2)
    sc = inputs.scenario("tgv_d3q27")
    a.tau = sc["tau"] * 0.02 / sc["nu"]             # lattice viscosity 0.02 on this small box
    rho, u, T, ref = device_fields(a, "fp64", 10)
    first = noalloc_totals(a, rho, u, T)
    assert close(first, ref, 1e-12), (first, ref)

    # second call, different lattice and size, same shared scratch
    b = inputs.riemann(Nx=300, Ny=5)
    rho2, u2, T2, ref2 = device_fields(b, "fp64", 20)
    second = noalloc_totals(b, rho2, u2, T2)
    assert close(second, ref2, 1e-12), (second, ref2)

    # and the first input again: the result is reproduced exactly
    again = noalloc_totals(a, rho, u, T)
    assert np.array_equal(again, first)


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    import torch
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(P.LbmError) as ei:
        P.lbm_totals_noalloc(27, 67108864 + 1, t, t, t, 0.3, 8.0, t)
    assert ei.value.code == P.LBM_EINVAL and "67108864" in str(ei.value)
    with pytest.raises(P.LbmError):
        P.lbm_totals_noalloc(10, 4, t, t, t, 0.3, 8.0, t)
