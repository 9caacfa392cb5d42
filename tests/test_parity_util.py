"""The parity check itself (no GPU): a single wrong node that a relative L2
bound lets through is caught by the per-node bound, while errors spread over
the box at the tolerance pass."""
import numpy as np
import pytest

from parity_util import NODE_MULT, NODE_MULT_FP32, assert_parity, parity_errors


def _fields(shape=(13, 21, 37), seed=0):
    rng = np.random.default_rng(seed)
    rho = 0.6 + 0.01 * rng.standard_normal(shape)
    u = 0.1 * rng.standard_normal((3,) + shape)
    T = 0.15 + 0.001 * rng.standard_normal(shape)
    return dict(rho=rho, u=u, T=T)


def test_single_wrong_node_is_caught_by_the_node_bound():
    want = _fields()
    got = {k: v.copy() for k, v in want.items()}
    n = want["rho"].size
    tol = 1e-5
    # one node at a tile seam off by half of what the L2 bound would allow
    d = 0.5 * tol * np.sqrt(n) * np.sqrt(np.mean(want["rho"] ** 2))
    got["rho"][5, 8, 31] += d
    l2, node = parity_errors(got, want)
    assert l2["rho"] <= tol                      # the norm alone would pass
    assert node["rho"] > NODE_MULT_FP32 * tol
    with pytest.raises(AssertionError, match="per-node"):
        assert_parity(got, want, tol, "planted")


def test_spread_errors_at_the_tolerance_pass():
    want = _fields()
    rng = np.random.default_rng(1)
    tol = 1e-5
    got = {k: v * (1 + 0.5 * tol * rng.standard_normal(v.shape)) for k, v in want.items()}
    l2 = assert_parity(got, want, tol, "spread")
    assert max(l2.values()) <= tol


def test_l2_bound_still_applies():
    want = _fields()
    got = {k: v * (1 + 3e-5) for k, v in want.items()}
    with pytest.raises(AssertionError, match="relative L2"):
        assert_parity(got, want, 1e-5, "scaled")


def test_fp64_tolerances_get_the_tight_node_bound():
    want = _fields()
    got = {k: v.copy() for k, v in want.items()}
    tol = 1e-12
    got["T"][0, 0, 0] += 30 * tol * np.sqrt(np.mean(want["T"] ** 2))     # 30x tol at one node
    with pytest.raises(AssertionError, match="per-node"):
        assert_parity(got, want, tol, "fp64 planted")
    assert_parity(got, want, tol, "fp64 planted, loose", node_mult=NODE_MULT_FP32)
