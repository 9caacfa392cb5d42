"""Pins of the FP64 MLP oracle of the learned closure (oracle/mlp.py)."""
import math

import numpy as np
import pytest
from scipy.stats import norm

import inputs
from oracle import mlp, thermo


def params(seed=3):
    return mlp.init_params(inputs.uniform(seed, mlp.NPARAM))


def data(n=37, seed=9):
    X = np.stack([inputs.uniform(seed, n), inputs.uniform(seed + 1, n)], axis=1)
    Y = np.stack([np.sin(X[:, 0]) * X[:, 1], X[:, 0] ** 2 - 0.3, np.cos(X[:, 1])], axis=1)
    return X, Y


def test_backward_matches_central_differences():
    theta = params()
    X, Y = data()
    _, g = mlp.loss_and_grad(theta, X, Y)
    rng = np.random.default_rng(0)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, X, Y)[0] - mlp.loss_and_grad(tm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-11, (k, fd, g[k])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.concatenate([inputs.uniform(5, 1000) * 10.0 ** np.arange(-5, 5).repeat(100),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.to_bf16(v), ref)
    assert mlp.to_bf16(np.float32(1.0 + 2 ** -8)) == 1.0            # tie to even
    assert mlp.to_bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6


def test_gelu_tanh_form_approximates_x_times_normal_cdf():
    """The tanh form stays within 5e-4 of z Phi(z) (Hendrycks & Gimpel) and is odd up to z."""
    z = np.linspace(-8, 8, 1601)
    err = np.abs(mlp.gelu(z) - z * norm.cdf(z))
    assert err.max() < 5e-4
    assert err.max() > 1e-5                      # it is the approximation, not the erf form
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14)
    assert mlp.gelu(0.0) == 0.0
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_quantize_rounds_weights_not_biases():
    th = params() + 1e-3 * inputs.uniform(11, mlp.NPARAM)
    q = mlp.unpack(mlp.quantize(th))
    p = mlp.unpack(th)
    for name, _ in mlp.SHAPES:
        if name.startswith("W"):
            assert np.array_equal(q[name], mlp.to_bf16(p[name]))
        else:
            assert np.array_equal(q[name], np.float32(p[name]).astype(np.float64))


def test_closure_gate_uses_exact_relations_outside_the_box():
    a, b, R, cv = 0.25, 1 / 3, 8 / 3, 8.0
    theta = params()
    scale = np.array([0.6, 0.3, 0.5, 0.2, 0.1, 0.05, 0.2, 0.1, 0.3, 0.1])
    rho = np.array([0.5, 0.95, 0.2, 0.61])
    e = np.array([0.45, 0.5, 0.5, 0.75])
    T, P, c2, used = mlp.closure(theta, scale, rho, e, a, b, R, cv)
    assert used.tolist() == [True, False, False, False]
    Te, Pe, ce = mlp.vdw_targets(rho, e, a, b, R, cv)
    assert np.array_equal(T[1:], Te[1:]) and np.array_equal(P[1:], Pe[1:]) and np.array_equal(c2[1:], ce[1:])
    y, _ = mlp.forward(theta, np.array([[(0.5 - 0.6) / 0.3, (0.45 - 0.5) / 0.2]]))
    assert np.allclose([T[0], P[0], c2[0]], [0.1 + 0.05 * y[0, 0], 0.2 + 0.1 * y[0, 1], 0.3 + 0.1 * y[0, 2]],
                       rtol=1e-15)


def test_adamw_first_step_is_signed_lr():
    """With m = v = 0 the bias-corrected first step is lr * g/(|g| + eps) (Kingma & Ba)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adamw_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    th, _, _ = mlp.adamw_step(np.ones(3), np.zeros(3), np.zeros(3), np.zeros(3), 1, lr=0.1, wd=0.5)
    assert np.allclose(th, 1.0 - 0.1 * 0.5)


def xphi(z):
    """z Phi(z): the GELU that the tanh form approximates within 5e-4 (pinned above)."""
    return z * 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))


def sparse_network():
    """Parameters with a few non-zero entries, so the outputs follow by hand.
    Layer 1: unit 0 sees x_0, unit 5 sees -x_1 + 0.25.  Layer 2: unit 3 sees h1_0,
    unit 7 sees 2 h1_5 - 0.5.  Outputs: y_0 = h2_3, y_1 = 0.1 - h2_7, y_2 = 0.3."""
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["W1"][0, 0] = 1.0
    p["W1"][5, 1], p["b1"][5] = -1.0, 0.25
    p["W2"][3, 0] = 1.0
    p["W2"][7, 5], p["b2"][7] = 2.0, -0.5
    p["W3"][0, 3] = 1.0
    p["W3"][1, 7], p["b3"][1] = -1.0, 0.1
    p["b3"][2] = 0.3
    return mlp.pack(p)


SPARSE_X = np.array([[0.7, -0.4], [-1.2, 0.9], [1.5, -1.1]])


def forward_wiring_error():
    """Largest deviation of mlp.forward on the sparse network from the hand composition."""
    y, _ = mlp.forward(sparse_network(), SPARSE_X)
    err = 0.0
    for (x0, x1), out in zip(SPARSE_X, y):
        want = (xphi(xphi(x0)), 0.1 - xphi(2.0 * xphi(0.25 - x1) - 0.5), 0.3)
        err = max(err, float(np.abs(out - np.array(want)).max()))
    return err


def test_forward_wiring_of_a_sparse_network():
    assert forward_wiring_error() < 3e-3          # the tanh GELU's own deviation, through two layers


def loss_normalisation_error():
    """The loss of outputs offset by (c_0, c_1, c_2) is (c_0^2 + c_1^2 + c_2^2)/3, whatever n."""
    theta = sparse_network()
    y, _ = mlp.forward(theta, SPARSE_X)
    c = np.array([0.2, -0.5, 0.1])
    loss, _ = mlp.loss_and_grad(theta, SPARSE_X, y - c)
    return abs(loss / (np.sum(c * c) / 3.0) - 1.0)


def test_loss_is_the_mean_square_over_samples_and_outputs():
    assert loss_normalisation_error() < 1e-12


def adamw_constant_gradient_error(steps=25):
    """With a constant gradient g the bias-corrected moments are g and g^2 at every t,
    so each step moves theta by lr g/(|g| + eps) (Kingma & Ba; wd = 0)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    err = 0.0
    for t in range(1, steps + 1):
        th, m, v = mlp.adamw_step(th, g, m, v, t, lr=0.01)
        want = -0.01 * t * g / (np.abs(g) + 1e-8)
        err = max(err, float(np.abs(th / want - 1.0).max()))
    return err


def test_adamw_bias_correction_keeps_constant_gradient_steps_equal():
    assert adamw_constant_gradient_error() < 1e-9


def test_targets_are_the_oracle_closure():
    rho = np.array([0.3, 0.6, 0.9]); T = np.array([0.09, 0.15, 0.12])
    a, b, R, cv = 0.25, 1 / 3, 8 / 3, 8.0
    e = thermo.internal_energy(rho, T, a, cv)
    Tt, P, cs2 = mlp.vdw_targets(rho, e, a, b, R, cv)
    assert np.allclose(Tt, T, rtol=1e-15)
    assert np.allclose(P, thermo.pressure(rho, T, a, b, R), rtol=1e-15)
    assert np.allclose(cs2, thermo.sound_speed_sq(rho, T, a, b, R, cv), rtol=1e-15)


def test_training_reduces_loss():
    theta = params()
    X, Y = data(200)
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    l0 = mlp.loss_and_grad(theta, X, Y)[0]
    for t in range(1, 301):
        _, g = mlp.loss_and_grad(theta, X, Y)
        theta, m, v = mlp.adamw_step(theta, g, m, v, t, lr=3e-3)
    assert mlp.loss_and_grad(theta, X, Y)[0] < 0.05 * l0


def test_oracle_closure_hook_with_exact_relations_reproduces_the_exact_step():
    """The Model closure hook, fed the exact relations, gives the standard step (round-off)."""
    from oracle import lbm
    import mlp_util
    a, b, R, cv = mlp_util.shock_eos()
    c = mlp_util.shock_tube(2, (96, 3))
    runs = []
    for hook in (None, lambda rho, e: mlp.vdw_targets(rho, e, a, b, R, cv)):
        m = lbm.Model(c.D, c.shape, c.eos, c.tau, c.Pr, c.cv, c.x_low, c.x_high)
        m.closure = hook
        s = lbm.Sim(m, c.rho, c.u, c.T)
        s.step(40)
        runs.append(s.fields())
    for k in ("rho", "T"):
        assert np.allclose(runs[0][k], runs[1][k], rtol=1e-12, atol=0)
    assert np.allclose(runs[0]["u"], runs[1]["u"], rtol=0, atol=1e-13)


def test_oracle_training_fits_the_closure():
    """The oracle's own AdamW loop fits the closure on its box (normalised RMS < 2e-2)."""
    import mlp_util
    theta, scale, losses = mlp_util.oracle_network(steps=600)
    assert losses[-50:].mean() < 0.02 * losses[:10].mean()
    a, b, R, cv = mlp_util.shock_eos()
    rho = 0.385 + 0.1 * inputs.uniform(99, 500)
    T = 0.105 + 0.018 * inputs.uniform(98, 500)
    e = cv * T - a * rho
    Tn, Pn, cn, used = mlp.closure(mlp.quantize(theta), scale, rho, e, a, b, R, cv)
    Te, Pe, ce = mlp.vdw_targets(rho, e, a, b, R, cv)
    assert used.all()
    assert np.sqrt(np.mean(((Pn - Pe) / scale[7]) ** 2)) < 2e-2
