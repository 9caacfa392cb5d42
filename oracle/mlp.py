"""FP64 CPU oracle of the learned thermodynamic closure (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the CUDA path never does.

The closure maps the normalised state x = ((rho - c0)/s0, (e - c1)/s1) to
the normalised outputs y = ((T - m0)/r0, (P - m1)/r1, (c_s^2 - m2)/r2) of the
van der Waals fluid (Eqs. lbm_temp, Pvdw, vdW_speed_of_sound) with a
2 -> 64 -> 64 -> 3 multilayer perceptron:

    z1 = W1 x + b1,  h1 = gelu(z1)
    z2 = W2 h1 + b2, h2 = gelu(z2)
    y  = W3 h2 + b3

gelu is the tanh form of Hendrycks and Gimpel's Gaussian error linear unit,
gelu(z) = z (1 + tanh(k0 (z + k1 z^3))) / 2 with k0 = sqrt(2/pi), k1 =
0.044715, a smooth approximation of z Phi(z).  The loss is the mean squared
error over the batch and the three outputs.  The CUDA path keeps FP32 master
weights and evaluates the network with the weight matrices rounded to
bfloat16 (round to nearest even) and FP32 biases; ``quantize`` makes that
parameter vector and the oracle evaluates the same function from it in FP64.
Training uses AdamW (Loshchilov & Hutter's decoupled weight decay).

``closure`` is the gated closure as a solver step uses it: the network inside
the normalised training box |x0|, |x1| <= 1, the exact van der Waals
relations outside.
"""
import math

import numpy as np

H = 64
SHAPES = (("W1", (H, 2)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (3, H)), ("b3", (3,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Split a flat parameter vector (order of SHAPES) into named arrays."""
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def to_bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


K0, K1 = math.sqrt(2.0 / math.pi), 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def quantize(theta):
    """FP32 parameters with the weight matrices rounded to bfloat16, as float64."""
    q = np.asarray(theta, dtype=np.float32).astype(np.float64)
    k = 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        if name.startswith("W"):
            q[k:k + n] = to_bf16(q[k:k + n])
        k += n
    return q


def forward(theta, X):
    """X: (n, 2) normalised inputs -> (outputs (n, 3), cache)."""
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, Y):
    """Mean squared error over n samples x 3 outputs and its gradient (backpropagation)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    r = y - Y
    loss = float(np.sum(r * r) / (3 * n))
    dy = 2.0 * r / (3 * n)
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dz2 = (dy @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def init_params(u):
    """Initial weights from uniform numbers u in [-1, 1) (length NPARAM).

    W ~ U(-a, a) with a = sqrt(6 / (fan_in + fan_out)); biases zero.
    """
    theta = np.zeros(NPARAM)
    k = 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        if name.startswith("W"):
            a = math.sqrt(6.0 / (shape[0] + shape[1]))
            theta[k:k + n] = a * np.asarray(u[k:k + n])
        k += n
    return theta


def adamw_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (t counts from 1); returns the new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    theta = theta - lr * (mhat / (np.sqrt(vhat) + eps) + wd * theta)
    return theta, m, v


def vdw_targets(rho, e, a, b, R, cv):
    """Exact closure: T = (e + a rho)/c_v, P (Eq. Pvdw), c_s^2 (Eq. vdW_speed_of_sound)."""
    T = (e + a * rho) / cv
    P = rho * R * T / (1 - b * rho) - a * rho * rho
    cs2 = R * T * (1 + R / cv) / (1 - b * rho) ** 2 - 2 * a * rho
    return T, P, cs2


def closure(theta, scale, rho, e, a, b, R, cv):
    """Gated closure: (T, P, c_s^2, used) for arrays rho, e.

    scale = (c_rho, s_rho, c_e, s_e, m_T, r_T, m_P, r_P, m_c, r_c); the network
    (parameters theta as given) is used where both normalised inputs lie in
    [-1, 1], the exact relations (vdw_targets) elsewhere.
    """
    rho = np.asarray(rho, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    x = np.stack([(rho - scale[0]) / scale[1], (e - scale[2]) / scale[3]], axis=-1)
    used = np.all(np.abs(x) <= 1.0, axis=-1)
    y, _ = forward(theta, x.reshape(-1, 2))
    y = y.reshape(rho.shape + (3,))
    net = [scale[4] + scale[5] * y[..., 0], scale[6] + scale[7] * y[..., 1], scale[8] + scale[9] * y[..., 2]]
    ex = vdw_targets(rho, e, a, b, R, cv)
    return tuple(np.where(used, n, x_) for n, x_ in zip(net, ex)) + (used,)


def train(theta, X, Y, steps, batch, lr0, lr1, seed, wd=0.0):
    """AdamW on minibatches of (X, Y) with the forward pass on quantize(theta).

    The gradient of the rounded weights updates the full-precision master
    weights (straight-through).  Minibatch k of step t holds the samples
    floor((u + 1) n / 2) for the SplitMix64 values u of stream ``seed``
    (inputs.uniform) from index t * batch; the learning rate falls from lr0
    to lr1 along a half cosine.  Returns (theta, per-step losses).
    """
    import inputs
    n = X.shape[0]
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t in range(steps):
        u = inputs.uniform(seed, batch, start=t * batch)
        idx = np.minimum(((u + 1.0) * 0.5 * n).astype(np.int64), n - 1)
        loss, g = loss_and_grad(quantize(theta), X[idx], Y[idx])
        losses.append(loss)
        lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * t / steps))
        theta, m, v = adamw_step(theta, g, m, v, t + 1, lr, wd=wd)
    return theta, np.array(losses)
