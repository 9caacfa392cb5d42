"""GPU tests of the learned closure (include/lbm_mlp.h) against the MLP oracle.

* initial weights, loss and gradient, and the gated closure of the CUDA
  kernels against oracle/mlp.py on the same parameters;
* the fused step with the learned closure against the oracle step with the
  same (oracle-trained) network as its closure hook;
* training on solver states (GPU): what it gains over the untrained network,
  and the density error of a D3Q27 shock tube run with the learned closure
  against the exact closure (FP64, itself pinned to the oracle elsewhere).
"""
import numpy as np
import pytest

import inputs
import mlp_util
from oracle import lbm as olbm
from oracle import mlp
from parity_util import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32_SHOCK_TOL = 5e-5      # FP32 path on shock cases (as the exact-closure parity tests)


@pytest.fixture(scope="module")
def P():
    import paper_2510_14712_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()
    return P


@pytest.fixture(scope="module")
def onet():
    theta, scale, _ = mlp_util.oracle_network()
    return theta, scale


def make_net(P, seed=3):
    return P.Closure(*mlp_util.shock_eos(), seed=seed)


def perturbed_params(seed):
    th = mlp.init_params(inputs.uniform(seed, mlp.NPARAM)) + 0.05 * inputs.uniform(seed + 1, mlp.NPARAM)
    return th.astype(np.float32)


def test_initial_weights_match_oracle(P):
    net = make_net(P, seed=3)
    want = mlp.init_params(inputs.uniform(3, mlp.NPARAM)).astype(np.float32)
    assert np.array_equal(net.params, want)
    net.close()


# tolerances (relative L2) of the gradient against the FP64 oracle on the same
# bfloat16 weights.  Warp form: FP32 paths for b2, W3, b3; bfloat16-rounded
# dL/dz2 in dW2 and in the input gradient of layer 2 (W1, b1).  Tensor-core
# form: every product takes its FP32 operands as bfloat16 hi + lo, so all
# gradients are at the FP32 level.
GRAD_TOL = {"warp": dict(W1=1e-2, b1=1e-2, W2=1e-2, b2=1e-4, W3=1e-4, b3=1e-4),
            "tcgen05": dict(W1=1e-4, b1=1e-4, W2=1e-4, b2=1e-4, W3=1e-4, b3=1e-4)}


def check_loss_and_gradient(P, net, mma, n, seed):
    net.mma = P.LBM_MLP_MMA_TCGEN05 if mma == "tcgen05" else P.LBM_MLP_MMA_WARP
    th = perturbed_params(seed)
    net.params = th
    X = np.stack([inputs.uniform(seed + 2, n), inputs.uniform(seed + 3, n)], axis=1).astype(np.float32)
    Y = np.stack([np.sin(2 * X[:, 0]) * X[:, 1], X[:, 0] ** 2 - 0.3, np.cos(X[:, 1])], axis=1).astype(np.float32)
    loss, g = net.loss_grad(X, Y)
    lo, go = mlp.loss_and_grad(mlp.quantize(th), X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo, (loss, lo)
    gp, op = mlp.unpack(g), mlp.unpack(go)
    for name, _ in mlp.SHAPES:
        err = rel_l2(gp[name], op[name])
        assert err <= GRAD_TOL[mma][name], (mma, name, err)


@pytest.mark.parametrize("mma", ["tcgen05", "warp"])
@pytest.mark.parametrize("n", [1, 37, 1000, 4099])
def test_loss_and_gradient_match_oracle(P, n, mma):
    net = make_net(P)
    check_loss_and_gradient(P, net, mma, n, 5)
    net.close()


@pytest.mark.parametrize("n", [128, 129, 19457, 60001])
def test_tensor_core_gradient_over_many_groups(P, n):
    """Full and ragged groups of 128 samples; above 152 groups a block
    accumulates several groups in tensor memory."""
    net = make_net(P)
    assert net.mma == P.LBM_MLP_MMA_TCGEN05                 # the default path
    check_loss_and_gradient(P, net, "tcgen05", n, 11)
    net.close()


def test_closure_matches_oracle_inside_and_outside_the_box(P):
    net = make_net(P)
    th = perturbed_params(9)
    net.params = th
    a, b, R, cv = mlp_util.shock_eos()
    scale = np.array([0.4, 0.1, 0.8, 0.05, 0.11, 0.02, 0.5, 0.2, 0.4, 0.1])
    net.scaling = scale
    n = 3001
    x0 = 1.3 * inputs.uniform(31, n)
    x1 = 1.3 * inputs.uniform(32, n)
    keep = (np.abs(np.abs(x0) - 1) > 1e-4) & (np.abs(np.abs(x1) - 1) > 1e-4)
    rho = scale[0] + scale[1] * x0[keep]
    e = scale[2] + scale[3] * x1[keep]
    out = net.predict(torch.tensor(rho, device="cuda"), torch.tensor(e, device="cuda")).cpu().numpy()
    T, Pr, c2, used = mlp.closure(mlp.quantize(th), scale, rho, e, a, b, R, cv)
    assert np.array_equal(out[:, 3] == 1.0, used)
    assert 0.3 < used.mean() < 0.8
    for k, (want, r) in enumerate(((T, scale[5]), (Pr, scale[7]), (c2, scale[9]))):
        got = out[:, k]
        # network: a few 1e-6 of the output range; exact FP32 relations: FP32 rounding
        assert np.all(np.abs(got[used] - want[used]) <= 1e-5 * r + 1e-6 * np.abs(want[used])), k
        assert np.allclose(got[~used], want[~used], rtol=2e-5, atol=1e-7), k
    net.close()


def oracle_mlp_run(case, steps, closure):
    m = olbm.Model(case.D, case.shape, case.eos, case.tau, case.Pr, case.cv, case.x_low, case.x_high)
    m.closure = closure
    s = olbm.Sim(m, case.rho, case.u, case.T)
    s.step(steps)
    q = s.macroscopic()
    I = m.interior()
    # temperature from the exact caloric relation, as the C interface reports it
    T = (q["e"][I] + m.a * q["rho"][I]) / m.cv
    return dict(rho=q["rho"][I], u=np.stack([ua[I] for ua in q["u"]]), T=T)


def gpu_mlp_run(P, case, steps, theta, scale, chunk=None):
    net = make_net(P)
    net.params = theta
    net.scaling = scale
    s = P.Solver(case, precision="fp32").init()
    try:
        net.attach(s)
        assert P.lbm_get_closure(s.h) == P.LBM_CLOSURE_MLP
        done = 0
        while done < steps:
            k = steps - done if chunk is None else min(chunk, steps - done)
            s.step(k)
            done += k
        return s.fields()
    finally:
        s.close()
        net.close()


def test_mlp_every_tile_shape_gives_the_same_step(P, onet):
    """The learned closure's tile candidates (position-form stage A, row form on
    inflow / outflow faces) step a D3Q27 shock tube alike."""
    theta, scale = onet
    case = mlp_util.shock_tube(3, (96, 16, 6))
    net = make_net(P)
    net.params = theta
    net.scaling = scale
    s = P.Solver(case, precision="fp32")
    try:
        ref = None
        n = None
        for k in range(16):
            s.init()
            net.attach(s)
            if n is None:
                n = P.lbm_tile_count(s.h)
                assert n >= 2
            if k >= n:
                break
            P.lbm_set_tile(s.h, k)
            s.step(12)
            got = s.fields()
            if ref is None:
                ref = got
                continue
            for key in ("rho", "u", "T"):
                assert rel_l2(got[key], ref[key]) < 1e-6, "tile %d of %d: %s" % (k, n, key)
    finally:
        s.close()
        net.close()


@pytest.mark.parametrize("D,shape,steps", [(2, (256, 4), 300), (2, (197, 3), 120), (3, (72, 6, 5), 40)])
def test_mlp_step_matches_oracle(P, onet, D, shape, steps):
    theta, scale = onet
    case = mlp_util.shock_tube(D, shape)
    want = oracle_mlp_run(case, steps, mlp_util.oracle_closure(theta, scale))
    got = gpu_mlp_run(P, case, steps, theta, scale)
    errs = {k: rel_l2(got[k], want[k]) for k in ("rho", "u", "T")}
    assert all(v <= FP32_SHOCK_TOL for v in errs.values()), errs


def test_mlp_step_differs_from_exact_closure(P, onet):
    """The attached network is really used: its closure error shows in the state."""
    theta, scale = onet
    case = mlp_util.shock_tube(2, (256, 4))
    got = gpu_mlp_run(P, case, 300, theta, scale)
    s = P.Solver(case, precision="fp32").init().step(300)
    ex = s.fields()
    s.close()
    assert rel_l2(got["rho"], ex["rho"]) > 1e-6


def test_attach_rules(P, onet):
    theta, scale = onet
    net = make_net(P)
    case = mlp_util.shock_tube(2, (64, 2))
    s64 = P.Solver(case, precision="fp64").init()
    with pytest.raises(P.LbmError):
        net.attach(s64)                                  # no scaling yet
    net.params, net.scaling = theta, scale
    with pytest.raises(P.LbmError):
        net.attach(s64)                                  # FP64 storage
    s64.close()
    s = P.Solver(case, precision="fp32", step_kernel=P.LBM_STEP_MULTIPASS).init()
    net.attach(s)
    with pytest.raises(P.LbmError):
        s.step(1)                                        # learned closure: fused step only
    P.lbm_set_step_kernel(s.h, P.LBM_STEP_FUSED)
    s.step(2)
    P.Closure.detach(s)
    assert P.lbm_get_closure(s.h) == P.LBM_CLOSURE_EXACT
    s.step(1)
    s.close()
    net.close()


# ---- training on solver states ------------------------------------------------

@pytest.fixture(scope="module")
def trained(P):
    """A network trained on the GPU on ~10M states of the Riemann problem and
    12 D2Q9 shock tubes (Ma 1.1 .. 1.25), plus a held-out shock tube."""
    net = make_net(P, seed=11)
    runs = inputs.closure_training_runs()
    rho, e = net.collect_runs(runs, snapshots=50, every=20, precision="fp32")
    net.fit_scaling(rho, e)
    held = mlp_util.shock_tube(2, (2048, 3), Ma=1.17, seed=404)
    hrho, he = net.collect_runs([(held, 1.0)], snapshots=5, every=200, precision="fp32")
    before = net.predict(hrho, he).cpu().numpy()
    losses = net.train(rho, e, batch=8192, steps=60000, lr0=3e-3, lr1=1e-6, seed=5)
    after = net.predict(hrho, he).cpu().numpy()
    yield dict(net=net, n=rho.numel(), losses=losses, before=before, after=after,
               held=(hrho.cpu().numpy(), he.cpu().numpy()))
    net.close()


def closure_errors(out, rho, e):
    a, b, R, cv = mlp_util.shock_eos()
    want = mlp.vdw_targets(rho, e, a, b, R, cv)
    return [float(np.sqrt(np.mean(((out[:, k] - want[k]) / want[k]) ** 2))) for k in range(3)]


def test_training_on_solver_states(trained):
    assert trained["n"] > 9_500_000
    L = trained["losses"]
    assert np.all(np.isfinite(L))
    assert L[-100:].mean() < 1e-3 * L[:10].mean()
    rho, e = trained["held"]
    before = closure_errors(trained["before"], rho, e)
    after = closure_errors(trained["after"], rho, e)
    assert trained["after"][:, 3].mean() > 0.99          # held-out states inside the training box
    # what training gains: relative RMS closure error on held-out states
    for k in range(3):
        assert after[k] < 2e-4, (k, after)
        assert after[k] < 1e-2 * before[k], (k, before, after)


def test_learned_closure_shock_tube_d3q27(P, trained):
    """D3Q27 shock tube (Ma 1.15, 768 x 32 x 32, 1000 steps): density with the
    learned closure within 1e-3 (relative L2) of the exact closure in FP64."""
    net = trained["net"]
    case = inputs.shock_tube_3d(seed=21)
    ref = P.Solver(case, precision="fp64").init().step(1000)
    want = ref.fields()
    ref.close()
    s = P.Solver(case, precision="fp32").init()
    s.step(1000)
    exact32 = s.fields()
    s.close()
    s = P.Solver(case, precision="fp32").init()
    net.attach(s)
    s.step(1000)
    got = s.fields()
    s.close()
    err = rel_l2(got["rho"], want["rho"])
    err32 = rel_l2(exact32["rho"], want["rho"])
    print("rho rel L2: learned %.3e  exact fp32 %.3e" % (err, err32))
    assert err <= 1e-3, err
    # the state stayed inside the training box for almost every node
    r = torch.tensor(got["rho"].ravel(), device="cuda")
    u2 = (got["u"] ** 2).sum(axis=0).ravel()
    a, _, _, cv = mlp_util.shock_eos()
    e = torch.tensor(cv * got["T"].ravel() - a * got["rho"].ravel(), device="cuda")
    used = net.predict(r, e).cpu().numpy()[:, 3]
    assert used.mean() > 0.95, used.mean()
    assert np.isfinite(u2).all()


def test_mlp_argument_errors(P):
    net = make_net(P)
    r = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(P.LbmError):
        net.predict(r, r)                                # no scaling yet
    with pytest.raises(P.LbmError):
        net.scaling = np.array([0.4, 0.0, 0.8, 0.05, 0.1, 0.02, 0.5, 0.2, 0.4, 0.1])   # zero half-width
    net.scaling = np.array([0.4, 0.1, 0.8, 0.05, 0.1, 0.02, 0.5, 0.2, 0.4, 0.1])
    with pytest.raises(P.LbmError):
        net.train(r, r, batch=16, steps=1)               # batch below 32
    with pytest.raises(P.LbmError):
        net.params = np.full(mlp.NPARAM, np.nan, dtype=np.float32)
    e0 = torch.empty(0, dtype=torch.float64, device="cuda")
    with pytest.raises(P.LbmError):
        net.predict(e0, e0)                              # empty input
    out = net.predict(r, r)
    assert out.shape == (4, 4)
    net.close()


@pytest.fixture(scope="module")
def trained_strong(P):
    """A network trained on the Riemann problem and 12 D2Q9 tubes of Ma 1.1 .. 1.5 on the
    U^2 = 16 scale of the Ma 1.47 workload, run with shock capturing."""
    sc = inputs.scenario("strong_shock_d3q27")
    net = P.Closure(sc["eos"]["a"], sc["eos"]["b"], sc["eos"]["R"], sc["cv"], seed=11)
    runs = inputs.closure_training_runs(table="strong_posts_d2q9", Ma_max=1.5)
    rho, e = net.collect_runs(runs, snapshots=50, every=20, precision="fp32", shock_capturing=(0.3, 0.0, 0.3))
    net.fit_scaling(rho, e)
    net.train(rho, e, batch=8192, steps=60000, lr0=3e-3, lr1=1e-6, seed=5)
    yield net
    net.close()


def test_learned_closure_ma147_shock_d3q27(P, trained_strong):
    """The workloads' Ma 1.47 shock (D3Q27 768 x 32 x 32, shock capturing, 1000 steps)
    with the learned closure stays finite and within 1e-2 (relative L2 of rho) of the
    exact closure in FP64.  The strong shock amplifies any perturbation: the exact
    closure in FP32 is already 9e-4 away from FP64 here (the 1e-3 bar is met at
    Ma 1.15, test_learned_closure_shock_tube_d3q27)."""
    case = inputs.strong_shock(3, (768, 32, 32), seed=21)
    out = {}
    for name, prec, net in (("ref", "fp64", None), ("ex32", "fp32", None), ("mlp", "fp32", trained_strong)):
        s = P.Solver(case, precision=prec)
        P.lbm_set_shock_capturing(s.h, 0.3, 0.0, 0.3)
        if net is not None:
            net.attach(s)
        s.init().step(1000)
        out[name] = s.fields()
        s.close()
    err = rel_l2(out["mlp"]["rho"], out["ref"]["rho"])
    err32 = rel_l2(out["ex32"]["rho"], out["ref"]["rho"])
    print("Ma 1.47 rho rel L2 vs exact fp64: learned %.3e, exact fp32 %.3e" % (err, err32))
    assert np.isfinite(out["mlp"]["rho"]).all()
    assert err <= 1e-2, err
