"""Learned initial guess on the GPU against the oracle network (oracle/mlp.py).

* forward outputs, loss and every gradient block match the FP64 oracle run
  with the same BF16-rounded weight matrices, for batches that span several
  64-row tiles, several split-K chunks of 512 samples and a ragged tail;
* one Adam step from fresh moments matches the oracle's Adam step;
* repeated steps on one batch lower the loss (training works end to end);
* a sweep with the learned column gives the oracle's solution, and its guess
  residual is never above the plain extrapolation's from the same fit.
"""
import math

import numpy as np
import pytest

from oracle import kernels, mlp, sweep as osweep
from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu

MAT = kernels.Material(1.0, 0.25, 1.0)


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    c.set_material(MAT.E, MAT.nu, MAT.rho)
    yield c
    c.close()


def _theta(seed, scale=0.15):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=mlp.NPARAM) * scale).astype(np.float32)


def _batch(seed, n):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, mlp.IN)).astype(np.float32)
    t = rng.normal(size=(n, mlp.OUT)).astype(np.float32)
    return x, t


def _blocks(v):
    out, k = {}, 0
    for name, shape in mlp.SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(v[k:k + n], dtype=np.float64)
        k += n
    return out


def test_num_params(ctx):
    assert ctx.mlp_num_params() == mlp.NPARAM


@pytest.mark.parametrize("n", [1, 63, 1000, 1537])
def test_forward_matches_oracle(ctx, n):
    theta = _theta(1)
    ctx.mlp_set_weights(theta)
    assert np.array_equal(ctx.mlp_get_weights(), theta)
    x, _ = _batch(2, n)
    y = ctx.mlp_forward(x)
    y_ref, _ = mlp.forward(mlp.compute_weights(theta), x.astype(np.float64))
    # FP32 accumulation over 256 terms of O(0.1) products
    assert np.max(np.abs(y - y_ref)) <= 2e-5 * max(1.0, np.max(np.abs(y_ref)))


@pytest.mark.parametrize("n", [5, 700, 1537])
def test_gradient_matches_oracle(ctx, n):
    theta = _theta(3)
    ctx.mlp_set_weights(theta)
    x, t = _batch(4, n)
    loss, g = ctx.mlp_gradient(x, t)
    loss_ref, g_ref = mlp.loss_and_grad(mlp.compute_weights(theta), x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    gb = _blocks(g)
    for name, _ in mlp.SIZES:
        ref = np.asarray(g_ref[name], dtype=np.float64).ravel()
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(gb[name] - ref)) <= 1e-4 * scale + 1e-7, name


def test_adam_step_matches_oracle(ctx):
    theta = _theta(5)
    ctx.mlp_set_weights(theta)
    x, t = _batch(6, 800)
    lr = 1e-3
    ctx.mlp_train_step(x, t, lr)
    new = ctx.mlp_get_weights().astype(np.float64)
    _, g_ref = mlp.loss_and_grad(mlp.compute_weights(theta), x.astype(np.float64), t.astype(np.float64))
    g_ref = mlp.pack(g_ref)
    want, _, _ = mlp.adam_step(theta.astype(np.float64), g_ref, np.zeros_like(g_ref), np.zeros_like(g_ref), 1, lr)
    # the first Adam step moves each parameter by about lr * sign(g); where |g|
    # is at the FP32 noise level of the gradient the sign is not determined
    big = np.abs(g_ref) > 1e-3 * np.max(np.abs(g_ref))
    assert np.max(np.abs(new - want)[big]) <= 1e-6
    assert np.max(np.abs(new - theta)) <= lr * (1 + 1e-5)


def test_training_lowers_loss(ctx):
    ctx.mlp_init(7)
    x, _ = _batch(8, 2048)
    # a smooth target the network can fit
    t = np.stack([np.tanh(x[:, 0] - 0.5 * x[:, 3]), 0.3 * x[:, 1] * x[:, 2] / (1 + x[:, 1] ** 2)], axis=1)
    losses = [ctx.mlp_train_step(x, t.astype(np.float32), 3e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0]


def test_invalid_arguments(ctx, B):
    with pytest.raises(B.BemError):
        ctx.mlp_set_weights(np.zeros(10, dtype=np.float32))
    with pytest.raises(B.BemError):
        ctx.mlp_set_training(-1, 1e-3)
    with pytest.raises(B.BemError):
        ctx.mlp_set_training(2, float("nan"))


@pytest.fixture(scope="module")
def oracle_sweep():
    mesh = inputs.cavity_problem(4)
    T, N = 8.0, 32
    eta = 5.0 / T
    ref = osweep.solve_sweep(mesh, MAT, T, N, eta, inputs.heaviside_history(N))
    return mesh, T, N, eta, ref


def test_sweep_with_learned_guess(ctx, B, oracle_sweep):
    mesh, T, N, eta, ref = oracle_sweep
    o = B.default_opts(dense=1, precision=0, guess=B.GUESS_MLP, tol=1e-7, leaf_size=16)
    ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
    ctx.set_window(eta, 1)
    ctx.mlp_init(11)
    ctx.mlp_set_training(8, 1e-3)
    stats = ctx.solve_sweep(T, N, inputs.heaviside_history(N), mesh.pattern, o)
    assert all(s["converged"] == 1 for s in stats)
    for k in range(N // 2 + 1):
        a = ctx.get_frequency_solution(k)
        assert np.linalg.norm(a - ref["a"][k]) <= 1e-4 * np.linalg.norm(ref["a"][k]), k
        assert stats[k]["s_im"] == pytest.approx(k * 2 * math.pi / T)
    for s in stats[4:]:
        # the learned column widens the least-squares span: never worse than
        # the extrapolation alone (both measured with FP32 operator products)
        assert s["guess_residual"] <= s["sem_residual"] * (1 + 1e-3) + 1e-6, s["k"]
    # the weights moved (online training ran)
    th = ctx.mlp_get_weights()
    ctx2 = B.Context(0)
    try:
        ctx2.mlp_init(11)
        assert not np.array_equal(th, ctx2.mlp_get_weights())
    finally:
        ctx2.close()
