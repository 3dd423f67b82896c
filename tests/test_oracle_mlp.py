"""Pins of the oracle's learned-normal perceptron: the analytic gradient
against central finite differences, and Adam's first step (a closed form:
with bias correction the first update is -lr g / (|g| + eps))."""
import numpy as np

from oracle import mlp


def _batch(rng, B=16):
    X = rng.uniform(0, 1, (B, 27))
    n = rng.standard_normal((B, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    k = rng.uniform(-0.2, 0.2, B)
    return X, n, k


def test_parameter_count():
    assert mlp.NPARAM == 64 * 27 + 64 + 64 * 64 + 64 + 4 * 64 + 4 == 6212


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(1)
    theta[64 * 27:64 * 27 + 64] = rng.uniform(0.05, 0.2, 64)      # positive biases: few ReLU kinks
    X, n, k = _batch(rng)
    L, g = mlp.loss_and_grad(theta, X, n, k, lam=0.3)
    idx = rng.choice(mlp.NPARAM, 300, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        num = (mlp.loss_and_grad(tp, X, n, k, 0.3)[0] - mlp.loss_and_grad(tm, X, n, k, 0.3)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, num, g[i])


def test_adam_first_step_and_convergence():
    theta = np.array([3.0, -2.0])
    g = np.array([0.5, -4.0])
    t1, m, v = mlp.adam(theta, g, np.zeros(2), np.zeros(2), 1, lr=0.1)
    assert np.allclose(t1 - theta, -0.1 * g / (np.abs(g) + 1e-8), atol=1e-12)
    x, m, v = np.array([5.0]), np.zeros(1), np.zeros(1)
    for t in range(1, 3001):
        x, m, v = mlp.adam(x, 2 * (x - 1.0), m, v, t, lr=0.05)
    assert abs(x[0] - 1.0) < 1e-3


def test_training_reduces_the_loss_on_planes():
    rng = np.random.default_rng(3)
    C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], float)
    n = rng.standard_normal((256, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    X = np.clip(0.5 - (C @ n.T).T, 0, 1)         # linear fill field, gas side along +n
    k = np.zeros(256)
    theta = mlp.init(2)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = mlp.loss_and_grad(theta, X, n, k, 0.1)[0]
    for t in range(1, 301):
        L, g = mlp.loss_and_grad(theta, X, n, k, 0.1)
        theta, m, v = mlp.adam(theta, g, m, v, t, lr=3e-3)
    assert L < 0.1 * L0


def test_gradient_with_norm_penalty_matches_central_differences():
    rng = np.random.default_rng(7)
    theta = mlp.init(4)
    theta[64 * 27:64 * 27 + 64] = rng.uniform(0.05, 0.2, 64)
    X, n, k = _batch(rng, 12)
    L, g = mlp.loss_and_grad(theta, X, n, k, lam=0.4, mu=0.1)
    h = 1e-6
    for i in rng.choice(mlp.NPARAM, 200, replace=False):
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        num = (mlp.loss_and_grad(tp, X, n, k, 0.4, 0.1)[0] - mlp.loss_and_grad(tm, X, n, k, 0.4, 0.1)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, num, g[i])


def test_bf16_rounding_is_nearest_even():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2)
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -3.0, 0.0, 1e-3])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -3.0, 0.0, 0.00099945068359375])
    assert np.array_equal(mlp.round_bf16(vals), want)


def test_augmented_training_lowers_the_loss():
    from oracle import stencils
    from paper_2301_10674_gb300.workloads import surface_stencils
    fills, labs = stencils.make(surface_stencils(64, seed=12, kinds=[0]))
    theta = mlp.init(5)
    theta, losses = mlp.train(theta, fills, labs, steps=60, batch=32, lr=3e-3, lam=0.4, mu=0.1, seed=3)
    assert losses[-10:].mean() < 0.5 * losses[:5].mean()
