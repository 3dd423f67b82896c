"""FP64 oracle of the learned interface normal: a 27-64-64-4 perceptron
with ReLU that maps a 3x3x3 fill-level stencil to the interface normal
(3 components, pointing toward the gas) and the curvature.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline). Plain numpy,
written from the definition: affine layers, ReLU, the loss
L = mean over the batch of
    (1 - n_pred.n_true / |n_pred|) + lam (k_pred - k_true)^2 + mu (|n_pred| - 1)^2,
its gradient by the chain rule, and the Adam update (Kingma and Ba, with
bias correction). The last term keeps the raw normal near unit length, so
that a raw length far from 1 can mark an input the network does not know
(the inference falls back to the finite-difference normal there); mu = 0
gives the plain angular loss. The tests pin the gradient against central
finite differences.

Parameter layout (shared convention with the CUDA kernels, which store the
same matrices): W1 (64, 27), b1 (64), W2 (64, 64), b2 (64), W3 (4, 64), b3 (4).
"""
from __future__ import annotations

import numpy as np

SIZES = ((64, 27), (64,), (64, 64), (64,), (4, 64), (4,))
NPARAM = sum(int(np.prod(s)) for s in SIZES)   # 6212


def unpack(theta: np.ndarray):
    out, k = [], 0
    for s in SIZES:
        m = int(np.prod(s))
        out.append(theta[k:k + m].reshape(s))
        k += m
    return out


def init(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SIZES:
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def round_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 value (8 significant bits, ties to
    even), returned as float64."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                      # a = m 2^e, |m| in [1/2, 1)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def forward(theta: np.ndarray, X: np.ndarray, bf16: bool = False):
    """X: (B, 27) fill levels. Returns the output (B, 4) and the cache.
    With bf16, the operands of each product (weights, inputs and hidden
    activations) are rounded to bfloat16 first, as on the tensor cores;
    sums stay exact in FP64."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    r = round_bf16 if bf16 else (lambda a: a)
    z1 = r(X) @ r(W1).T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = r(h1) @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    y = r(h2) @ r(W3).T + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, n_true: np.ndarray, k_true: np.ndarray, lam: float,
                  mu: float = 0.0):
    """Loss and its gradient with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    n = y[:, :3]
    kap = y[:, 3]
    norm = np.linalg.norm(n, axis=1)
    cosv = np.sum(n * n_true, axis=1) / norm
    L = np.mean(1.0 - cosv + lam * (kap - k_true) ** 2 + mu * (norm - 1.0) ** 2)
    # d(1 - n.t/|n|)/dn = -(t/|n| - (n.t) n/|n|^3); d(|n| - 1)^2/dn = 2 (|n| - 1) n/|n|
    dn = -(n_true / norm[:, None] - (np.sum(n * n_true, axis=1) / norm ** 3)[:, None] * n) / B
    dn += (2.0 * mu * (norm - 1.0) / norm)[:, None] * n / B
    dk = 2.0 * lam * (kap - k_true) / B
    dy = np.concatenate([dn, dk[:, None]], axis=1)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new theta, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def mirror_index(m: int) -> np.ndarray:
    """Stencil indices under the mirror images of R-17g: index q of the
    mirrored stencil holds the value at mirror_index(m)[q] of the original
    (bit 0 of m reverses x, bit 1 reverses y)."""
    q = np.arange(27)
    a, b, c = q % 3, (q // 3) % 3, q // 9
    if m & 1:
        a = 2 - a
    if m & 2:
        b = 2 - b
    return a + 3 * b + 9 * c


def forward_mirror(theta: np.ndarray, X: np.ndarray, bf16: bool = False) -> np.ndarray:
    """The network averaged over the mirror images in x and y (R-17g): the
    output for each mirrored stencil, its mirrored components negated back,
    summed in the order identity, x, y, both, times 1/4."""
    y = forward(theta, X, bf16)[0].copy()
    for m in (1, 2, 3):
        ym = forward(theta, X[:, mirror_index(m)], bf16)[0]
        y[:, 0] += -ym[:, 0] if m & 1 else ym[:, 0]
        y[:, 1] += -ym[:, 1] if m & 2 else ym[:, 1]
        y[:, 2:] += ym[:, 2:]
    return 0.25 * y


def predict_normal(theta, X, bf16: bool = False):
    """Unit normal (toward the gas) and curvature predicted for stencils X."""
    y, _ = forward(theta, X, bf16)
    n = y[:, :3]
    return n / np.linalg.norm(n, axis=1, keepdims=True), y[:, 3]


def train(theta, fills, targets, steps, batch, lr, lam, mu, seed, augment=True):
    """Adam on batches drawn by the counter-based sampler, each stencil
    mapped by its drawn cube symmetry. Returns the parameters and the loss of
    every step (before that step's update)."""
    from oracle import stencils
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t in range(steps):
        idx, sym = stencils.draw(seed, t, batch, len(fills), augment)
        X = np.zeros((batch, 27))
        Y = np.zeros((batch, 4))
        for j in range(batch):
            X[j], Y[j] = stencils.apply_symmetry(fills[idx[j]], targets[idx[j]], int(sym[j]))
        L, g = loss_and_grad(theta, X, Y[:, :3], Y[:, 3], lam, mu)
        losses.append(L)
        theta, m, v = adam(theta, g, m, v, t + 1, lr)
    return theta, np.array(losses)
