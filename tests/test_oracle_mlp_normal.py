"""Pins of the oracle's learned-normal model inside the step: a network
built by hand computes a known function, so every cell's result follows
from the rules alone.

The network's first layer holds the Parker-Youngs weights (4 face, 2 edge,
1 corner) times +c and -c, so its six ReLU units carry the positive and
negative parts of the fill gradient g; the second layer passes them on; the
third forms s R (-g) for a rotation R and a scale s. The raw normal is then
the finite-difference normal rotated by R with length s |g|, and the oracle
must take it exactly where the block holds no wall or solid cell, where
s |g| lies in [1/2, 2] and where R n_fd is within 30 degrees of n_fd;
everywhere else it must keep n_fd."""
import math

import numpy as np

from oracle import GAS, INTERFACE, LIQUID, SOLID, F_NORMAL, F_PHI, F_TYPE, Oracle, OracleParams
from oracle import mlp

C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], float)
WPY = np.array([{0: 0.0, 1: 4.0, 2: 2.0, 3: 1.0}[int(np.abs(c).sum())] for c in C])


def _network(R, s):
    W1 = np.zeros((64, 27))
    W1[0:3] = (WPY[:, None] * C).T
    W1[3:6] = -(WPY[:, None] * C).T
    W2 = np.zeros((64, 64))
    W2[np.arange(6), np.arange(6)] = 1.0
    W3 = np.zeros((4, 64))
    W3[:3, 0:3] = -s * R
    W3[:3, 3:6] = s * R
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(4)])


def _rot_z(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])


def _state():
    nx, ny, nz = 24, 12, 16
    o = Oracle(OracleParams(nx=nx, ny=ny, nz=nz, omega=1.6, g=(0, 0, -1e-5)))
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    h = 8.0 + 2.5 * np.sin(2 * np.pi * x)[None, :] + 1.5 * np.cos(2 * np.pi * y)[:, None]
    o.init_surface(h)
    return o


def _expected(o, R, s):
    """Per interface cell: (finite-difference normal, gradient length,
    block clear of walls and solids)."""
    t = o.get(F_TYPE)
    phi = o.get(F_PHI)
    nz, ny, nx = t.shape
    out = {}
    for z, yy, xx in zip(*np.nonzero(t == INTERFACE)):
        g = np.zeros(3)
        clear = True
        for q in range(27):
            c = C[q].astype(int)
            X, Y, Z = (xx + c[0]) % nx, yy + c[1], z + c[2]
            if not (0 <= Y < ny and 0 <= Z < nz) or t[Z, Y, X] == SOLID:
                clear = False
                v = phi[z, yy, xx]
            else:
                v = 1.0 if t[Z, Y, X] == LIQUID else (phi[Z, Y, X] if t[Z, Y, X] == INTERFACE else 0.0)
            g += WPY[q] * C[q] * v
        out[(z, yy, xx)] = (g, clear)
    return out


def test_huge_scale_always_falls_back():
    o = _state()
    n_fd = o.get(F_NORMAL)
    o.set_mlp(_network(_rot_z(10.0), 1e7), bf16=False)
    assert np.array_equal(o.get(F_NORMAL), n_fd)


def test_rotated_gradient_is_taken_within_the_rules():
    o = _state()
    n_fd = o.get(F_NORMAL)
    for deg, s in ((20.0, 0.08), (40.0, 0.08), (20.0, 0.3)):
        R = _rot_z(deg)
        o.set_mlp(_network(R, s), bf16=False)
        n_ml = o.get(F_NORMAL)
        cells = _expected(o, R, s)
        taken = fell_back = 0
        for (z, y, x), (g, clear) in cells.items():
            fd = n_fd[:, z, y, x]
            L = s * np.linalg.norm(g)
            rot = R @ fd
            use = clear and 0.5 <= L <= 2.0 and float(rot @ fd) >= math.cos(math.radians(30.0))
            want = rot if use else fd
            assert np.allclose(n_ml[:, z, y, x], want, atol=1e-12), ((z, y, x), deg, s, use)
            taken += use
            fell_back += not use
        assert fell_back > 0
        if deg < 30.0 and s == 0.08:
            assert taken > 0
        o.set_mlp(None)
        assert np.array_equal(o.get(F_NORMAL), n_fd)


def test_trained_flavour_forward_matches_numpy():
    """With random weights and every rule bypassed in the numpy reference,
    the cells the oracle takes from the network carry the numpy forward's
    normalised output (BF16 operand rounding included)."""
    o = _state()
    rng = np.random.default_rng(3)
    theta = _network(np.eye(3), 0.08) + rng.normal(0, 0.02, mlp.NPARAM)
    theta = mlp.round_bf16(theta)
    o.set_mlp(theta, bf16=True)
    n_ml = o.get(F_NORMAL)
    t = o.get(F_TYPE)
    phi = o.get(F_PHI)
    nz, ny, nx = t.shape
    checked = 0
    n_fd_state = _state().get(F_NORMAL)
    for z, y, x in zip(*np.nonzero(t == INTERFACE)):
        if np.array_equal(n_ml[:, z, y, x], n_fd_state[:, z, y, x]):
            continue
        X = np.zeros(27)
        for q in range(27):
            c = C[q].astype(int)
            tt = t[z + c[2], y + c[1], (x + c[0]) % nx]
            X[q] = 1.0 if tt == LIQUID else (min(max(phi[z + c[2], y + c[1], (x + c[0]) % nx], 0), 1)
                                             if tt == INTERFACE else 0.0)
        n_np, _ = mlp.predict_normal(theta, X[None, :], bf16=True)
        assert np.allclose(n_ml[:, z, y, x], n_np[0], atol=1e-12)
        checked += 1
    assert checked > 20


# ---------------------------------------------------------------- mirror averaging (R-17g)
def test_mirror_average_of_a_rotated_gradient_is_its_symmetric_part():
    """Mirror images M in x and y conjugate the rotation: the average of
    M R M over the four is (R + R^T)/2, which for a rotation about z by a is
    diag(cos a, cos a, 1). The oracle must take s diag(cos a, cos a, 1) n_fd
    normalised, under the same rules as the plain network."""
    o = _state()
    n_fd = o.get(F_NORMAL)
    for deg, s in ((20.0, 0.08), (50.0, 0.08)):
        R = _rot_z(deg)
        S = np.diag([math.cos(math.radians(deg)), math.cos(math.radians(deg)), 1.0])
        o.set_mlp(_network(R, s), bf16=False, mirror=True)
        n_ml = o.get(F_NORMAL)
        taken = 0
        for (z, y, x), (g, clear) in _expected(o, R, s).items():
            fd = n_fd[:, z, y, x]
            raw = -s * (S @ g)
            L = np.linalg.norm(raw)
            m = raw / L
            use = clear and 0.5 <= L <= 2.0 and float(m @ fd) >= math.cos(math.radians(30.0))
            want = m if use else fd
            assert np.allclose(n_ml[:, z, y, x], want, atol=1e-12), ((z, y, x), deg, use)
            taken += use
        assert taken > 0
        o.set_mlp(None)


def _stencil(t, phi, z, y, x):
    nx = t.shape[2]
    X = np.zeros(27)
    for q in range(27):
        c = C[q].astype(int)
        tt = t[z + c[2], y + c[1], (x + c[0]) % nx]
        X[q] = 1.0 if tt == LIQUID else (min(max(phi[z + c[2], y + c[1], (x + c[0]) % nx], 0), 1)
                                         if tt == INTERFACE else 0.0)
    return X


def test_mirror_averaged_forward_matches_numpy():
    """Random weights with BF16 operands: where the oracle takes the
    network, its normal is numpy's mirror-averaged forward, normalised."""
    o = _state()
    rng = np.random.default_rng(7)
    theta = mlp.round_bf16(_network(np.eye(3), 0.08) + rng.normal(0, 0.02, mlp.NPARAM))
    o.set_mlp(theta, bf16=True, mirror=True)
    n_ml = o.get(F_NORMAL)
    t, phi = o.get(F_TYPE), o.get(F_PHI)
    n_fd = _state().get(F_NORMAL)
    checked = 0
    for z, y, x in zip(*np.nonzero(t == INTERFACE)):
        if np.array_equal(n_ml[:, z, y, x], n_fd[:, z, y, x]):
            continue
        yv = mlp.forward_mirror(theta, _stencil(t, phi, z, y, x)[None, :], bf16=True)[0]
        assert np.allclose(n_ml[:, z, y, x], yv[:3] / np.linalg.norm(yv[:3]), atol=1e-12)
        checked += 1
    assert checked > 20


def test_flat_layer_keeps_a_vertical_normal_only_with_mirror_averaging():
    """A flat layer is its own mirror image in x and y, so the averaged
    normal has no horizontal component at all; the plain network of the
    same weights tilts it."""
    nx, ny, nz = 12, 8, 12
    o = Oracle(OracleParams(nx=nx, ny=ny, nz=nz, omega=1.6, g=(0, 0, 0)))
    o.init_surface(np.full((ny, nx), 6.37))
    rng = np.random.default_rng(11)
    theta = mlp.round_bf16(_network(np.eye(3), 0.08) + rng.normal(0, 0.02, mlp.NPARAM))
    ifc = o.get(F_TYPE) == INTERFACE
    assert ifc.sum() == nx * ny
    ifc[:, [0, ny - 1], :] = False   # blocks with a y wall keep the finite-difference normal
    o.set_mlp(theta, bf16=True, mirror=False)
    plain = o.get(F_NORMAL)[:, ifc]
    o.set_mlp(theta, bf16=True, mirror=True)
    avg = o.get(F_NORMAL)[:, ifc]
    assert np.abs(plain[:2]).max() > 1e-3
    assert np.all(avg[:2] == 0.0) and np.all(avg[2] > 0.99)
