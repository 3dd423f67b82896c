"""Oracle of the learned normal's training data: 3x3x3 fill stencils of
analytic surfaces, with the exact normal and curvature at the surface point,
the 48 symmetries of the cube used for augmentation, and the counter-based
sampler that picks training batches.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline). Plain numpy and
exact rational arithmetic, written from the definitions:

* Cell q has offset c = (q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1) and covers
  the cube [c - 1/2, c + 1/2]^3; its fill level is the liquid volume fraction
  of that cube.
* Plane: the exact volume of {xi in [0,1]^d : m.xi <= alpha} by
  inclusion-exclusion over the cube's corners,
  V = sum_v (-1)^|v| max(0, alpha - m.v)^d / (d! prod m), evaluated in
  rational arithmetic on the FP64 parameters, so it carries no rounding.
* Liquid / gas sphere: 64 x 64 rows along x through the sample points
  ((j + 1/2)/64 - 1/2) in y and z; each row contributes the exact length of
  its chord inside the sphere (or outside it, for the gas sphere).
* Sine wave w <= A (sin(k u + phase) - sin(phase)), with w = (x - P).n0 and
  u = (x - P).e1: 64^3 midpoint samples per cell.
* Labels at P: the unit normal toward the gas and the mean curvature,
  positive for a convex liquid body (1/r for a droplet).

Parameters come from the shared seeded generator (one row per surface; see
``surface_stencils`` in the workloads module for the row layout).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

CELLS = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], dtype=np.int64)
SUB = 64                                         # sub-samples per cell edge


def qindex(c) -> int:
    return int((c[0] + 1) + 3 * (c[1] + 1) + 9 * (c[2] + 1))


# ---------------------------------------------------------------- planes
def _box_volume_below(m, alpha) -> Fraction:
    """Exact volume of {xi in [0,1]^d : m.xi <= alpha}, m_i > 0 (Fractions)."""
    d = len(m)
    if d == 0:
        return Fraction(1) if alpha >= 0 else Fraction(0)
    total = Fraction(0)
    for v in itertools.product((0, 1), repeat=d):
        t = alpha - sum(mi for mi, vi in zip(m, v) if vi)
        if t > 0:
            total += (-1) ** sum(v) * t ** d
    den = Fraction(math.factorial(d))
    for mi in m:
        den *= mi
    return total / den


def plane_fill(n0, P, c) -> float:
    """Liquid fraction of cell c below the plane (x - P).n0 <= 0."""
    n = [Fraction(float(a)) for a in n0]
    p = [Fraction(float(a)) for a in P]
    # x = c - 1/2 + xi: n.xi <= n.P - n.(c - 1/2)
    beta = sum(ni * (pi - (ci - Fraction(1, 2))) for ni, pi, ci in zip(n, p, c))
    # reflect the negative components: xi_i -> 1 - xi_i
    alpha = beta - sum(ni for ni in n if ni < 0)
    m = [abs(ni) for ni in n if ni != 0]
    return float(_box_volume_below(m, alpha))


# ---------------------------------------------------------------- spheres
def _row_points():
    t = (np.arange(SUB) + 0.5) / SUB - 0.5
    Y, Z = np.meshgrid(t, t, indexing="ij")
    return Y.ravel(), Z.ravel()


def sphere_fill(C, r, c, inside: bool) -> float:
    """Fraction of cell c inside (or outside) the sphere |x - C| <= r, from
    the exact x-chords of 64 x 64 rows."""
    y, z = _row_points()
    dy = c[1] + y - C[1]
    dz = c[2] + z - C[2]
    h2 = r * r - dy * dy - dz * dz
    h = np.sqrt(np.maximum(h2, 0.0))
    lo = np.maximum(C[0] - h, c[0] - 0.5)
    hi = np.minimum(C[0] + h, c[0] + 0.5)
    length = np.where(h2 > 0.0, np.maximum(hi - lo, 0.0), 0.0)
    frac = float(np.sum(length)) / (SUB * SUB)
    return frac if inside else 1.0 - frac


# ---------------------------------------------------------------- sine waves
def sine_fill(P, n0, e1, A, k, phase, c, sub: int = SUB) -> float:
    """Fraction of cell c below the sine surface, from sub^3 midpoints."""
    t = (np.arange(sub) + 0.5) / sub - 0.5
    X, Y, Z = np.meshgrid(c[0] + t, c[1] + t, c[2] + t, indexing="ij")
    d = np.stack([X - P[0], Y - P[1], Z - P[2]], axis=-1)
    u = d @ np.asarray(e1)
    w = d @ np.asarray(n0)
    liq = w <= A * (np.sin(k * u + phase) - math.sin(phase))
    return float(np.count_nonzero(liq)) / sub ** 3


# ---------------------------------------------------------------- one surface
def stencil(row) -> tuple[np.ndarray, np.ndarray]:
    """Fill levels (27) and labels (n_x, n_y, n_z, kappa) of one surface."""
    kind = int(row[0])
    n0 = np.asarray(row[1:4], dtype=float)
    s = float(row[4])
    r, A, k, phase = (float(v) for v in row[5:9])
    e1 = np.asarray(row[9:12], dtype=float)
    P = s * n0
    fill = np.zeros(27)
    for q in range(27):
        c = CELLS[q]
        if kind == 0:
            fill[q] = plane_fill(n0, P, c)
        elif kind == 1:
            fill[q] = sphere_fill(P - r * n0, r, c, inside=True)
        elif kind == 2:
            fill[q] = sphere_fill(P + r * n0, r, c, inside=False)
        else:
            fill[q] = sine_fill(P, n0, e1, A, k, phase, c)
    return fill, labels(row)


def labels(row) -> np.ndarray:
    """Unit normal toward the gas and mean curvature at P (positive for a
    convex liquid body)."""
    kind = int(row[0])
    n0 = np.asarray(row[1:4], dtype=float)
    r, A, k, phase = (float(v) for v in row[5:9])
    e1 = np.asarray(row[9:12], dtype=float)
    if kind == 0:
        return np.array([*n0, 0.0])
    if kind == 1:
        return np.array([*n0, 1.0 / r])
    if kind == 2:
        return np.array([*n0, -1.0 / r])
    # graph w = f(u), f(u) = A (sin(k u + phase) - sin(phase)); liquid below.
    # normal toward the gas: (n0 - f' e1) / sqrt(1 + f'^2); the surface is
    # a cylinder, whose mean curvature is half the profile's curvature
    fp = A * k * math.cos(phase)
    fpp = -A * k * k * math.sin(phase)
    q = math.sqrt(1.0 + fp * fp)
    n = (n0 - fp * e1) / q
    return np.array([*n, -fpp / (2.0 * q ** 3)])


def make(params: np.ndarray):
    """Fill levels (n, 27) and labels (n, 4) of a block of surface rows."""
    fills = np.zeros((len(params), 27))
    labs = np.zeros((len(params), 4))
    for i, row in enumerate(params):
        fills[i], labs[i] = stencil(row)
    return fills, labs


# ---------------------------------------------------------------- cube symmetries
PERMS = list(itertools.permutations(range(3)))   # lexicographic order


def symmetry(k: int) -> np.ndarray:
    """Matrix T of symmetry k in [0, 48): (T v)_i = s_i v_perm(i), with
    perm = PERMS[k // 8] and s_i = -1 where bit i of k % 8 is set."""
    perm = PERMS[k // 8]
    T = np.zeros((3, 3), dtype=np.int64)
    for i in range(3):
        T[i, perm[i]] = -1 if (k % 8) >> i & 1 else 1
    return T


def apply_symmetry(fill27, target4, k: int):
    """Stencil and labels of the surface mapped by symmetry k: the cell at
    offset T c receives the fill of the cell at c; the normal becomes T n;
    the curvature is unchanged."""
    T = symmetry(k)
    out = np.zeros(27)
    for q in range(27):
        out[qindex(T @ CELLS[q])] = fill27[q]
    t = np.asarray(target4, dtype=float)
    return out, np.array([*(T @ t[:3]), t[3]])


# ---------------------------------------------------------------- batch sampler
GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, counter: int) -> int:
    """Output number ``counter`` (from 0) of the SplitMix64 generator seeded
    with ``seed`` (Steele, Lea and Flood 2014, with Vigna's mixing
    constants): the state advances by the golden-ratio increment and each
    state is passed through the 64-bit finaliser."""
    z = (seed + (counter + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw(seed: int, step: int, batch: int, n: int, augment: bool = True):
    """Stencil indices and symmetries of one training batch: slot j of step
    t uses output t * batch + j; index = value mod n, symmetry =
    (value >> 32) mod 48 (identity without augmentation)."""
    idx = np.zeros(batch, dtype=np.int64)
    sym = np.zeros(batch, dtype=np.int64)
    for j in range(batch):
        v = splitmix64(seed, step * batch + j)
        idx[j] = v % n
        sym[j] = (v >> 32) % 48 if augment else 0
    return idx, sym


# ---------------------------------------------------------------- height function
# Labels of interface stencils taken from a run's own state (the logged
# stencils of the learned normal). The height-function method: along the
# axis a of the largest component of the Parker-Youngs normal (gas toward the
# sign sg of that component), the fill levels of the 3 x 3 columns of seven
# cells centred on the cell's row, summed, give the surface's height above
# each column's centre plane, eta = sum - 7/2, measured toward the gas; the
# normal toward the gas and the mean curvature follow from the central
# differences of eta (the surface is t = eta(u, v), liquid below).
LIQ, IFC, GAS, SOL, WALL = 1, 2, 0, 3, -1


def block7(phi, types, cell, periodic):
    """Fill levels (raw phi for interface cells, liquid 1, gas 0) and types
    of the 7 x 7 x 7 block around `cell` of (nz, ny, nx) fields, indexed
    [dz + 3, dy + 3, dx + 3]; cells beyond a wall face get type WALL."""
    nz, ny, nx = types.shape
    z, rem = divmod(int(cell), nx * ny)
    y, x = divmod(rem, nx)
    f = np.zeros((7, 7, 7))
    t = np.full((7, 7, 7), WALL, dtype=np.int64)
    for k in range(7):
        for j in range(7):
            for i in range(7):
                c = [x + i - 3, y + j - 3, z + k - 3]
                ok = True
                for a, L in enumerate((nx, ny, nz)):
                    if c[a] < 0 or c[a] >= L:
                        if periodic[a]:
                            c[a] %= L
                        else:
                            ok = False
                if ok:
                    ty = int(types[c[2], c[1], c[0]])
                    t[k, j, i] = ty
                    f[k, j, i] = 1.0 if ty == LIQ else (float(phi[c[2], c[1], c[0]]) if ty == IFC else 0.0)
    return f, t


def parker_youngs32(f27):
    """The Parker-Youngs gradient of a 27-stencil of raw fill levels in FP32,
    summed in stencil order (the precision and order in which the logging
    kernel forms it; every product is exact, weight and offset being small
    powers of two), and the normal -g/|g|; None for a zero gradient."""
    g = np.zeros(3, dtype=np.float32)
    for q in range(27):
        if q == 13:
            continue
        c = CELLS[q]
        w = np.float32({1: 4.0, 2: 2.0, 3: 1.0}[int(np.abs(c).sum())])
        for a in range(3):
            g[a] = np.float32(g[a] + np.float32(w * np.float32(c[a])) * np.float32(f27[q]))
    L = math.sqrt(float(g[0]) ** 2 + float(g[1]) ** 2 + float(g[2]) ** 2)
    if not L > 0:
        return None
    return g, -g.astype(np.float64) / L


def height_function_label(f7, t7):
    """(input27, label4, fd3) of the centre cell of a 7 x 7 x 7 block, or
    None where the stencil is not logged (a wall or solid cell in the 3x3x3
    block, or a column without a liquid end on the liquid side and a gas end
    on the gas side). input27: fill levels clamped to [0, 1]; label4: normal
    toward the gas and mean curvature (positive for a convex liquid body),
    FP64; fd3: the Parker-Youngs normal."""
    inner_t = t7[2:5, 2:5, 2:5]
    if np.any((inner_t == WALL) | (inner_t == SOL)):
        return None
    f27 = np.array([f7[c[2] + 3, c[1] + 3, c[0] + 3] for c in CELLS])
    py = parker_youngs32(f27)
    if py is None:
        return None
    g, n = py
    ag = np.abs(g)
    a = 0 if (ag[0] >= ag[1] and ag[0] >= ag[2]) else (1 if ag[1] >= ag[2] else 2)
    u, v = [b for b in range(3) if b != a]
    sg = 1 if g[a] < 0 else -1
    eta = np.zeros((3, 3))
    for iu in (-1, 0, 1):
        for iv in (-1, 0, 1):
            total = 0.0
            for tt in range(-3, 4):
                d = [0, 0, 0]
                d[u], d[v], d[a] = iu, iv, sg * tt
                ty = t7[d[2] + 3, d[1] + 3, d[0] + 3]
                if ty in (WALL, SOL):
                    return None
                if (tt == -3 and ty != LIQ) or (tt == 3 and ty != GAS):
                    return None
                total += min(max(f7[d[2] + 3, d[1] + 3, d[0] + 3], 0.0), 1.0)
            eta[iu + 1, iv + 1] = total - 3.5
    eu = 0.5 * (eta[2, 1] - eta[0, 1])
    ev = 0.5 * (eta[1, 2] - eta[1, 0])
    euu = eta[2, 1] - 2.0 * eta[1, 1] + eta[0, 1]
    evv = eta[1, 2] - 2.0 * eta[1, 1] + eta[1, 0]
    euv = 0.25 * (eta[2, 2] - eta[2, 0] - eta[0, 2] + eta[0, 0])
    g2 = 1.0 + eu * eu + ev * ev
    m = np.zeros(3)
    m[a] = sg / math.sqrt(g2)
    m[u] = -eu / math.sqrt(g2)
    m[v] = -ev / math.sqrt(g2)
    kappa = -(euu * (1.0 + ev * ev) + evv * (1.0 + eu * eu) - 2.0 * eu * ev * euv) / (2.0 * g2 ** 1.5)
    return np.clip(f27, 0.0, 1.0), np.array([m[0], m[1], m[2], kappa]), n
