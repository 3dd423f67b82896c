"""Pins of the oracle's training-data generator for the learned normal:
fill levels of analytic surfaces against closed forms, complements and
brute-force sampling; labels against numerical differentiation of the
surface; the 48 cube symmetries against the group axioms and against the
exact plane fill; the batch sampler against SplitMix64's published outputs."""
import math

import numpy as np
import pytest

from oracle import stencils as S
from paper_2301_10674_gb300.workloads import surface_stencils


def _row(kind, n0, s=0.0, r=0.0, A=0.0, k=0.0, phase=0.0, e1=(1.0, 0.0, 0.0)):
    n0 = np.asarray(n0, float)
    n0 = n0 / np.linalg.norm(n0)
    return np.array([kind, *n0, s, r, A, k, phase, *e1], float)


def _brute(pred, c, sub=96):
    t = (np.arange(sub) + 0.5) / sub - 0.5
    X, Y, Z = np.meshgrid(c[0] + t, c[1] + t, c[2] + t, indexing="ij")
    return float(np.count_nonzero(pred(X, Y, Z))) / sub ** 3


# ---------------------------------------------------------------- planes
def test_axis_aligned_plane_is_the_offset():
    # plane z = s, liquid below: the centre cell holds s + 1/2, the layer
    # above is empty and the layer below full
    for s in (-0.5, -0.3, 0.0, 0.17, 0.5):
        fill, lab = S.stencil(_row(0, (0, 0, 1), s=s))
        for q in range(27):
            cz = S.CELLS[q][2]
            assert fill[q] == (s + 0.5 if cz == 0 else (1.0 if cz < 0 else 0.0))
        assert np.allclose(lab, [0, 0, 1, 0])


def test_plane_through_the_centre_halves_the_block():
    # central symmetry of the block maps liquid onto gas
    rng = np.random.default_rng(1)
    for _ in range(5):
        n = rng.standard_normal(3)
        fill, _ = S.stencil(_row(0, n, s=0.0))
        assert abs(fill.sum() - 13.5) < 1e-12
        assert abs(fill[13] - 0.5) < 1e-12


def test_diagonal_plane_closed_form():
    fill, _ = S.stencil(_row(0, (1, 1, 0), s=0.0))
    # x + y <= 0: cells with cx + cy < 0 full, > 0 empty, = 0 half
    for q in range(27):
        c = S.CELLS[q]
        want = 0.5 if c[0] + c[1] == 0 else (1.0 if c[0] + c[1] < 0 else 0.0)
        assert abs(fill[q] - want) < 1e-12


def test_plane_complement_and_brute_force():
    rng = np.random.default_rng(2)
    for _ in range(3):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        s = rng.uniform(-0.5, 0.5)
        P = s * n
        f1 = np.array([S.plane_fill(n, P, c) for c in S.CELLS])
        f2 = np.array([S.plane_fill(-n, P, c) for c in S.CELLS])
        assert np.allclose(f1 + f2, 1.0, atol=1e-14)
        for q in (13, 4, 22, 0, 26, 10):
            c = S.CELLS[q]
            b = _brute(lambda X, Y, Z: (X - P[0]) * n[0] + (Y - P[1]) * n[1] + (Z - P[2]) * n[2] <= 0, c)
            assert abs(b - f1[q]) < 3e-3, (q, b, f1[q])


def test_plane_with_tiny_components_is_continuous():
    # a normal almost along z: the fill tends to the axis-aligned value
    for eps in (1e-3, 1e-6, 1e-9):
        fill, _ = S.stencil(_row(0, (eps, 2 * eps, 1.0), s=0.2))
        assert abs(fill[13] - 0.7) < 4 * eps + 1e-12


# ---------------------------------------------------------------- spheres
def test_droplet_and_bubble_with_one_centre_are_complements():
    rng = np.random.default_rng(3)
    for _ in range(3):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        r = rng.uniform(2, 30)
        s = rng.uniform(-0.5, 0.5)
        fd, ld = S.stencil(_row(1, n, s=s, r=r))
        fb, lb = S.stencil(_row(2, -n, s=-s, r=r))   # same point P, same centre
        assert np.allclose(fd + fb, 1.0, atol=1e-12)
        assert ld[3] == pytest.approx(1 / r) and lb[3] == pytest.approx(-1 / r)


def test_sphere_rows_match_brute_force():
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    r, s = 2.5, 0.21
    C = s * n - r * n
    fill, _ = S.stencil(_row(1, n, s=s, r=r))
    for q in (13, 12, 14, 22, 4, 16):
        c = S.CELLS[q]
        b = _brute(lambda X, Y, Z: (X - C[0]) ** 2 + (Y - C[1]) ** 2 + (Z - C[2]) ** 2 <= r * r, c)
        assert abs(b - fill[q]) < 3e-3, (q, b, fill[q])


def test_large_droplet_approaches_the_plane():
    n = np.array([0.2, 0.4, 0.9])
    n /= np.linalg.norm(n)
    fs, _ = S.stencil(_row(1, n, s=0.1, r=1e6))
    fp, _ = S.stencil(_row(0, n, s=0.1))
    assert np.max(np.abs(fs - fp)) < 1e-3


# ---------------------------------------------------------------- sine waves
def test_sine_labels_match_numerical_differentiation():
    rng = np.random.default_rng(4)
    p = surface_stencils(40, seed=7, kinds=[3])
    for row in p[:5]:
        n0, s = row[1:4], row[4]
        A, k, ph = row[6:9]
        e1 = row[9:12]
        P = s * n0

        def F(x):   # positive in the gas
            d = x - P
            return d @ n0 - A * (math.sin(k * (d @ e1) + ph) - math.sin(ph))

        def grad(x, h=1e-5):
            return np.array([(F(x + h * e) - F(x - h * e)) / (2 * h) for e in np.eye(3)])

        g = grad(P)
        n_num = g / np.linalg.norm(g)
        h = 1e-3
        div = sum((grad(P + h * e)[i] / np.linalg.norm(grad(P + h * e))
                   - grad(P - h * e)[i] / np.linalg.norm(grad(P - h * e))) / (2 * h)
                  for i, e in enumerate(np.eye(3)))
        lab = S.labels(row)
        assert np.allclose(lab[:3], n_num, atol=1e-8)
        assert abs(lab[3] - 0.5 * div) < 1e-5


def test_flat_sine_is_the_plane():
    n = np.array([0.1, 0.7, -0.3])
    n /= np.linalg.norm(n)
    e1 = np.cross(n, [1.0, 0, 0])
    e1 /= np.linalg.norm(e1)
    fs, ls = S.stencil(_row(3, n, s=0.05, A=1e-9, k=0.1, phase=1.0, e1=e1))
    fp, lp = S.stencil(_row(0, n, s=0.05))
    assert np.max(np.abs(fs - fp)) < 4e-3
    assert np.allclose(ls, lp, atol=1e-9)


def test_sine_samples_match_a_finer_grid():
    row = surface_stencils(20, seed=9, kinds=[3])[0]
    n0, s = row[1:4], row[4]
    A, k, ph = row[6:9]
    e1 = row[9:12]
    P = s * n0
    for q in (13, 4, 22):
        c = S.CELLS[q]
        a = S.sine_fill(P, n0, e1, A, k, ph, c)
        b = S.sine_fill(P, n0, e1, A, k, ph, c, sub=100)
        assert abs(a - b) < 3e-3


# ---------------------------------------------------------------- symmetries
def test_symmetries_form_the_cube_group():
    mats = [S.symmetry(k) for k in range(48)]
    keys = {m.tobytes() for m in mats}
    assert len(keys) == 48
    assert np.array_equal(mats[0], np.eye(3, dtype=np.int64))
    for a in mats[::5]:
        assert abs(round(np.linalg.det(a))) == 1
        for b in mats[::7]:
            assert (a @ b).tobytes() in keys


def test_symmetry_maps_plane_stencils_exactly():
    rng = np.random.default_rng(5)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    fill, lab = S.stencil(_row(0, n, s=0.13))
    for k in range(48):
        T = S.symmetry(k)
        f2, l2 = S.apply_symmetry(fill, lab, k)
        direct, ld = S.stencil(_row(0, T @ n, s=0.13))
        assert np.allclose(f2, direct, atol=1e-12), k
        assert np.allclose(l2, ld, atol=1e-12)


# ---------------------------------------------------------------- sampler
def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 0
    assert S.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert S.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert S.splitmix64(0, 2) == 0x06C45D188009454F


def test_draw_covers_indices_and_symmetries():
    idx, sym = S.draw(11, 3, 4096, 1000)
    assert idx.min() >= 0 and idx.max() < 1000 and len(np.unique(idx)) > 950
    assert sym.min() >= 0 and sym.max() == 47
    idx2, sym2 = S.draw(11, 3, 4096, 1000, augment=False)
    assert np.array_equal(idx, idx2) and not sym2.any()


# ---------------------------------------------------------------- height function
def _block(fillfun):
    """7 x 7 x 7 block of fill levels fillfun(c) and their types."""
    f = np.zeros((7, 7, 7))
    for k in range(7):
        for j in range(7):
            for i in range(7):
                f[k, j, i] = fillfun((i - 3, j - 3, k - 3))
    t = np.where(f >= 1.0, S.LIQ, np.where(f <= 0.0, S.GAS, S.IFC))
    return f, t


@pytest.mark.parametrize("n0,s", [((0.1, -0.2, 1.0), 0.2), ((-1.0, 0.3, 0.25), -0.1), ((0.4, 1.0, -0.35), 0.4),
                                  ((0.0, 0.0, -1.0), 0.0)])
def test_height_function_is_exact_on_planes(n0, s):
    """A column's fill levels integrate the plane's height over its cross
    section, whose mean is the height at the column's centre: the heights are
    exact, so the normal is n0 and the curvature 0 to rounding."""
    n0 = np.asarray(n0) / np.linalg.norm(n0)
    P = s * n0
    f, t = _block(lambda c: S.plane_fill(n0, P, c))
    out = S.height_function_label(f, t)
    assert out is not None
    fill27, lab, fd = out
    assert np.allclose(lab[:3], n0, atol=1e-12, rtol=0), (lab, n0)
    assert abs(lab[3]) < 1e-12
    # the input is the 3x3x3 block of clamped fill levels, stencil order
    for q in range(27):
        c = S.CELLS[q]
        assert fill27[q] == f[c[2] + 3, c[1] + 3, c[0] + 3]
    assert np.dot(fd, n0) > 0.99


def _sphere_fill_fine(C, r, c, inside, sub=512):
    """Fraction of cell c inside (or outside) the sphere from the exact
    x-chords of sub x sub rows (finer than the training data's 64 x 64, so
    that the reference fills resolve a large sphere's curvature)."""
    t = (np.arange(sub) + 0.5) / sub - 0.5
    Y, Z = np.meshgrid(t, t, indexing="ij")
    dy = c[1] + Y.ravel() - C[1]
    dz = c[2] + Z.ravel() - C[2]
    h2 = r * r - dy * dy - dz * dz
    h = np.sqrt(np.maximum(h2, 0.0))
    lo = np.maximum(C[0] - h, c[0] - 0.5)
    hi = np.minimum(C[0] + h, c[0] + 0.5)
    frac = float(np.where(h2 > 0.0, np.maximum(hi - lo, 0.0), 0.0).sum()) / (sub * sub)
    return frac if inside else 1.0 - frac


@pytest.mark.parametrize("R,inside,tol", [(8.0, True, 0.015), (16.0, True, 0.005), (12.0, False, 0.01)])
def test_height_function_on_spheres(R, inside, tol):
    """A droplet (liquid inside) and a bubble (liquid outside) of radius R
    above or below the cell: the mean curvature is +1/R and -1/R within the
    method's second-order error (0.7% at R = 8, 0.2% at R = 16), the normal
    within half a degree of the sphere's normal at the surface point above
    the cell centre."""
    off = np.array([0.3, -0.2, 0.1])
    C = np.array([off[0], off[1], (off[2] - R) if inside else (off[2] + R)])
    f, t = _block(lambda c: _sphere_fill_fine(C, R, c, inside))
    out = S.height_function_label(f, t)
    assert out is not None
    _, lab, _ = out
    zs = C[2] + (1 if inside else -1) * math.sqrt(R * R - C[0] ** 2 - C[1] ** 2)
    nx = (np.array([0.0, 0.0, zs]) - C) / R
    n_true = nx if inside else -nx
    ang = math.degrees(math.acos(min(1.0, float(np.dot(lab[:3], n_true)))))
    assert ang < 0.5, ang
    k_true = (1.0 if inside else -1.0) / R
    assert abs(lab[3] - k_true) < tol * abs(k_true), (lab[3], k_true)


def test_height_function_rejects_incomplete_blocks():
    # a droplet of radius 2: the columns beside it have no liquid end
    f, t = _block(lambda c: S.sphere_fill((0.0, 0.0, -1.8), 2.0, c, inside=True))
    assert S.height_function_label(f, t) is None
    # a plane with a solid cell, and with a wall, in the 3x3x3 block
    n0 = np.array([0.0, 0.0, 1.0])
    f, t = _block(lambda c: S.plane_fill(n0, 0.1 * n0, c))
    assert S.height_function_label(f, t) is not None
    t2 = t.copy()
    t2[3, 3, 4] = S.SOL
    assert S.height_function_label(f, t2) is None
    t3 = t.copy()
    t3[2, :, :] = S.WALL
    assert S.height_function_label(f, t3) is None
    # a solid cell in a column (outside the 3x3x3 block) drops the label too
    t4 = t.copy()
    t4[0, 3, 3] = S.SOL
    assert S.height_function_label(f, t4) is None


def test_height_function_block_from_fields_wraps_periodic_axes():
    """block7 reads the fields around a cell with the periodic x wrap and
    walls beyond non-periodic faces."""
    nz, ny, nx = 8, 5, 6
    types = np.full((nz, ny, nx), S.GAS)
    types[:4] = S.LIQ
    phi = np.zeros((nz, ny, nx))
    phi[:4] = 1.0
    cell = 4 * nx * ny + 2 * nx + 0          # x = 0, y = 2, z = 4
    f, t = S.block7(phi, types, cell, (1, 0, 0))
    assert t[3, 3, 0] == types[4, 2, nx - 3]  # x = -3 wraps to nx - 3
    assert (t[:, 0, :] == S.WALL).all()       # y = -1 lies beyond the wall
    assert f[2, 3, 3] == 1.0 and f[3, 3, 3] == 0.0
