"""Pins of the bed-height oracle (Section 3.2): closed forms of sharp and
partly filled beds, a monotone column against numpy's own interpolation,
and the limits of the lattice (empty and full columns)."""
import numpy as np
import pytest

from oracle import diagnostics as D

NX, NY, NZ = 12, 8, 20


def _types(heights, ny=NY, nz=NZ, fill_y=None):
    """Solid (3) below heights[x] in every column, liquid (1) above; with
    fill_y only the first fill_y rows of y are solid."""
    t = np.ones((nz, ny, len(heights)), np.uint8)
    for x, H in enumerate(heights):
        rows = slice(0, ny if fill_y is None else fill_y)
        t[:H, rows, x] = D.SOLID
    return t


def test_sharp_bed_closed_form():
    # top solid layer H - 1: phi = 1 at z = H - 1/2 and 0 at z = H + 1/2,
    # so the 0.3 crossing lies 0.7 above the last solid centre
    H = [3, 5, 5, 6, 9, 1, 2, 7, 7, 7, 4, 10]
    h = D.bed_height(_types(H))
    assert np.allclose(h, np.array(H) + 0.2, atol=1e-14)


def test_other_threshold():
    H = [4] * NX
    assert np.allclose(D.bed_height(_types(H), 0.5), 4.0, atol=1e-14)
    assert np.allclose(D.bed_height(_types(H), 1.0), 3.5, atol=1e-14)


def test_partly_filled_rows():
    # half of y solid below H: phi = 1/2 >= 0.3 up to H - 1, then 0
    H = [6] * NX
    h = D.bed_height(_types(H, fill_y=NY // 2))
    assert np.allclose(h, 6 - 0.5 + (0.5 - 0.3) / 0.5, atol=1e-14)
    # a quarter of y: phi = 1/4 never reaches 0.3; the crossing lies
    # between the wall (phi = 1 at z = -1/2) and cell 0 (phi = 1/4)
    h = D.bed_height(_types(H, fill_y=NY // 4))
    assert np.allclose(h, -0.5 + (1.0 - 0.3) / (1.0 - 0.25), atol=1e-14)


def test_monotone_column_matches_numpy_interpolation():
    # strictly falling solid counts (ny = 64 > nz): phi_b has one crossing,
    # which numpy's interpolation finds from the other side
    ny = 64
    rng = np.random.default_rng(3)
    t = np.ones((NZ, ny, NX), np.uint8)
    for x in range(NX):
        counts = np.sort(rng.choice(np.arange(1, ny), NZ - 1, replace=False))[::-1]
        counts = np.concatenate([[ny], counts])
        for z, c in enumerate(counts):
            t[z, :c, x] = D.SOLID
    h = D.bed_height(t)
    phi = D.solid_fraction(t)
    for x in range(NX):
        zz = np.concatenate([np.arange(NZ) + 0.5, [NZ + 0.5]])[::-1]    # from the top
        pp = np.concatenate([phi[:, x], [0.0]])[::-1]                  # increasing
        assert h[x] == pytest.approx(np.interp(0.3, pp, zz), abs=1e-12), x


def test_empty_and_full_columns():
    t = np.ones((NZ, NY, 3), np.uint8)
    t[:, :, 1] = D.SOLID
    h = D.bed_height(t)
    assert h[0] == pytest.approx(0.2, abs=1e-14)          # no bed: wall crossing
    assert h[1] == pytest.approx(NZ + 0.2, abs=1e-14)     # solid to the top
    assert h[2] == pytest.approx(0.2, abs=1e-14)


def test_topmost_crossing_is_taken():
    # a solid slab floating above a gap: the crossing above the slab counts
    t = np.ones((NZ, NY, 1), np.uint8)
    t[:3, :, 0] = D.SOLID
    t[10:13, :, 0] = D.SOLID
    assert D.bed_height(t)[0] == pytest.approx(13.2, abs=1e-14)
