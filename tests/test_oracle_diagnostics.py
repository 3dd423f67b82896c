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


# ---------------------------------------------------------------- Section 4
import os  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2.txt")


def _table2():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        lab, h0, hbar, tanpsi, theta = line.split()
        rows[lab] = (float(h0), float(hbar), float(tanpsi), float(theta))
    return rows


def test_shields_number_reproduces_table2():
    """Theta of Table 2 from its own depth and slope columns (density ratio
    2.55), to the printed rounding: E1 from the mean depth h_bar as the text
    says; E4's printed Theta matches the initial depth h0 instead (the mean
    depth gives 0.102), a discrepancy of the paper recorded here as it is."""
    t = _table2()
    h0, hbar, tp, theta = t["E1"]
    assert abs(D.shields(hbar, tp, 2.55, 1.0) - theta) <= 0.0005 + 1e-12
    h0, hbar, tp, theta = t["E4"]
    assert abs(D.shields(h0, tp, 2.55, 1.0) - theta) <= 0.0015
    assert abs(D.shields(hbar, tp, 2.55, 1.0) - theta) > 0.01


def test_einstein_number_hand_value():
    # (2.55 - 1) * 1e-5 * 10^3 = 0.0155, sqrt = 0.12449899...; 1e-3 / that
    assert D.einstein(1e-3, 2.55, 1e-5, 10.0) == pytest.approx(0.00803219329, rel=1e-9)


def test_surface_elevation_and_water_depth_of_a_layered_column():
    nz, ny, nx = 20, 4, 6
    t = np.zeros((nz, ny, nx), np.uint8)
    phi = np.zeros((nz, ny, nx))
    t[:5] = D.SOLID                  # sharp bed, top solid layer 4: h_b = 5.2
    t[5:12] = 1
    t[12] = 2
    phi[12] = 0.25                   # surface at 12.25
    eta = D.surface_elevation(t, phi)
    assert np.allclose(eta, 12.25)
    assert D.mean_water_depth(t, phi) == pytest.approx(12.25 - 5.2, abs=1e-12)


def test_bed_spectrum_of_a_travelling_wave():
    """h = 3 + A sin(2 pi (m x / nx - p t / nt)): the largest value of the
    PSD sits at wavenumber m (lambda = nx dx / m), period nt dt / p, celerity
    +lambda / T and amplitude A; reversed in time it travels the other way;
    Parseval: the PSD sums to the squared deviations."""
    nx, nt, m, p, A, dx, dt = 64, 50, 3, 2, 0.7, 1.0, 10.0
    x = np.arange(nx) * dx
    t = np.arange(nt)[:, None] * dt
    h = 3.0 + A * np.sin(2 * np.pi * (m * x / (nx * dx) - p * t / (nt * dt)))
    psd, (lam, T, c, amp) = D.bed_spectrum(h, dx, dt)
    assert lam == pytest.approx(64 / 3) and T == pytest.approx(250.0)
    assert c == pytest.approx(64 / 3 / 250.0) and amp == pytest.approx(A, rel=1e-12)
    assert psd.sum() == pytest.approx(((h - h.mean()) ** 2).sum(), rel=1e-12)
    _, (lam2, T2, c2, amp2) = D.bed_spectrum(h[::-1], dx, dt)
    assert lam2 == pytest.approx(lam) and T2 == pytest.approx(T) and c2 == pytest.approx(-c)
    # a standing pattern has no period
    hs = A * np.cos(2 * np.pi * 5 * x / nx) + 0 * t
    _, (lam3, T3, c3, _) = D.bed_spectrum(hs)
    assert lam3 == pytest.approx(64 / 5) and np.isinf(T3) and c3 == 0.0
