"""Oracle of the bed-topography evaluation quantity of Section 3.2 (after
Kidanemariam and Uhlmann): the y-averaged solid-volume fraction
phi_b(x, z) of every cell of the x-z plane, and the bed height h_b(x), the
linearly interpolated z at which phi_b(x, z) = 0.3.

TEST INFRASTRUCTURE ONLY (tests, smoke check). Plain numpy, written from the
definition:

* A cell is solid (fraction 1) when a particle's map covers it, else 0, so
  phi_b(x, z) is the number of solid cells of the column (x, ., z) over ny.
* The value of cell k is placed at its centre z = k + 1/2.
* h_b(x) is the topmost crossing of the threshold: with k the highest cell
  whose phi_b reaches the threshold, h_b lies between the centres of k and
  k + 1, h_b = (k + 1/2) + (phi_k - phi_b) / (phi_k - phi_{k+1}).
* Above the lattice phi_b is 0. Below it the bottom wall counts as solid
  (phi_b = 1 at z = -1/2), so a column with no cell at the threshold has its
  crossing between the wall and cell 0.

These three rules are readings of a definition the paper states in one
sentence; a sharp bed whose top solid layer is H - 1 gives h_b = H - 1/2 +
(1 - phi_b), that is H + 0.2 at phi_b = 0.3.
"""
from __future__ import annotations

import numpy as np

SOLID = 3


def solid_fraction(types: np.ndarray) -> np.ndarray:
    """phi_b(x, z) as an (nz, nx) array from cell types of shape (nz, ny, nx)."""
    t = np.asarray(types)
    return (t == SOLID).sum(axis=1) / float(t.shape[1])


def bed_height(types: np.ndarray, phi_b: float = 0.3) -> np.ndarray:
    """h_b(x) for every x, from cell types of shape (nz, ny, nx)."""
    phi = solid_fraction(types)
    nz, nx = phi.shape
    h = np.zeros(nx)
    for x in range(nx):
        col = phi[:, x]
        above = np.nonzero(col >= phi_b)[0]
        if len(above) == 0:
            k, pk, pn = -1, 1.0, col[0]          # the wall below, then cell 0
        else:
            k = int(above.max())
            pk = col[k]
            pn = col[k + 1] if k + 1 < nz else 0.0
        h[x] = (k + 0.5) + (pk - phi_b) / (pk - pn)
    return h


# ---------------------------------------------------------------- Section 4
# Evaluation quantities of the results (Sections 4.1 and 4.2), written from
# their definitions. Readings (the paper names each quantity in a sentence):
#
# * Free-surface elevation of a column (x, y): its liquid and solid volume,
#   sum over z of 1 (liquid, solid), phi (interface), 0 (gas); the mean water
#   depth h_bar is its y-average above the bed height h_b(x), averaged over x.
# * Power spectral density of h_b(x, t): the squared modulus of the
#   two-dimensional discrete Fourier transform over x and t of the series with
#   its mean removed, divided by the number of samples nx * nt. The dominant
#   bedform is the largest value at a positive wavenumber; for the transform
#   kernel exp(-2 pi i (j x / nx + l t / nt)) a pattern travelling toward +x
#   at positive wavenumber j has a negative frequency index l, so its celerity
#   lambda / T carries the sign of -l.
# * Shields number Theta = R_b tan(psi) / (d50 (rho_p / rho_l - 1)) with the
#   hydraulic radius R_b taken as the mean water depth (periodic spanwise
#   boundaries) and tan(psi) the slope of the imposed body force,
#   g_x / |g_z|.
# * Einstein bedload number q_b* = q_b / ((rho_p / rho_l - 1) g d50^3)^(1/2),
#   g the magnitude of the body acceleration.


def surface_elevation(types: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """(ny, nx) liquid plus solid volume of every column, from cell types and
    fill levels of shape (nz, ny, nx)."""
    t = np.asarray(types)
    vol = np.where((t == 1) | (t == SOLID), 1.0, np.where(t == 2, np.asarray(phi), 0.0))
    return vol.sum(axis=0)


def mean_water_depth(types: np.ndarray, phi: np.ndarray, phi_b: float = 0.3) -> float:
    """h_bar: mean over x of (y-mean surface elevation - h_b(x))."""
    eta = surface_elevation(types, phi).mean(axis=0)
    return float(np.mean(eta - bed_height(types, phi_b)))


def shields(depth: float, tan_psi: float, density_ratio: float, d50: float) -> float:
    return depth * tan_psi / (d50 * (density_ratio - 1.0))


def einstein(q_b: float, density_ratio: float, g: float, d50: float) -> float:
    return q_b / np.sqrt((density_ratio - 1.0) * g * d50 ** 3)


def bed_spectrum(h_xt: np.ndarray, dx: float = 1.0, dt: float = 1.0):
    """PSD of h_b(x, t) given as (nt, nx), and the dominant bedform
    (wavelength, period, signed celerity, amplitude) at the largest value
    with wavenumber index 1 <= j <= nx / 2."""
    h = np.asarray(h_xt, dtype=np.float64)
    nt, nx = h.shape
    X = np.fft.fft2(h - h.mean())
    psd = np.abs(X) ** 2 / (nt * nx)
    half = psd[:, 1:nx // 2 + 1]
    l, j = np.unravel_index(int(np.argmax(half)), half.shape)
    j += 1
    lsig = l if l <= nt // 2 else l - nt
    lam = nx * dx / j
    T = np.inf if lsig == 0 else nt * dt / abs(lsig)
    c = 0.0 if lsig == 0 else -np.sign(lsig) * lam / T
    amp = 2.0 * np.sqrt(psd[l, j] / (nt * nx))
    return psd, (lam, T, c, amp)
