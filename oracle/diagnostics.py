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
