"""Shared test set-up: the same seeded workload handed to the oracle and to
the CUDA library (argument marshalling only)."""
import numpy as np

import oracle as O


def oracle_from_workload(w, spheres=True):
    o = O.Oracle(O.OracleParams(
        nx=w.nx, ny=w.ny, nz=w.nz, periodic=tuple(w.periodic), omega=w.omega, g=tuple(w.g),
        rho_gas=w.rho_gas, liquid_height=w.liquid_height, eps_conv=w.eps_conv, eps_normal=w.eps_normal,
        reconstruct_normal=w.reconstruct_normal, rho_p=w.rho_p, restitution=w.restitution,
        friction=w.friction, poisson=w.poisson, collision_time=w.collision_time,
        dem_substeps=w.dem_substeps))
    if spheres and w.nspheres:
        o.add_spheres(w.xyz, w.radius, w.fixed)
    return o


def weights():
    C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)])
    k = np.abs(C).sum(1)
    return np.select([k == 0, k == 1, k == 2, k == 3], [8 / 27, 2 / 27, 1 / 54, 1 / 216])


def pdf_rel_err(fg, fo, types):
    """max over fluid cells and directions of |f_gpu - f_oracle| / |f_oracle|"""
    fluid = (types == 1) | (types == 2)
    if not fluid.any():
        return 0.0
    a = fg[:, fluid]
    b = fo[:, fluid]
    return float(np.max(np.abs(a - b) / np.abs(b)))
