"""Shared test set-up: the same seeded workload handed to the oracle and to
the CUDA library (argument marshalling only)."""
import numpy as np

import oracle as O


def oracle_from_workload(w, spheres=True, **overrides):
    kw = dict(
        nx=w.nx, ny=w.ny, nz=w.nz, periodic=tuple(w.periodic), omega=w.omega, g=tuple(w.g),
        rho_gas=w.rho_gas, liquid_height=w.liquid_height, eps_conv=w.eps_conv, eps_normal=w.eps_normal,
        reconstruct_normal=w.reconstruct_normal, rho_p=w.rho_p, restitution=w.restitution,
        friction=w.friction, poisson=w.poisson, collision_time=w.collision_time,
        dem_substeps=w.dem_substeps, lubrication=w.lubrication, galilean_correction=w.galilean_correction)
    kw.update(overrides)
    o = O.Oracle(O.OracleParams(**kw))
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


def pdf_dev_err(fg, fo, types):
    """max over fluid cells and directions of |f_gpu - f_oracle|, relative to
    the largest deviation |f_oracle - w| of those cells: the error measured on
    f - w, the part of the PDFs that carries the flow"""
    fluid = (types == 1) | (types == 2)
    if not fluid.any():
        return 0.0
    w = weights()[:, None]
    a = fg[:, fluid]
    b = fo[:, fluid]
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b - w)))


def py_network(scale, kappa0):
    """A hand-built learned-normal network (parameter layout of the library
    and of oracle.mlp) whose raw normal is -scale times the Parker-Youngs
    gradient of its input block and whose curvature is the constant kappa0:
    the first layer forms the gradient's positive and negative parts, the
    second passes them on, the third recombines them."""
    C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], float)
    WPY = np.array([{0: 0.0, 1: 4.0, 2: 2.0, 3: 1.0}[int(np.abs(c).sum())] for c in C])
    W1 = np.zeros((64, 27))
    W1[0:3] = (WPY[:, None] * C).T
    W1[3:6] = -(WPY[:, None] * C).T
    W2 = np.zeros((64, 64))
    W2[np.arange(6), np.arange(6)] = 1.0
    W3 = np.zeros((4, 64))
    W3[:3, 0:3] = -scale * np.eye(3)
    W3[:3, 3:6] = scale * np.eye(3)
    b3 = np.array([0.0, 0.0, 0.0, kappa0])
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), b3])
