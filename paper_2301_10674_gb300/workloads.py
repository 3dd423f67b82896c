"""Seeded synthetic workloads for the coupled free-surface LBM / DEM step.

Both the CUDA path and the FP64 oracle are driven from these generators; the
module holds geometry and parameters only, none of the method's arithmetic.

The paper's runs (Section 3.1, Table 1) use a flume with a particle bed of
polydisperse spheres (diameters uniform in [0.9, 1.1] d50, density ratio
2.55), a bottom layer of fixed particles below 1.5 d50, and a free surface
above the bed. The flume measurements the paper compares against are not
needed here; these seeded inputs stand in for the paper's workloads with the
same structure: sizes, sphere distribution, fixed bottom layer, bed height,
liquid depth and slope forcing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC_X = 1
PERIODIC_Y = 2
PERIODIC_Z = 4


@dataclass
class Workload:
    """Lattice, physical parameters and particle bed of one run (lattice units)."""
    name: str
    nx: int
    ny: int
    nz: int
    periodic: tuple = (1, 0, 0)            # x periodic, y and z no-slip walls
    tau: float = 0.51
    g: tuple = (2e-6, 0.0, -1e-5)
    rho_gas: float = 1.0
    liquid_height: float = 26.0
    rho_p: float = 2.55
    restitution: float = 0.88
    friction: float = 0.5
    poisson: float = 0.22
    diameter: float = 6.0                  # nominal d50 (cells)
    dem_substeps: int = 10
    eps_conv: float = 1e-2
    eps_normal: float = 1e-2
    reconstruct_normal: int = 1
    lubrication: int = 1                   # DEM lubrication corrections (Section 2.2)
    galilean_correction: int = 0           # Galilean correction of the collision (off: the paper's runs)
    steps: int = 1000
    seed: int = 1
    spheres_nominal: int = 0
    bed_height: float = 0.0
    bed: str = "hex"                       # "hex" (jittered hexagonal) or "rsd" (deposition)
    polydispersity: float = 0.0            # half-width of the uniform diameter spread
    xyz: np.ndarray = field(default=None, repr=False)
    radius: np.ndarray = field(default=None, repr=False)
    fixed: np.ndarray = field(default=None, repr=False)

    @property
    def omega(self) -> float:
        return 1.0 / self.tau

    @property
    def collision_time(self) -> float:
        # T_c = 4 d50 time steps (Section 2.2)
        return 4.0 * self.diameter

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nspheres(self) -> int:
        return 0 if self.radius is None else int(len(self.radius))

    def generate(self) -> "Workload":
        """Place the particle bed (seeded, deterministic) and return self."""
        rng = np.random.default_rng(self.seed)
        if self.bed == "hex":
            xyz, rad = _jittered_hex(self, rng)
        elif self.bed == "rsd":
            xyz, rad = _deposition(self, rng)
        elif self.bed == "none":
            xyz, rad = np.zeros((0, 3)), np.zeros(0)
        else:
            raise ValueError(self.bed)
        self.xyz = np.ascontiguousarray(xyz, np.float64)
        self.radius = np.ascontiguousarray(rad, np.float64)
        # fixed rough bottom: centres below 1.5 d50 (Section 3.1)
        self.fixed = (self.xyz[:, 2] < 1.5 * self.diameter).astype(np.uint8) if len(rad) else np.zeros(0, np.uint8)
        return self

    def crop_x(self, nx: int, name: str | None = None) -> "Workload":
        """Same workload restricted to x in [0, nx): spheres whose centre lies in
        the crop are kept (those crossing the new periodic seam are dropped)."""
        w = replace(self, nx=nx, name=name or f"{self.name}-crop{nx}")
        if self.xyz is not None:
            keep = (self.xyz[:, 0] - self.radius >= 0) & (self.xyz[:, 0] + self.radius <= nx)
            w.xyz = self.xyz[keep].copy()
            w.radius = self.radius[keep].copy()
            w.fixed = self.fixed[keep].copy()
        return w

    def describe(self) -> dict:
        return {
            "workload": self.name, "lattice": [self.nx, self.ny, self.nz], "cells": self.ncells,
            "spheres": self.nspheres, "spheres_nominal": self.spheres_nominal,
            "d50": self.diameter, "tau": self.tau, "g": list(self.g),
            "liquid_height": self.liquid_height, "bed_height": self.bed_height, "seed": self.seed,
        }


def _diameters(w: Workload, rng, n):
    if w.polydispersity > 0:
        return rng.uniform(w.diameter * (1 - w.polydispersity), w.diameter * (1 + w.polydispersity), n)
    return np.full(n, w.diameter)


def _jittered_hex(w: Workload, rng):
    """Hexagonal close packing with spacing d+1, uniform jitter of +-0.5 cell
    per axis (redrawn while it would overlap a placed sphere), centres kept
    inside the walls and below the bed height."""
    d = w.diameter
    r = d / 2
    s = d + 1.0
    jitter = 0.5
    per_row = max(1, int(w.nx // s))
    sx = w.nx / per_row
    dy = s * math.sqrt(3) / 2
    dz = s * math.sqrt(2.0 / 3.0)
    centres = []
    layer = 0
    z = r + jitter
    while z + r + jitter <= w.bed_height:
        row = 0
        y = r + jitter + (dy / 3 if layer % 2 else 0.0)
        while y + r + jitter <= w.ny:
            for i in range(per_row):
                x = (i + 0.5 * (row % 2) + 0.5 * (layer % 2)) * sx
                centres.append((x % w.nx, y, z))
            row += 1
            y += dy
        layer += 1
        z += dz
    placed = []
    for (x, y, z) in centres:
        for _ in range(100):
            p = np.array([x, y, z]) + rng.uniform(-jitter, jitter, 3)
            p[0] %= w.nx
            ok = True
            for q in placed:
                dd = p - q
                dd[0] -= w.nx * round(dd[0] / w.nx)
                if dd @ dd < d * d:
                    ok = False
                    break
            if ok:
                placed.append(p)
                break
    xyz = np.array(placed).reshape(-1, 3)
    return xyz, np.full(len(xyz), r)


def _deposition(w: Workload, rng, max_fail: int = 400, candidates: int = 24):
    """Random sequential deposition with settling: each sphere is dropped
    near a uniform random (x, y); among `candidates` drop points within one
    diameter of it, the one where the falling sphere first touches the floor
    or a placed sphere at the lowest height is kept (a greedy stand-in for
    rolling into a hollow). Spheres whose top would exceed the bed height are
    rejected; generation stops after `max_fail` consecutive rejections or at
    the nominal count."""
    d_max = w.diameter * (1 + w.polydispersity)
    cell = d_max
    ncx = max(1, int(w.nx // cell))
    ncy = max(1, int(w.ny // cell))
    gx = w.nx / ncx
    gy = w.ny / ncy
    grid: dict = {}
    cap = 1 << 16
    X = np.zeros((cap, 4))
    n = 0
    fails = 0
    target = w.spheres_nominal if w.spheres_nominal > 0 else 10 ** 9
    while fails < max_fail and n < target:
        r = _diameters(w, rng, 1)[0] / 2
        x0 = rng.uniform(0, w.nx)
        y0 = r + rng.uniform(0, 1) * (w.ny - 2 * r)
        ang = rng.uniform(0, 2 * np.pi, candidates)
        rad = w.diameter * np.sqrt(rng.uniform(0, 1, candidates))
        cx = np.concatenate([[x0], (x0 + rad * np.cos(ang)) % w.nx])
        cy = np.concatenate([[y0], np.clip(y0 + rad * np.sin(ang), r, w.ny - r)])
        ix = int(x0 // gx) % ncx
        iy = min(ncy - 1, int(y0 // gy))
        idx = []
        for ddx in (-2, -1, 0, 1, 2):
            for ddy in (-2, -1, 0, 1, 2):
                jy = iy + ddy
                if 0 <= jy < ncy:
                    idx.extend(grid.get(((ix + ddx) % ncx, jy), ()))
        z = np.full(len(cx), r)
        if idx:
            P = X[np.array(idx)]
            dx = P[None, :, 0] - cx[:, None]
            dx -= w.nx * np.round(dx / w.nx)
            dy = P[None, :, 1] - cy[:, None]
            rr = r + P[None, :, 3]
            h2 = rr * rr - dx * dx - dy * dy
            zc = np.where(h2 > 0, P[None, :, 2] + np.sqrt(np.maximum(h2, 0)), -np.inf)
            z = np.maximum(z, zc.max(axis=1))
        k = int(np.argmin(z))
        if z[k] + r > w.bed_height:
            fails += 1
            continue
        fails = 0
        if n == cap:
            cap *= 2
            X = np.concatenate([X, np.zeros_like(X)])
        X[n] = (cx[k], cy[k], z[k], r)
        kx = int(cx[k] // gx) % ncx
        ky = min(ncy - 1, int(cy[k] // gy))
        grid.setdefault((kx, ky), []).append(n)
        n += 1
    return X[:n, :3].copy(), X[:n, 3].copy()


def _gx_for_froude(fr: float, depth: float, gz: float, tau: float) -> float:
    """Slope forcing from a Froude target: U = Fr sqrt(|g_z| h0) and the
    laminar open-channel estimate g_x = 3 nu U / h0^2."""
    nu = (tau - 0.5) / 3.0
    U = fr * math.sqrt(abs(gz) * depth)
    return 3.0 * nu * U / depth ** 2


def tiny() -> Workload:
    """64x16x32 lattice, d = 6 spheres on a jittered hexagonal bed below z = 14,
    liquid to z = 26, tau = 0.51, g = (2e-6, 0, -1e-5)."""
    return Workload(name="tiny-64x16x32", nx=64, ny=16, nz=32, tau=0.51, g=(2e-6, 0.0, -1e-5),
                    liquid_height=26.0, diameter=6.0, bed="hex", bed_height=14.0,
                    spheres_nominal=180, steps=1000, seed=1)


def mid() -> Workload:
    """512x40x96 lattice, d = 8 +-10 %, deposition to bed height 40, depth 30, Fr ~ 1.2."""
    gz = -1e-5
    return Workload(name="mid-512x40x96", nx=512, ny=40, nz=96, tau=0.51,
                    g=(_gx_for_froude(1.2, 30.0, gz, 0.51), 0.0, gz), liquid_height=70.0,
                    diameter=8.0, polydispersity=0.1, bed="rsd", bed_height=40.0,
                    spheres_nominal=7000, steps=20000, seed=2)


def precision() -> Workload:
    """1024x64x128 lattice, d = 8 +-10 %, bed 56, depth 40, Fr ~ 1.3."""
    gz = -1e-5
    return Workload(name="precision-1024x64x128", nx=1024, ny=64, nz=128, tau=0.51,
                    g=(_gx_for_froude(1.3, 40.0, gz, 0.51), 0.0, gz), liquid_height=96.0,
                    diameter=8.0, polydispersity=0.1, bed="rsd", bed_height=56.0,
                    spheres_nominal=30000, steps=10000, seed=3)


def large() -> Workload:
    """3072x96x320 lattice (~94 M cells), d = 10 +-10 %, bed 150, depth 110, Fr ~ 1.2."""
    gz = -1e-5
    return Workload(name="large-3072x96x320", nx=3072, ny=96, nz=320, tau=0.51,
                    g=(_gx_for_froude(1.2, 110.0, gz, 0.51), 0.0, gz), liquid_height=260.0,
                    diameter=10.0, polydispersity=0.1, bed="rsd", bed_height=150.0,
                    spheres_nominal=200000, steps=50000, seed=5)


WORKLOADS = {"tiny": tiny, "mid": mid, "precision": precision, "large": large}


# ---------------------------------------------------------------- surface stencils
# Training and evaluation data of the learned interface normal: analytic
# surfaces passing near the centre of a 3x3x3 block of cells. This function
# draws the surfaces' random parameters only; the fill levels and the exact
# normal and curvature at the surface point are computed from them by the
# CUDA path and, independently, by the oracle.
#
# Row layout (float64, STENCIL_PARAMS columns):
#   0 kind (0 plane, 1 liquid sphere, 2 gas sphere, 3 sine wave)
#   1..3 n0: unit normal toward the gas at the surface point P = s n0
#   4 s in [-1/2, 1/2] (signed offset of P from the centre cell's centre)
#   5 r: sphere radius in [2, 30] cells (kinds 1, 2)
#   6 A: sine amplitude in [1, 8] cells (kind 3)
#   7 k: sine wavenumber 2 pi / lambda, lambda in [16, 256] cells (kind 3)
#   8 phase in [0, 2 pi) (kind 3)
#   9..11 e1: unit vector orthogonal to n0, the direction the sine varies along
STENCIL_PARAMS = 12
STENCIL_KIND_SHARES = (0.35, 0.20, 0.20, 0.25)


def surface_stencils(n: int, seed: int = 4, kinds=None) -> np.ndarray:
    """Seeded parameters of n analytic surfaces (see the row layout above).
    ``kinds`` restricts the draw to the listed kinds (equal shares)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, STENCIL_PARAMS))
    if kinds is None:
        cdf = np.cumsum(STENCIL_KIND_SHARES)
        kind = np.searchsorted(cdf, rng.uniform(0.0, 1.0, n), side="right")
    else:
        kind = np.asarray(kinds)[rng.integers(0, len(kinds), n)]
    kind = np.minimum(kind, 3)
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    n0 = np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)
    # e1: a random direction in the plane orthogonal to n0
    a = np.where(np.abs(n0[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    u = a - np.sum(a * n0, axis=1, keepdims=True) * n0
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(n0, u)
    rot = rng.uniform(0.0, 2.0 * math.pi, n)[:, None]
    e1 = np.cos(rot) * u + np.sin(rot) * v
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    out[:, 0] = kind
    out[:, 1:4] = n0
    out[:, 4] = rng.uniform(-0.5, 0.5, n)
    r = rng.uniform(2.0, 30.0, n)
    out[:, 5] = np.where((kind == 1) | (kind == 2), r, 0.0)
    amp = rng.uniform(1.0, 8.0, n)
    lam = rng.uniform(16.0, 256.0, n)
    phase = rng.uniform(0.0, 2.0 * math.pi, n)
    sine = kind == 3
    out[:, 6] = np.where(sine, amp, 0.0)
    out[:, 7] = np.where(sine, 2.0 * math.pi / lam, 0.0)
    out[:, 8] = np.where(sine, phase, 0.0)
    out[:, 9:12] = e1
    return out


def mlp_initial_weights(seed: int) -> np.ndarray:
    """Seeded initial parameters of the 27-64-64-4 learned normal (FP32):
    He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in)), zero biases, in
    the order W1 (64x27), b1, W2 (64x64), b2, W3 (4x64), b3."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in ((64, 27), (64,), (64, 64), (64,), (4, 64), (4,)):
        if len(shape) == 2:
            lim = math.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-lim, lim, shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)
