"""FP64 CPU oracle for the coupled free-surface LBM / DEM time step.

TEST INFRASTRUCTURE ONLY. The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The GPU product path
never imports this package and shares no code with it.

The arithmetic lives in ``fslbm_oracle.c`` (plain C, FP64). This module builds
it with gcc and wraps it with ctypes. Helpers that only marshal arguments live
here; nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fslbm_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

# field identifiers of orc_get / orc_set
F_PDF, F_TYPE, F_MASS, F_PHI, F_RHO, F_U, F_NORMAL, F_OWNER, F_CURV = range(9)
P_X, P_U, P_W, P_F, P_T, P_R = 16, 17, 18, 19, 20, 21

GAS, LIQUID, INTERFACE, SOLID = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("omega", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("rho_gas", ctypes.c_double),
        ("liquid_height", ctypes.c_double),
        ("eps_conv", ctypes.c_double),
        ("eps_normal", ctypes.c_double),
        ("reconstruct_normal", ctypes.c_int),
        ("rho_p", ctypes.c_double),
        ("restitution", ctypes.c_double),
        ("friction", ctypes.c_double),
        ("poisson", ctypes.c_double),
        ("collision_time", ctypes.c_double),
        ("dem_substeps", ctypes.c_int),
        ("link_mass_correction", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("excess_even", ctypes.c_int),
        ("lubrication", ctypes.c_int),
        ("galilean_correction", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Params)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_add_spheres.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_init_surface.argtypes = [ctypes.c_void_p, dp]
        L.orc_get.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.orc_set.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.orc_ncells.restype = ctypes.c_long
        L.orc_ncells.argtypes = [ctypes.c_void_p]
        L.orc_nparticles.argtypes = [ctypes.c_void_p]
        L.orc_violations.restype = ctypes.c_long
        L.orc_violations.argtypes = [ctypes.c_void_p]
        L.orc_pool.restype = ctypes.c_double
        L.orc_pool.argtypes = [ctypes.c_void_p]
        L.orc_reduce.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_gravity.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_collide.argtypes = [dp, dp, ctypes.c_double, dp]
        L.orc_feq.argtypes = [ctypes.c_double, dp, dp]
        L.orc_normal_stencil.argtypes = [dp, dp]
        L.orc_set_mlp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.orc_set_mlp_mirror.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_threads.restype = ctypes.c_int
        u8p = ctypes.c_void_p
        L.orc_excess_shares.restype = ctypes.c_int
        L.orc_excess_shares.argtypes = [ctypes.c_int, ctypes.c_double, dp, u8p, ctypes.c_int, dp]
        L.orc_new_interface_mean.restype = ctypes.c_int
        L.orc_new_interface_mean.argtypes = [u8p, dp, dp, dp, dp]
        L.orc_uncovered_state.restype = ctypes.c_int
        L.orc_uncovered_state.argtypes = [u8p, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_set_pool.argtypes = [ctypes.c_void_p, ctypes.c_double]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class OracleParams:
    nx: int
    ny: int
    nz: int
    periodic: tuple = (1, 0, 0)
    omega: float = 1.0
    g: tuple = (0.0, 0.0, 0.0)
    rho_gas: float = 1.0
    liquid_height: float = 1e9
    eps_conv: float = 1e-2
    eps_normal: float = 1e-2
    reconstruct_normal: int = 1
    rho_p: float = 2.55
    restitution: float = 0.88
    friction: float = 0.5
    poisson: float = 0.22
    collision_time: float = 24.0
    dem_substeps: int = 10
    link_mass_correction: int = 1
    sigma: float = 0.0
    excess_even: int = 0
    lubrication: int = 1
    galilean_correction: int = 0

    def _c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.periodic[:] = list(self.periodic)
        p.omega = self.omega
        p.g[:] = list(self.g)
        p.rho_gas = self.rho_gas
        p.liquid_height = self.liquid_height
        p.eps_conv = self.eps_conv
        p.eps_normal = self.eps_normal
        p.reconstruct_normal = self.reconstruct_normal
        p.rho_p = self.rho_p
        p.restitution = self.restitution
        p.friction = self.friction
        p.poisson = self.poisson
        p.collision_time = self.collision_time
        p.dem_substeps = self.dem_substeps
        p.link_mass_correction = self.link_mass_correction
        p.sigma = self.sigma
        p.excess_even = self.excess_even
        p.lubrication = self.lubrication
        p.galilean_correction = self.galilean_correction
        return p


class Oracle:
    """One oracle simulation. Fields come back as numpy arrays shaped
    (nz, ny, nx) (x fastest), PDFs as (27, nz, ny, nx)."""

    def __init__(self, params: OracleParams):
        self.params = params
        self._h = lib().orc_create(ctypes.byref(params._c()))
        self.n = params.nx * params.ny * params.nz
        self.shape = (params.nz, params.ny, params.nx)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_spheres(self, xyz, radius, fixed=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        radius = np.ascontiguousarray(radius, dtype=np.float64).reshape(-1)
        fx = None
        if fixed is not None:
            fx = np.ascontiguousarray(fixed, dtype=np.uint8).reshape(-1)
        lib().orc_add_spheres(self._h, len(radius), _dp(xyz), _dp(radius),
                              fx.ctypes.data if fx is not None else None)

    def init_surface(self, height_xy):
        """Re-initialise the liquid from a surface height per column, shape (ny, nx)."""
        h = np.ascontiguousarray(height_xy, dtype=np.float64).reshape(self.params.ny, self.params.nx)
        lib().orc_init_surface(self._h, _dp(h))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def get(self, which: int) -> np.ndarray:
        n = self.n
        if which == F_PDF:
            a = np.empty((27,) + self.shape, np.float64)
        elif which == F_TYPE:
            a = np.empty(self.shape, np.uint8)
        elif which in (F_U, F_NORMAL):
            a = np.empty((3,) + self.shape, np.float64)
        elif which == F_OWNER:
            a = np.empty(self.shape, np.int32)
        elif which in (P_X, P_U, P_W, P_F, P_T):
            a = np.empty((self.nparticles, 3), np.float64)
        elif which == P_R:
            a = np.empty((self.nparticles,), np.float64)
        else:
            a = np.empty(self.shape, np.float64)
        lib().orc_get(self._h, which, a.ctypes.data)
        del n
        return a

    def set(self, which: int, arr: np.ndarray):
        if which in (F_TYPE, F_OWNER):
            raise ValueError("read-only field")
        a = np.ascontiguousarray(arr, dtype=np.float64)
        lib().orc_set(self._h, which, a.ctypes.data)

    @property
    def nparticles(self) -> int:
        return lib().orc_nparticles(self._h)

    @property
    def violations(self) -> int:
        return lib().orc_violations(self._h)

    @property
    def pool(self) -> float:
        return lib().orc_pool(self._h)

    def set_gravity(self, g) -> None:
        """Body-force acceleration for the following steps (fluid and particles)."""
        self.params.g = tuple(float(v) for v in g)
        lib().orc_set_gravity(self._h, *self.params.g)

    def set_pool(self, value: float) -> None:
        """Test set-up: the mass pool that the next step spreads."""
        lib().orc_set_pool(self._h, float(value))

    def reduce(self) -> np.ndarray:
        out = np.zeros(8, np.float64)
        lib().orc_reduce(self._h, _dp(out))
        return out

    def set_mlp(self, theta, bf16: bool = True, mirror: bool = False) -> None:
        """Learned normal with parameters theta (6212 values, the layout of
        oracle.mlp); None restores the finite-difference normal. mirror
        averages the network over the stencil's mirror images in x and y
        (R-17g)."""
        if theta is None:
            lib().orc_set_mlp(self._h, None, 0)
            return
        a = np.ascontiguousarray(theta, dtype=np.float64)
        assert a.size == 6212
        lib().orc_set_mlp_mirror(self._h, int(mirror))
        if lib().orc_set_mlp(self._h, a.ctypes.data, int(bf16)) != 0:
            raise MemoryError("orc_set_mlp")


def threads() -> int:
    return int(lib().orc_threads())


def collide(f: np.ndarray, g, omega: float) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    out = np.empty(27, np.float64)
    lib().orc_collide(_dp(f), _dp(gg), float(omega), _dp(out))
    return out


def feq(rho: float, u) -> np.ndarray:
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(27, np.float64)
    lib().orc_feq(float(rho), _dp(uu), _dp(out))
    return out


def normal_stencil(phi27) -> np.ndarray:
    a = np.ascontiguousarray(phi27, dtype=np.float64).reshape(27)
    out = np.empty(3, np.float64)
    lib().orc_normal_stencil(_dp(a), _dp(out))
    return out


# Blocks of 3x3x3 cells, index q = (cx+1) + 3(cy+1) + 9(cz+1); WALL marks a
# position beyond a wall face.
WALL = 255


def excess_shares(to_liquid: bool, ex: float, n, receivers, even: bool = False):
    """Shares of a converting cell's excess mass among its block (27,);
    returns (to_pool, shares)."""
    nn = np.ascontiguousarray(n, dtype=np.float64)
    rc = np.ascontiguousarray(receivers, dtype=np.uint8).reshape(27)
    out = np.empty(27, np.float64)
    r = lib().orc_excess_shares(int(bool(to_liquid)), float(ex), _dp(nn), rc.ctypes.data, int(bool(even)), _dp(out))
    return bool(r), out


def new_interface_mean(types, rho, u):
    """(count, rho_bar, u_bar) a new interface cell starts from."""
    t = np.ascontiguousarray(types, dtype=np.uint8).reshape(27)
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(27)
    uu = np.ascontiguousarray(u, dtype=np.float64).reshape(27, 3)
    rb = np.zeros(1)
    ub = np.zeros(3)
    cnt = lib().orc_new_interface_mean(t.ctypes.data, _dp(r), _dp(uu), _dp(rb), _dp(ub))
    return int(cnt), float(rb[0]), ub


def uncovered_state(types, rho, U, W, d):
    """(type, f, rho_bar, u_b, mass) of a cell a particle uncovers."""
    t = np.ascontiguousarray(types, dtype=np.uint8).reshape(27)
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(27)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (U, W, d)]
    f = np.zeros(27)
    rb = np.zeros(1)
    ub = np.zeros(3)
    m = np.zeros(1)
    typ = lib().orc_uncovered_state(t.ctypes.data, _dp(r), _dp(a[0]), _dp(a[1]), _dp(a[2]), _dp(f), _dp(rb),
                                    _dp(ub), _dp(m))
    return int(typ), f, float(rb[0]), ub, float(m[0])
