"""Python binding of libfslbm.so (declared in include/fslbm.h).

Argument marshalling only: every step of the method runs in the CUDA
library. The functions keep the C names (fslbm_create, fslbm_add_spheres,
fslbm_step, fslbm_get_fields, ...); ``Simulation`` wraps one handle with numpy
or torch buffers. PyTorch supplies the CUDA stream (and device buffers when a
caller passes torch tensors); nothing here falls back to a CPU computation:
if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfslbm.so")

FSLBM_OK = 0
ERRORS = {
    -1: "EINVAL", -2: "ENOMEM", -3: "ECAPACITY", -4: "ENAN", -5: "EDEVICE", -6: "ESTATE", -7: "EINVARIANT",
    -8: "ETIMEOUT",
}
PERIODIC_X, PERIODIC_Y, PERIODIC_Z = 1, 2, 4
STORE_FP32, STORE_FP16, STORE_BF16 = 0, 1, 2
GAS, LIQUID, INTERFACE, SOLID = 0, 1, 2, 3

FIELD_PDF = 1 << 0
FIELD_TYPE = 1 << 1
FIELD_MASS = 1 << 2
FIELD_PHI = 1 << 3
FIELD_RHO = 1 << 4
FIELD_U = 1 << 5
FIELD_NORMAL = 1 << 6
FIELD_OWNER = 1 << 7
FIELD_P_X = 1 << 16
FIELD_P_U = 1 << 17
FIELD_P_OMEGA = 1 << 18
FIELD_P_F = 1 << 19
FIELD_P_T = 1 << 20
FIELD_P_R = 1 << 21

# every entry point declared in include/fslbm.h
EXPORTED = (
    "fslbm_default_params", "fslbm_create", "fslbm_add_spheres", "fslbm_init_surface", "fslbm_step",
    "fslbm_get_fields", "fslbm_set_fields", "fslbm_reduce", "fslbm_sync", "fslbm_steps_done",
    "fslbm_num_spheres", "fslbm_invariant_violations", "fslbm_timing", "fslbm_timing_read",
    "fslbm_cell_counts", "fslbm_reduce_fields_noalloc", "fslbm_destroy", "fslbm_strerror",
    "fslbm_set_normal_model", "fslbm_set_normal_mirror", "fslbm_normal_stats", "fslbm_mlp_stencils", "fslbm_mlp_gradient",
    "fslbm_mlp_train", "fslbm_mlp_infer", "fslbm_bed_height", "fslbm_set_body_force",
    "fslbm_get_body_force", "fslbm_set_flow_control", "fslbm_set_wait_limit", "fslbm_transport_numbers",
    "fslbm_bed_spectrum", "fslbm_log_stencils",
)

MLP_NPARAM = 6212


class FslbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_strerror(code)})")


class FslbmParams(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc_flags", ctypes.c_uint32),
        ("omega", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("rho_gas", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("liquid_height", ctypes.c_double),
        ("init_profile", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("normal_model", ctypes.c_int32),
        ("reconstruct_normal", ctypes.c_int32),
        ("eps_conv", ctypes.c_double),
        ("eps_normal", ctypes.c_double),
        ("rho_p", ctypes.c_double),
        ("restitution", ctypes.c_double),
        ("friction", ctypes.c_double),
        ("poisson", ctypes.c_double),
        ("collision_time", ctypes.c_double),
        ("dem_substeps", ctypes.c_int32),
        ("link_mass_correction", ctypes.c_int32),
        ("capacity_particles", ctypes.c_int64),
        ("capacity_interface", ctypes.c_int64),
        ("excess_even", ctypes.c_int32),
        ("lubrication", ctypes.c_int32),
        ("galilean_correction", ctypes.c_int32),
        ("link_mode", ctypes.c_int32),
    ]


_lib = None


def load():
    """Loads libfslbm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    L.fslbm_default_params.argtypes = [ctypes.POINTER(FslbmParams)]
    L.fslbm_default_params.restype = None
    L.fslbm_create.argtypes = [ctypes.POINTER(FslbmParams), vp, ctypes.POINTER(vp)]
    L.fslbm_add_spheres.argtypes = [vp, ctypes.c_int64, vp, vp, vp, ctypes.c_int]
    L.fslbm_init_surface.argtypes = [vp, vp, ctypes.c_int]
    L.fslbm_step.argtypes = [vp, ctypes.c_int64]
    L.fslbm_get_fields.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.c_int]
    L.fslbm_set_fields.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.c_int]
    L.fslbm_reduce.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fslbm_sync.argtypes = [vp]
    L.fslbm_steps_done.argtypes = [vp]
    L.fslbm_steps_done.restype = ctypes.c_int64
    L.fslbm_num_spheres.argtypes = [vp]
    L.fslbm_num_spheres.restype = ctypes.c_int64
    L.fslbm_invariant_violations.argtypes = [vp]
    L.fslbm_invariant_violations.restype = ctypes.c_int64
    L.fslbm_timing.argtypes = [vp, ctypes.c_int]
    L.fslbm_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)]
    L.fslbm_cell_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.fslbm_bed_height.argtypes = [vp, ctypes.c_double, vp, vp, ctypes.c_int]
    L.fslbm_set_body_force.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fslbm_get_body_force.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fslbm_set_flow_control.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int64]
    L.fslbm_set_wait_limit.argtypes = [vp, ctypes.c_int64]
    L.fslbm_transport_numbers.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.fslbm_bed_spectrum.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp,
                                     ctypes.POINTER(ctypes.c_double), vp]
    L.fslbm_reduce_fields_noalloc.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), vp, vp]
    L.fslbm_set_normal_model.argtypes = [vp, vp, ctypes.c_int64]
    L.fslbm_set_normal_mirror.argtypes = [vp, ctypes.c_int32]
    L.fslbm_normal_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    L.fslbm_mlp_stencils.argtypes = [vp, ctypes.c_int64, vp, vp, vp]
    L.fslbm_mlp_gradient.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp, vp, vp]
    L.fslbm_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                  vp, vp]
    L.fslbm_mlp_infer.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    L.fslbm_log_stencils.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    L.fslbm_destroy.argtypes = [vp]
    L.fslbm_destroy.restype = None
    L.fslbm_strerror.argtypes = [ctypes.c_int]
    L.fslbm_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def _strerror(code: int) -> str:
    try:
        return load().fslbm_strerror(code).decode()
    except Exception:
        return "?"


def _check(code: int, where: str):
    if code != FSLBM_OK:
        raise FslbmError(code, where)


# ------------------------------------------------------------------ C names

def fslbm_default_params() -> FslbmParams:
    p = FslbmParams()
    load().fslbm_default_params(ctypes.byref(p))
    return p


def fslbm_create(params: FslbmParams, stream: int | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().fslbm_create(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.byref(h)),
           "fslbm_create")
    return h


def fslbm_add_spheres(h, xyz, radius, fixed=None, on_device: bool = False) -> int:
    return load().fslbm_add_spheres(h, len(radius), _ptr(xyz), _ptr(radius), _ptr(fixed) if fixed is not None else None,
                                    int(on_device))


def fslbm_init_surface(h, height_xy, on_device: bool = False) -> int:
    return load().fslbm_init_surface(h, _ptr(height_xy), int(on_device))


def fslbm_step(h, n: int) -> int:
    return load().fslbm_step(h, int(n))


def fslbm_get_fields(h, mask: int, dsts, on_device: bool = False) -> int:
    arr = (ctypes.c_void_p * len(dsts))(*[_ptr(d) for d in dsts])
    return load().fslbm_get_fields(h, ctypes.c_uint32(mask), arr, int(on_device))


def fslbm_set_fields(h, mask: int, srcs, on_device: bool = False) -> int:
    arr = (ctypes.c_void_p * len(srcs))(*[_ptr(d) for d in srcs])
    return load().fslbm_set_fields(h, ctypes.c_uint32(mask), arr, int(on_device))


def fslbm_reduce(h) -> tuple[int, np.ndarray]:
    out = np.zeros(8, np.float64)
    rc = load().fslbm_reduce(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return rc, out


def fslbm_sync(h) -> int:
    return load().fslbm_sync(h)


def fslbm_destroy(h):
    load().fslbm_destroy(h)


def fslbm_reduce_fields_noalloc(pdf, types, mass, ncells: int, g, out, stream: int | None = None) -> int:
    """Allocation-free reduction of caller-held device fields (see the C
    declaration); pdf, types, mass and out are device buffers."""
    gg = (ctypes.c_double * 3)(*[float(v) for v in g])
    return load().fslbm_reduce_fields_noalloc(_ptr(pdf), _ptr(types), _ptr(mass), int(ncells), gg, _ptr(out),
                                              ctypes.c_void_p(stream or 0))


def _stream(stream):
    return ctypes.c_void_p(stream or 0)


def fslbm_bed_spectrum(h, nt: int, nx: int, dx: float, dt: float, psd, stream=None) -> tuple[int, np.ndarray]:
    """PSD of a device bed-height series h (nt, nx) into the device buffer
    psd; returns (code, [wavelength, period, celerity, amplitude])."""
    peak = np.zeros(4, np.float64)
    rc = load().fslbm_bed_spectrum(_ptr(h), int(nt), int(nx), float(dx), float(dt), _ptr(psd),
                                   peak.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream))
    return rc, peak


def fslbm_set_normal_model(h, w_bf16_bits) -> int:
    """w_bf16_bits: host uint16 array of 6212 BF16 bit patterns, or None."""
    if w_bf16_bits is None:
        return load().fslbm_set_normal_model(h, None, 0)
    w = np.ascontiguousarray(w_bf16_bits, np.uint16).reshape(-1)
    return load().fslbm_set_normal_model(h, ctypes.c_void_p(w.ctypes.data), int(w.size))


def fslbm_set_normal_mirror(h, on: bool) -> int:
    return load().fslbm_set_normal_mirror(h, int(bool(on)))


def fslbm_normal_stats(h) -> tuple[int, np.ndarray]:
    out = (ctypes.c_uint64 * 2)()
    rc = load().fslbm_normal_stats(h, out)
    return rc, np.array(list(out), np.uint64)


def fslbm_mlp_stencils(params, n: int, fill, target, stream=None) -> int:
    return load().fslbm_mlp_stencils(_ptr(params), int(n), _ptr(fill), _ptr(target), _stream(stream))


def fslbm_mlp_gradient(theta, fill, target, n: int, lam: float, mu: float, grad, loss, stream=None) -> int:
    return load().fslbm_mlp_gradient(_ptr(theta), _ptr(fill), _ptr(target), int(n), float(lam), float(mu),
                                     _ptr(grad), _ptr(loss), _stream(stream))


def fslbm_mlp_train(theta, fill, target, n: int, steps: int, batch: int, lr: float, lam: float, mu: float,
                    seed: int, augment: bool, loss_curve, stream=None, lr_end: float = 0.0) -> int:
    return load().fslbm_mlp_train(_ptr(theta), _ptr(fill), _ptr(target), int(n), int(steps), int(batch),
                                  float(lr), float(lr_end), float(lam), float(mu), int(seed), int(bool(augment)),
                                  _ptr(loss_curve), _stream(stream))


def fslbm_mlp_infer(theta, fill, n: int, out, stream=None) -> int:
    return load().fslbm_mlp_infer(_ptr(theta), _ptr(fill), int(n), _ptr(out), _stream(stream))


def bf16_bits(theta) -> np.ndarray:
    """BF16 bit patterns (round to nearest even) of FP32 parameters."""
    a = np.ascontiguousarray(theta, np.float32).reshape(-1).view(np.uint32).astype(np.uint64)
    rounded = (a + 0x7FFF + ((a >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):                      # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError(type(a))


# ------------------------------------------------------------------ wrapper

def params_from_workload(w, storage: int = STORE_FP32, link_mode: int = 0) -> FslbmParams:
    p = fslbm_default_params()
    p.nx, p.ny, p.nz = w.nx, w.ny, w.nz
    p.bc_flags = (PERIODIC_X if w.periodic[0] else 0) | (PERIODIC_Y if w.periodic[1] else 0) | \
                 (PERIODIC_Z if w.periodic[2] else 0)
    p.omega = w.omega
    p.g[:] = list(w.g)
    p.rho_gas = w.rho_gas
    p.liquid_height = w.liquid_height
    p.storage = storage
    p.reconstruct_normal = w.reconstruct_normal
    p.eps_conv = w.eps_conv
    p.eps_normal = w.eps_normal
    p.rho_p = w.rho_p
    p.restitution = w.restitution
    p.friction = w.friction
    p.poisson = w.poisson
    p.collision_time = w.collision_time
    p.dem_substeps = w.dem_substeps
    p.lubrication = w.lubrication
    p.galilean_correction = w.galilean_correction
    p.capacity_particles = max(1024, 2 * (w.nspheres or 0))
    p.link_mode = int(link_mode)
    return p


class Simulation:
    """One simulation on the current CUDA device, on a torch stream."""

    def __init__(self, params: FslbmParams, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = params
        self.n = params.nx * params.ny * params.nz
        self.shape = (params.nz, params.ny, params.nx)
        self.h = fslbm_create(params, stream.cuda_stream)

    @classmethod
    def from_workload(cls, w, storage: int = STORE_FP32, stream=None, spheres: bool = True, link_mode: int = 0):
        sim = cls(params_from_workload(w, storage, link_mode), stream)
        if spheres and w.nspheres:
            sim.add_spheres(w.xyz, w.radius, w.fixed)
        return sim

    def close(self):
        if getattr(self, "h", None):
            fslbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_spheres(self, xyz, radius, fixed=None):
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        radius = np.ascontiguousarray(radius, np.float64).reshape(-1)
        fx = None if fixed is None else np.ascontiguousarray(fixed, np.uint8).reshape(-1)
        _check(fslbm_add_spheres(self.h, xyz, radius, fx), "fslbm_add_spheres")

    def init_surface(self, height_xy):
        h = np.ascontiguousarray(height_xy, np.float64).reshape(self.params.ny, self.params.nx)
        _check(fslbm_init_surface(self.h, h), "fslbm_init_surface")

    def step(self, n: int = 1):
        _check(fslbm_step(self.h, n), "fslbm_step")

    def sync(self):
        _check(fslbm_sync(self.h), "fslbm_sync")

    @property
    def nspheres(self) -> int:
        return int(load().fslbm_num_spheres(self.h))

    @property
    def steps_done(self) -> int:
        return int(load().fslbm_steps_done(self.h))

    @property
    def violations(self) -> int:
        return int(load().fslbm_invariant_violations(self.h))

    def _alloc(self, field: int) -> np.ndarray:
        np_ = self.nspheres
        if field == FIELD_PDF:
            return np.empty((27,) + self.shape, np.float64)
        if field == FIELD_TYPE:
            return np.empty(self.shape, np.uint8)
        if field == FIELD_OWNER:
            return np.empty(self.shape, np.int32)
        if field in (FIELD_U, FIELD_NORMAL):
            return np.empty((3,) + self.shape, np.float64)
        if field in (FIELD_P_X, FIELD_P_U, FIELD_P_OMEGA, FIELD_P_F, FIELD_P_T):
            return np.empty((np_, 3), np.float64)
        if field == FIELD_P_R:
            return np.empty((np_,), np.float64)
        return np.empty(self.shape, np.float64)

    def get(self, field: int) -> np.ndarray:
        out = self._alloc(field)
        _check(fslbm_get_fields(self.h, field, [out]), "fslbm_get_fields")
        return out

    def set(self, field: int, arr):
        a = np.ascontiguousarray(arr, np.float64)
        _check(fslbm_set_fields(self.h, field, [a]), "fslbm_set_fields")

    def reduce(self) -> np.ndarray:
        rc, out = fslbm_reduce(self.h)
        _check(rc, "fslbm_reduce")
        return out

    def set_normal_model(self, theta_or_bits, mirror: bool = False):
        """Learned normal from FP32 parameters (rounded to BF16) or BF16 bit
        patterns (uint16); None returns to the finite-difference normal.
        mirror averages the network over the block's mirror images in x and y
        (fslbm_set_normal_mirror)."""
        if theta_or_bits is None:
            _check(fslbm_set_normal_model(self.h, None), "fslbm_set_normal_model")
            return
        a = np.asarray(theta_or_bits)
        bits = a if a.dtype == np.uint16 else bf16_bits(a)
        _check(fslbm_set_normal_mirror(self.h, mirror), "fslbm_set_normal_mirror")
        _check(fslbm_set_normal_model(self.h, bits), "fslbm_set_normal_model")

    def normal_stats(self) -> np.ndarray:
        rc, out = fslbm_normal_stats(self.h)
        _check(rc, "fslbm_normal_stats")
        return out

    def timing(self, on: bool):
        _check(load().fslbm_timing(self.h, int(on)), "fslbm_timing")

    def timing_read(self) -> tuple[float, int, int]:
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        k = ctypes.c_int64()
        _check(load().fslbm_timing_read(self.h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)),
               "fslbm_timing_read")
        return ms.value, n.value, k.value

    def body_force(self) -> np.ndarray:
        g = np.zeros(3)
        _check(load().fslbm_get_body_force(self.h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "fslbm_get_body_force")
        return g

    def set_body_force(self, g) -> None:
        a = np.ascontiguousarray(g, dtype=np.float64)
        _check(load().fslbm_set_body_force(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "fslbm_set_body_force")

    def set_flow_control(self, target_u: float, gain: float, interval: int) -> None:
        _check(load().fslbm_set_flow_control(self.h, float(target_u), float(gain), int(interval)),
               "fslbm_set_flow_control")

    def bed_height(self, level: float = 0.3, with_fraction: bool = False):
        """Bed height h_b(x) (nx,) of Section 3.2 at solid fraction `level`;
        with_fraction also returns phi_b(x, z) as (nz, nx)."""
        h = np.zeros(self.shape[2])
        phi = np.zeros((self.shape[0], self.shape[2])) if with_fraction else None
        _check(load().fslbm_bed_height(self.h, float(level), h.ctypes.data,
                                       phi.ctypes.data if phi is not None else None, 0), "fslbm_bed_height")
        return (h, phi) if with_fraction else h

    def log_stencils(self, capacity: int | None = None):
        """Interface stencils of the current state with height-function labels
        (see fslbm_log_stencils): device tensors fill (n, 27), target (n, 4),
        fd (n, 4) and cells (n,) int32, n the number found (all of them when
        capacity is None)."""
        import torch
        found = ctypes.c_int64()
        if capacity is None:
            _check(load().fslbm_log_stencils(self.h, 0, None, None, None, None, ctypes.byref(found)),
                   "fslbm_log_stencils")
            capacity = int(found.value)
        cap = max(int(capacity), 1)
        dev = torch.device("cuda", torch.cuda.current_device())
        fill = torch.empty((cap, 27), dtype=torch.float32, device=dev)
        target = torch.empty((cap, 4), dtype=torch.float32, device=dev)
        fd = torch.empty((cap, 4), dtype=torch.float32, device=dev)
        cells = torch.empty(cap, dtype=torch.int32, device=dev)
        _check(load().fslbm_log_stencils(self.h, cap, _ptr(fill), _ptr(target), _ptr(fd), _ptr(cells),
                                         ctypes.byref(found)), "fslbm_log_stencils")
        n = min(int(found.value), cap)
        return fill[:n], target[:n], fd[:n], cells[:n]

    def set_wait_limit(self, polls: int) -> None:
        """Polls before a bounded device wait gives up (test hook of the
        error path; see fslbm_set_wait_limit)."""
        _check(load().fslbm_set_wait_limit(self.h, int(polls)), "fslbm_set_wait_limit")

    def transport_numbers(self, d50: float) -> dict:
        """Mean water depth, slope, Shields and Einstein numbers, bedload rate
        and mean bed height of the current state (fslbm_transport_numbers)."""
        out = np.zeros(6, np.float64)
        _check(load().fslbm_transport_numbers(self.h, float(d50), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "fslbm_transport_numbers")
        keys = ("water_depth", "tan_psi", "shields", "q_b", "einstein", "bed_height")
        return dict(zip(keys, (float(v) for v in out)))

    def cell_counts(self) -> np.ndarray:
        out = np.zeros(4, np.int64)
        _check(load().fslbm_cell_counts(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "fslbm_cell_counts")
        return out
