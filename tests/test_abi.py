"""The C-ABI library builds, loads and exports every entry point that
include/fslbm.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2301_10674_gb300 import build as B
from paper_2301_10674_gb300 import fslbm as F

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fslbm.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fslbm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(F.EXPORTED)


def test_params_struct_matches_c_layout(lib):
    p = F.fslbm_default_params()
    assert p.struct_size == ctypes.sizeof(F.FslbmParams)
    assert p.dem_substeps == 10 and abs(p.omega - 1 / 0.51) < 1e-15


def test_invalid_parameters_are_rejected_before_any_device_work(lib):
    bad = []
    for field, value in (("nx", 0), ("omega", 2.0), ("sigma", -0.1), ("sigma", float("nan")), ("storage", 7),
                         ("dem_substeps", 0), ("restitution", 0.0), ("normal_model", 2),
                         ("normal_model", -1)):
        p = F.fslbm_default_params()
        p.nx = p.ny = p.nz = 4
        setattr(p, field, value)
        h = ctypes.c_void_p()
        rc = lib.fslbm_create(ctypes.byref(p), None, ctypes.byref(h))
        bad.append((field, rc))
    assert all(rc == -1 for _, rc in bad), bad
    p = F.fslbm_default_params()
    p.struct_size = 8
    h = ctypes.c_void_p()
    assert lib.fslbm_create(ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert lib.fslbm_strerror(-3).decode() == "device list capacity exceeded"


def test_new_entry_points_reject_a_missing_handle(lib):
    g = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    h = (ctypes.c_double * 4)()
    assert lib.fslbm_bed_height(None, 0.3, ctypes.cast(h, ctypes.c_void_p), None, 0) == -1
    assert lib.fslbm_set_body_force(None, g) == -1
    assert lib.fslbm_get_body_force(None, g) == -1
    assert lib.fslbm_set_flow_control(None, 1e-3, 1e-4, 100) == -1
    assert lib.fslbm_set_wait_limit(None, 0) == -1
    assert lib.fslbm_set_normal_mirror(None, 1) == -1
    assert lib.fslbm_strerror(-8).decode() == "a bounded device wait gave up"
