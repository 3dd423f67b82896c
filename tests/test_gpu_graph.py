"""Graph replay of the time step: a simulation on a captured stream (steps
replayed from CUDA graphs from the third step on) and one on the legacy
default stream (direct launches) give bitwise the same state, also across a
change of the body force (the graphs are captured again), and the sweep
timing hooks still see every step."""
import numpy as np
import pytest

from paper_2301_10674_gb300 import fslbm as F
from paper_2301_10674_gb300 import workloads as W

from helpers import py_network

pytestmark = pytest.mark.gpu

FIELDS = (F.FIELD_PDF, F.FIELD_MASS, F.FIELD_TYPE, F.FIELD_OWNER, F.FIELD_P_X, F.FIELD_P_U, F.FIELD_P_OMEGA)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_10674_gb300 import build as B
    B.build()
    F.load()


def _pair(storage, learned, spheres=True):
    import torch
    w = W.tiny().generate()
    legacy = torch.cuda.default_stream()
    assert legacy.cuda_stream == 0
    a = F.Simulation.from_workload(w, storage=storage, stream=legacy, spheres=spheres)
    b = F.Simulation.from_workload(w, storage=storage, stream=torch.cuda.Stream(), spheres=spheres)
    if learned:
        net = py_network(1.0 / 16.0, 0.0)
        a.set_normal_model(net)
        b.set_normal_model(net)
    return w, a, b


def _same(a, b, fields=FIELDS):
    for f in fields:
        assert np.array_equal(a.get(f), b.get(f)), f


def _close(a, b):
    """Types and owners exact; PDFs, masses and particle states within the
    run-to-run spread of the FP64 atomics (hydrodynamic force and torque per
    particle, the mass pool), which sum in no fixed order: a few FP32 units in
    the last place (a stale launch argument, such as the body force of before
    a change, would leave differences of 1e-4)."""
    for f in (F.FIELD_TYPE, F.FIELD_OWNER):
        assert np.array_equal(a.get(f), b.get(f)), f
    assert np.abs(a.get(F.FIELD_PDF) - b.get(F.FIELD_PDF)).max() < 1e-6
    assert np.abs(a.get(F.FIELD_MASS) - b.get(F.FIELD_MASS)).max() < 1e-6
    # contacts amplify the order of the force sums: 3e-10 seen after 25 steps
    assert np.abs(a.get(F.FIELD_P_X) - b.get(F.FIELD_P_X)).max() < 1e-8


@pytest.mark.parametrize("storage,learned", [(F.STORE_FP32, False), (F.STORE_FP16, True), (F.STORE_BF16, False)])
def test_graph_replay_is_bitwise_direct_launches(storage, learned):
    """Without particles no floating-point atomic decides the state: the
    replayed graphs must give bitwise the direct launches' state."""
    w, a, b = _pair(storage, learned, spheres=False)
    for s in (a, b):
        s.step(25)
    _same(a, b, (F.FIELD_PDF, F.FIELD_MASS, F.FIELD_TYPE))
    g = np.array(w.g) * 1.5
    for s in (a, b):
        s.set_body_force(g)
        s.step(14)
    _same(a, b, (F.FIELD_PDF, F.FIELD_MASS, F.FIELD_TYPE))
    assert a.steps_done == b.steps_done == 39
    a.close()
    b.close()


def test_graph_replay_with_moving_particles():
    """Moving spheres (particle map, DEM on the side stream, pool) across a
    change of the body force, which makes the graphs be captured again."""
    w, a, b = _pair(F.STORE_FP32, True)
    u0 = a.get(F.FIELD_P_U)
    u0[w.fixed == 0, 0] = 0.02
    for s in (a, b):
        s.set(F.FIELD_P_U, u0)
        s.step(25)
    _close(a, b)
    for s in (a, b):
        s.set_body_force(np.array(w.g) * 1.5)
        s.step(14)
    _close(a, b)
    a.close()
    b.close()


def test_timing_hooks_see_replayed_steps():
    _, a, b = _pair(F.STORE_FP32, False)
    counts = []
    for s in (a, b):
        s.step(4)
        s.timing(True)
        s.step(6)
        ms, sweeps, launches = s.timing_read()
        s.timing(False)
        assert sweeps == 6 and ms > 0.0
        counts.append(launches)
    # the graphs hold the same kernels as the direct launches
    assert counts[0] == counts[1] > 0
    _close(a, b)
    a.close()
    b.close()
