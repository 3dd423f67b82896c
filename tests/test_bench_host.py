"""Host-side bookkeeping of bench.py's roofline: algorithmic bytes per sweep
from the cell counts, the achieved bandwidth from the sweep time, and the
ncu traffic figure, which is reported only while the sweep sources are the
ones it was captured from."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(sweep_ms=2.0, sweeps=4):
    # gas, liquid, interface, solid before and after the timed steps
    return {"counts": [100, 700, 20, 180], "counts_after": [100, 690, 30, 180],
            "sweep_ms": sweep_ms, "sweeps": sweeps}


def test_algorithmic_bytes_and_bandwidth(monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: (6000.0, "measured"))
    r = bench._roofline(_run(), "fp16", 1000)
    fluid = (700 + 20 + 690 + 30) / 2.0                     # mean over the two counts
    per_sweep = fluid * (54 * 2 + 1) + (1000 - fluid) * 1
    assert r["bytes_per_launch"] == int(per_sweep)
    assert r["launch_ms"] == pytest.approx(0.5)             # 2 ms over 4 sweeps
    assert r["achieved"] == pytest.approx(per_sweep / 0.5e-3 / 1e9, abs=0.05)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, abs=1e-4)
    assert r["bytes_per_cell"] == {"fluid": 109, "gas_or_solid": 1}
    assert bench._roofline(_run(), "fp32", 1000)["bytes_per_cell"]["fluid"] == 217


def test_traffic_only_for_the_captured_sources(monkeypatch):
    import hashlib
    h = hashlib.sha256()
    for rel in bench.SWEEP_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    current = h.hexdigest()[:16]
    monkeypatch.setattr(bench, "SWEEP_TRAFFIC", {"sources": current, "workload": "w",
                                                 "per_fluid_cell": {"fp16": 200.0, "fp32": None}})
    t, note = bench._sweep_traffic("fp16", 1000.0)
    assert t == 200000 and "w" in note
    assert bench._sweep_traffic("fp32", 1000.0)[0] is None  # no capture for this storage
    monkeypatch.setattr(bench, "SWEEP_TRAFFIC", {"sources": "0" * 16, "workload": "w",
                                                 "per_fluid_cell": {"fp16": 200.0}})
    assert bench._sweep_traffic("fp16", 1000.0)[0] is None  # the sources changed since the capture
