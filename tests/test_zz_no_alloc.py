"""The allocation-free reduction entry point (for callers that cannot call
cudaMalloc, e.g. code inside another framework's memory pool) against the
library's own reduction, on two calls in a row. Collected last on purpose."""
import numpy as np
import pytest

from paper_2301_10674_gb300 import fslbm as F
from paper_2301_10674_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_fslbm_reduce():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_10674_gb300 import build as B
    B.build()
    w = W.tiny().generate()
    sim = F.Simulation.from_workload(w)
    sim.step(10)
    ref = sim.reduce()
    n = sim.n
    dev = torch.device("cuda")
    pdf = torch.empty((27, n), dtype=torch.float64, device=dev)
    typ = torch.empty(n, dtype=torch.uint8, device=dev)
    mass = torch.empty(n, dtype=torch.float64, device=dev)
    rc = F.fslbm_get_fields(sim.h, F.FIELD_PDF | F.FIELD_TYPE | F.FIELD_MASS, [pdf, typ, mass], on_device=True)
    assert rc == 0
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
        assert F.fslbm_reduce_fields_noalloc(pdf, typ, mass, n, w.g, out, stream) == 0
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    mass_ref = ref[0] - ref[7]
    for o in outs:
        assert abs(o[0] - mass_ref) <= 1e-6 * abs(mass_ref)
        assert np.abs(o[1:] - ref[1:4]).max() <= 1e-6 * abs(mass_ref)
    assert np.array_equal(outs[0], outs[1])
    # sizes beyond the scratch are refused before any work
    assert F.fslbm_reduce_fields_noalloc(pdf, typ, mass, 4096 * 65536 + 1, w.g, out, stream) == -3
    sim.close()
