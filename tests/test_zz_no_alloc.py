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


def test_noalloc_reduction_spans_many_blocks_and_keeps_no_stale_rows():
    """Synthetic FP64 fields of 3 * 65536 + 17 cells (four blocks of partial
    sums, the last one ragged) against numpy's FP64 sums; then a call on the
    first 1000 cells after the large one: the rows the large call left in the
    shared scratch must not leak into it, and it must repeat bit for bit."""
    import torch
    from paper_2301_10674_gb300 import build as B
    B.build()
    dev = torch.device("cuda")
    n = 3 * 65536 + 17
    rng = np.random.default_rng(7)
    pdf = rng.uniform(0.0, 0.2, (27, n))
    typ = rng.integers(0, 4, n).astype(np.uint8)
    mass = rng.uniform(0.0, 1.0, n)
    g = (1e-5, -2e-5, 3e-5)
    C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], np.float64)

    def expected(k):
        f, t, m = pdf[:, :k], typ[:k], mass[:k]
        fluid = (t == F.LIQUID) | (t == F.INTERFACE)
        rho = f.sum(axis=0)
        j = C.T @ f
        tot = np.where(t == F.LIQUID, rho, 0.0).sum() + np.where(t == F.INTERFACE, m, 0.0).sum()
        mom = [(j[a] - 0.5 * rho * g[a])[fluid].sum() for a in range(3)]
        return np.array([tot] + mom)

    d_pdf = torch.from_numpy(pdf).to(dev)
    d_typ = torch.from_numpy(typ).to(dev)
    d_mass = torch.from_numpy(mass).to(dev)
    stream = torch.cuda.current_stream().cuda_stream

    def call(k, pdf_view):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
        assert F.fslbm_reduce_fields_noalloc(pdf_view, d_typ, d_mass, k, g, out, stream) == 0
        torch.cuda.synchronize()
        return out.cpu().numpy()

    small = 1000
    d_small = d_pdf[:, :small].contiguous()
    first_small = call(small, d_small)
    big = call(n, d_pdf)
    after_small = call(small, d_small)
    for got, k in ((big, n), (first_small, small)):
        ref = expected(k)
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref).max()), (got, ref)
    assert np.array_equal(first_small, after_small)
    assert np.array_equal(big, call(n, d_pdf))
