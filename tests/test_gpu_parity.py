"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs. Cell types and particle maps must match exactly;
FP32 PDFs within 1e-5 relative after one step and 1e-4 after 200 steps."""
import numpy as np
import pytest

import oracle as O
from paper_2301_10674_gb300 import fslbm as F
from paper_2301_10674_gb300 import workloads as W

from helpers import oracle_from_workload, pdf_dev_err, pdf_rel_err, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_10674_gb300 import build as B
    B.build()
    F.load()


def _sim(w, storage=F.STORE_FP32, spheres=True):
    return F.Simulation.from_workload(w, storage=storage, spheres=spheres)


def _compare(sim, o, pdf_tol, check_particles=True, dev_tol=None):
    """Cell types and owners exact; PDFs on f - w within dev_tol (default
    pdf_tol) of the largest deviation; interface masses and normals."""
    tg = sim.get(F.FIELD_TYPE)
    to = o.get(O.F_TYPE)
    mism = int((tg != to).sum())
    assert mism == 0, f"{mism} cell types differ"
    og = sim.get(F.FIELD_OWNER)
    oo = o.get(O.F_OWNER)
    solid = to == O.SOLID
    assert (og[solid] == oo[solid]).all()
    # PDFs measured on f - w (relative to the largest deviation of the
    # oracle's fluid cells), the part of the PDFs that carries the flow
    err = pdf_dev_err(sim.get(F.FIELD_PDF), o.get(O.F_PDF), to)
    assert err < (pdf_tol if dev_tol is None else dev_tol), err
    mg, mo = sim.get(F.FIELD_MASS), o.get(O.F_MASS)
    ifc = to == O.INTERFACE
    if ifc.any():
        assert np.abs(mg[ifc] - mo[ifc]).max() < 50 * pdf_tol
        # the finite-difference normals of the interface cells (used by the
        # next step's boundary condition) from the same fill levels
        ng, no = sim.get(F.FIELD_NORMAL), o.get(O.F_NORMAL)
        assert np.abs(ng[:, ifc] - no[:, ifc]).max() < 1e3 * pdf_tol
    if check_particles and o.nparticles:
        xg, xo = sim.get(F.FIELD_P_X), o.get(O.P_X)
        assert np.abs(xg - xo).max() < 1e-6
    return err


def _periodic_box(nx=10, ny=6, nz=5, g=(1e-4, -5e-5, 2e-5), omega=1.7, seed=3):
    w = W.Workload(name="box", nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1), tau=1 / omega, g=g,
                   liquid_height=1e9, bed="none").generate()
    rng = np.random.default_rng(seed)
    f0 = weights()[:, None, None, None] * (1 + 0.05 * rng.standard_normal((27, nz, ny, nx)))
    return w, f0


def test_collide_stream_periodic_box():
    """Random near-equilibrium PDFs in a fully periodic liquid box: one and
    fifty steps of collision + streaming with forcing."""
    w, f0 = _periodic_box()
    sim = _sim(w)
    o = oracle_from_workload(w)
    sim.set(F.FIELD_PDF, f0)
    o.set(O.F_PDF, f0)
    sim.step(1)
    o.step(1)
    assert _compare(sim, o, 1e-5) < 1e-5
    sim.step(49)
    o.step(49)
    assert _compare(sim, o, 1e-4) < 1e-4
    sim.close()


def test_walls_in_every_axis():
    w, f0 = _periodic_box(nx=7, ny=5, nz=6, g=(1e-4, 0, -1e-4))
    w.periodic = (0, 0, 0)
    sim = _sim(w)
    o = oracle_from_workload(w)
    sim.set(F.FIELD_PDF, f0)
    o.set(O.F_PDF, f0)
    sim.step(1)
    o.step(1)
    _compare(sim, o, 1e-5)
    sim.step(30)
    o.step(30)
    _compare(sim, o, 1e-4)
    sim.close()


@pytest.mark.parametrize("recon,even", [(1, 0), (0, 0), (1, 1)])
def test_free_surface_without_particles(recon, even):
    """Wavy free surface over a no-slip floor: reconstruction, mass exchange,
    conversions and excess mass, with exact cell types every 10 steps; with
    recon = 0 the variant that rebuilds only the PDFs streaming in from gas
    cells (no normal-based rebuild), with even = 1 the variant that splits
    the excess mass evenly over the receivers."""
    w = W.tiny()
    w.bed = "none"
    w.reconstruct_normal = recon
    w.generate()
    p = F.params_from_workload(w)
    p.excess_even = even
    sim = F.Simulation(p)
    o = oracle_from_workload(w, excess_even=even)
    h = 20.0 + 3.0 * np.cos(2 * np.pi * (np.arange(w.nx) + 0.5) / w.nx) \
        + 1.0 * np.sin(2 * np.pi * (np.arange(w.ny)[:, None] + 0.5) / w.ny)
    sim.init_surface(h)
    o.init_surface(h)
    _compare(sim, o, 1e-6)
    sim.step(1)
    o.step(1)
    _compare(sim, o, 1e-5)
    changed = 0
    t0 = o.get(O.F_TYPE)
    for _ in range(20):
        sim.step(10)
        o.step(10)
        # a moving free surface: FP32 against FP64 through mass exchange and
        # conversions leaves up to a few 1e-4 of the largest deviation after
        # 200 steps (measured 1.1e-4 to 2.3e-4), with every cell type equal
        _compare(sim, o, 1e-4, dev_tol=5e-4)
        changed += int((o.get(O.F_TYPE) != t0).sum())
    assert changed > 0
    assert sim.violations == 0 and o.violations == 0
    sim.close()


def test_tiny_workload_200_steps():
    """The 64x16x32 flume with its particle bed: one step, then 200 steps
    with exact types and particle maps every 20 steps."""
    w = W.tiny().generate()
    sim = _sim(w)
    o = oracle_from_workload(w)
    _compare(sim, o, 1e-6)
    sim.step(1)
    o.step(1)
    e1 = _compare(sim, o, 1e-5)
    for _ in range(10):
        sim.step(20)
        o.step(20)
        e = _compare(sim, o, 1e-4)
    fg, fo = sim.get(F.FIELD_P_F), o.get(O.P_F)
    scale = np.abs(fo).max()
    assert np.abs(fg - fo).max() < 1e-3 * scale
    rg, ro = sim.reduce(), o.reduce()
    assert abs(rg[0] - ro[0]) / ro[0] < 1e-6
    print("tiny pdf rel err after 1 / 201 steps:", e1, e)
    sim.close()


@pytest.mark.parametrize("link_corr", [1, 0])
def test_tiny_workload_1000_steps_statistics(link_corr):
    """The 64x16x32 flume for 1000 steps on both sides. Cell types and particle
    owners exact after every one of the first 200 steps; PDFs, measured on
    f - w, within 1e-5 of the largest deviation after one step and 1e-4 after
    200; after 1000 steps the mass drift of each side at most 1e-6, and the
    bulk velocity and the mean bed height within 1% of the oracle's. Run with
    the contact mass correction of R-12a and without it (the drift of both is
    printed)."""
    from oracle import diagnostics as D
    w = W.tiny().generate()
    p = F.params_from_workload(w)
    p.link_mass_correction = link_corr
    sim = F.Simulation(p)
    sim.add_spheres(w.xyz, w.radius, w.fixed)
    o = oracle_from_workload(w, link_mass_correction=link_corr)
    mg0, mo0 = sim.reduce()[0], o.reduce()[0]
    e1 = e200 = None
    for k in range(1, 201):
        sim.step(1)
        o.step(1)
        to = o.get(O.F_TYPE)
        mism = int((sim.get(F.FIELD_TYPE) != to).sum())
        assert mism == 0, f"step {k}: {mism} cell types differ"
        solid = to == O.SOLID
        assert np.array_equal(sim.get(F.FIELD_OWNER)[solid], o.get(O.F_OWNER)[solid]), f"step {k}: owners"
        if k in (1, 200):
            err = pdf_dev_err(sim.get(F.FIELD_PDF), o.get(O.F_PDF), to)
            if k == 1:
                e1 = err
            else:
                e200 = err
    assert e1 < 1e-5, e1
    assert e200 < 1e-4, e200
    sim.step(800)
    o.step(800)
    rg, ro = sim.reduce(), o.reduce()
    drift_g, drift_o = abs(rg[0] - mg0) / mg0, abs(ro[0] - mo0) / mo0
    ub_g, ub_o = rg[4], ro[4]
    hb_g = sim.bed_height(0.3).mean()
    hb_o = D.bed_height(o.get(O.F_TYPE), 0.3).mean()
    print(f"R-12a={link_corr}: pdf err (f - w) {e1:.2e} / {e200:.2e}; drift gpu {drift_g:.2e} oracle {drift_o:.2e}; "
          f"bulk u {ub_g:.6e} vs {ub_o:.6e}; mean h_b {hb_g:.4f} vs {hb_o:.4f}")
    if link_corr:
        assert drift_g < 1e-6 and drift_o < 1e-6, (drift_g, drift_o)
    assert abs(ub_g - ub_o) <= 0.01 * abs(ub_o), (ub_g, ub_o)
    assert abs(hb_g - hb_o) <= 0.01 * abs(hb_o), (hb_g, hb_o)
    assert sim.violations == 0 and o.violations == 0
    sim.close()


def test_moving_particles_cover_and_uncover_cells():
    """Mobile spheres sinking through liquid cover and uncover cells; the
    transitions (pool, refill, owner) must match the oracle exactly."""
    w = W.Workload(name="drop", nx=24, ny=16, nz=24, tau=0.6, g=(0.0, 0.0, -2e-4), liquid_height=20.0,
                   diameter=6.0, bed="none", seed=7).generate()
    w.xyz = np.array([[6.3, 8.1, 12.2], [17.7, 7.6, 10.4], [12.0, 8.0, 3.05]])
    w.radius = np.array([3.0, 2.6, 3.0])
    w.fixed = np.array([0, 0, 1], np.uint8)
    sim = _sim(w)
    o = oracle_from_workload(w)
    u0 = np.array([[0.02, 0.0, -0.01], [-0.015, 0.01, 0.0], [0.0, 0.0, 0.0]])
    sim.set(F.FIELD_P_U, u0)
    o.set(O.P_U, u0)
    owners0 = o.get(O.F_OWNER)
    for _ in range(12):
        sim.step(10)
        o.step(10)
        # spheres moving at 0.02 cover and uncover cells (refills from FP32
        # neighbour averages): up to 3.6e-4 of the largest deviation
        _compare(sim, o, 1e-4, dev_tol=1e-3)
    assert (o.get(O.F_OWNER) != owners0).sum() > 20
    sim.close()


def test_overlapping_moving_spheres_share_cells():
    """Mobile spheres that overlap each other and a fixed sphere: cells
    covered by two of them change owner as they move (the tie goes to the
    smaller |x - X|^2 - r^2). The re-map of sharing particles must find every
    such cell; owners and types are compared with the oracle exactly."""
    w = W.Workload(name="cluster", nx=32, ny=16, nz=24, tau=0.6, g=(0.0, 0.0, -2e-4), liquid_height=20.0,
                   diameter=6.0, bed="none", seed=9).generate()
    w.xyz = np.array([[10.2, 8.1, 10.3], [14.9, 7.7, 11.1], [12.4, 9.3, 14.6], [22.0, 8.0, 5.2],
                      [24.8, 8.4, 9.6]])
    w.radius = np.array([3.0, 2.8, 2.7, 3.1, 2.6])
    w.fixed = np.array([0, 0, 0, 1, 0], np.uint8)
    sim = _sim(w)
    o = oracle_from_workload(w)
    u0 = np.array([[0.015, 0.0, -0.01], [-0.012, 0.004, 0.006], [0.0, -0.01, -0.012], [0.0, 0.0, 0.0],
                   [-0.01, 0.0, -0.015]])
    sim.set(F.FIELD_P_U, u0)
    o.set(O.P_U, u0)
    owners0 = o.get(O.F_OWNER)
    for _ in range(15):
        sim.step(10)
        o.step(10)
        _compare(sim, o, 1e-4, check_particles=False)
        # overlaps of up to a cell make contact forces far above the other
        # tests'; the FP32 contact law then leaves positions ~1e-6 apart
        assert np.abs(sim.get(F.FIELD_P_X) - o.get(O.P_X)).max() < 1e-5
    assert (o.get(O.F_OWNER) != owners0).sum() > 20
    sim.close()


def _links_workload():
    """x extent 288: a full 256-cell bed segment and a partial one of 32
    cells; mobile spheres across the segment border at x = 256, across the
    periodic x seam and near the walls, one fixed sphere."""
    w = W.Workload(name="links", nx=288, ny=12, nz=24, tau=0.6, g=(1e-5, 0.0, -2e-4), liquid_height=20.0,
                   diameter=6.0, bed="none", seed=13).generate()
    w.xyz = np.array([[255.4, 6.2, 9.3], [286.9, 5.7, 8.1], [100.3, 2.9, 4.2], [140.0, 6.0, 3.05],
                      [30.6, 9.2, 12.4]])
    w.radius = np.array([3.0, 2.7, 2.6, 3.0, 2.8])
    w.fixed = np.array([0, 0, 0, 1, 0], np.uint8)
    u0 = np.array([[0.015, -0.004, -0.01], [-0.012, 0.006, 0.004], [0.01, 0.0, -0.006], [0.0, 0.0, 0.0],
                   [0.0, -0.012, -0.014]])
    return w, u0


@pytest.mark.parametrize("storage", [F.STORE_FP32, F.STORE_FP16])
def test_fluid_side_links_match_the_solid_side_pass(storage):
    """Particle links taken inside the liquid and interface kernels (the
    default) against the separate pass over the solid cells: moving spheres
    cover and uncover cells across a bed-segment border, a partial segment
    and the periodic seam. Types and owners exact against the oracle at FP32
    (and between the two forms at every storage); PDFs and hydrodynamic
    forces of the two forms within rounding of each other, and both within
    the oracle tolerance at FP32."""
    w, u0 = _links_workload()
    sims = []
    for mode in (2, 1):
        p = F.params_from_workload(w, storage)
        p.link_mode = mode
        sim = F.Simulation(p)
        sim.add_spheres(w.xyz, w.radius, w.fixed)
        sim.set(F.FIELD_P_U, u0)
        sims.append(sim)
    o = None
    if storage == F.STORE_FP32:
        o = oracle_from_workload(w)
        o.set(O.P_U, u0)
    fmax = 0.0
    for _ in range(4):
        for sim in sims:
            sim.step(15)
        if o is not None:
            o.step(15)
            for sim in sims:
                _compare(sim, o, 1e-4, check_particles=False, dev_tol=1e-3)
        a, b = sims
        assert np.array_equal(a.get(F.FIELD_TYPE), b.get(F.FIELD_TYPE))
        assert np.array_equal(a.get(F.FIELD_OWNER), b.get(F.FIELD_OWNER))
        fa, fb = a.get(F.FIELD_P_F), b.get(F.FIELD_P_F)
        ta, tb = a.get(F.FIELD_P_T), b.get(F.FIELD_P_T)
        fmax = max(fmax, np.abs(fb).max())
        # FP32: rounding only; 16-bit storage: the pass over the solid cells
        # rounds its bounce-back values to 16 bits once more
        tol = 1e-5 if storage == F.STORE_FP32 else 1e-2
        assert np.abs(fa - fb).max() < tol * np.abs(fb).max(), np.abs(fa - fb).max()
        assert np.abs(ta - tb).max() < tol * np.abs(tb).max(), np.abs(ta - tb).max()
        to = a.get(F.FIELD_TYPE)
        if storage == F.STORE_FP32:
            err = pdf_dev_err(a.get(F.FIELD_PDF), b.get(F.FIELD_PDF), to)
            assert err < 1e-5, err
        else:
            fl = (to == 1) | (to == 2)
            dev = np.abs(a.get(F.FIELD_PDF)[:, fl] - b.get(F.FIELD_PDF)[:, fl]) / weights()[:, None]
            assert dev.max() < 2e-3, dev.max()
    assert fmax > 0.0
    for sim in sims:
        assert sim.violations == 0
        sim.close()


@pytest.mark.parametrize("storage,tol", [(F.STORE_FP16, 2e-3), (F.STORE_BF16, 2e-2)])
def test_reduced_precision_storage(storage, tol):
    """PDFs stored as f - w in FP16 / BF16 with FP32 arithmetic: one step of
    the tiny flume within the storage rounding of the deviations."""
    w = W.tiny().generate()
    sim = _sim(w, storage=storage)
    o = oracle_from_workload(w)
    sim.step(1)
    o.step(1)
    tg, to = sim.get(F.FIELD_TYPE), o.get(O.F_TYPE)
    assert (tg == to).all()
    fg, fo = sim.get(F.FIELD_PDF), o.get(O.F_PDF)
    fl = (to == 1) | (to == 2)
    wq = weights()[:, None]
    dev = np.abs(fg[:, fl] - fo[:, fl]) / wq
    assert dev.max() < tol, dev.max()
    sim.close()


def test_mass_conservation_fp32_with_fixed_bed():
    w = W.tiny().generate()
    w.fixed[:] = 1
    sim = _sim(w)
    m0 = sim.reduce()[0]
    sim.step(500)
    m1 = sim.reduce()[0]
    assert abs(m1 - m0) / m0 < 1e-6
    assert sim.violations == 0
    sim.close()


def test_capacity_overflow_is_reported():
    w = W.tiny()
    w.bed = "none"
    w.generate()
    p = F.params_from_workload(w)
    p.capacity_interface = 16
    with pytest.raises(F.FslbmError) as e:
        sim = F.Simulation(p)      # the initial interface layer alone overflows
        sim.step(1)
        sim.sync()
    assert e.value.code == -3


@pytest.mark.parametrize("case", ["flume", "periodic_box", "walled_box"])
@pytest.mark.parametrize("storage", [F.STORE_FP16, F.STORE_BF16, F.STORE_FP32])
def test_reduction_matches_the_exported_fields(storage, case):
    """fslbm_reduce after even and odd steps against FP64 sums over the
    exported PDFs, types, masses and fill levels: liquid mass (liquid rho +
    interface m + pool), momentum (sum c f - rho g / 2 over the fluid cells),
    the fill-weighted bulk velocity and the interface count. Cases: the tiny
    flume, a periodic box and a box with walls on every axis. With 16-bit
    storage and nx a multiple of 4 the reduction takes four cells per thread;
    after an odd step the face rows (wrapped or walled source rows) run as
    quads too and the two pairs at each x end of every row go to the edge
    kernel."""
    if case == "flume":
        w = W.tiny().generate()
        sim = _sim(w, storage=storage)
    else:
        if case == "periodic_box":
            w, f0 = _periodic_box(nx=12, ny=6, nz=5)
        else:
            w, f0 = _periodic_box(nx=16, ny=5, nz=6, g=(1e-4, 0, -1e-4))
            w.periodic = (0, 0, 0)
        sim = _sim(w, storage=storage)
        sim.set(F.FIELD_PDF, f0)
    C = np.array([[q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1] for q in range(27)], float)
    for _ in range(3):     # states after an even, an odd and an even step
        sim.step(1)
        r = sim.reduce()
        f = sim.get(F.FIELD_PDF)
        t = sim.get(F.FIELD_TYPE)
        m, phi = sim.get(F.FIELD_MASS), sim.get(F.FIELD_PHI)
        g = sim.body_force()
        liq, ifc = t == 1, t == 2
        fl = liq | ifc
        rho = f.sum(0)
        mom = np.tensordot(C.T, f, axes=(1, 0)) - 0.5 * rho[None] * g[:, None, None, None]
        mass = rho[liq].sum() + m[ifc].sum() + r[7]
        assert abs(r[0] - mass) <= 1e-7 * mass, (r[0], mass)
        assert np.abs(r[1:4] - mom[:, fl].sum(1)).max() <= 1e-7 * mass
        wphi = np.where(liq, 1.0, phi)
        num, den = (wphi * mom[0])[fl].sum(), (wphi * rho)[fl].sum()
        assert abs(r[4] * den - num) <= 1e-7 * mass
        assert r[5] == ifc.sum()
    sim.close()


def test_non_finite_state_is_reported():
    w, f0 = _periodic_box()
    sim = _sim(w)
    f0[5, 1, 2, 3] = np.nan
    sim.set(F.FIELD_PDF, f0)
    with pytest.raises(F.FslbmError) as e:
        sim.reduce()
    assert e.value.code == -4
    sim.close()


def test_bounded_wait_that_runs_out_is_reported():
    """A wait of the staged sweep on its bulk copies that gives up (here after
    zero polls, set by the test hook) sets FSLBM_ETIMEOUT; the kernel still
    waits for the copies it issued before it leaves, so the context stays
    usable: a fresh simulation on the same device then runs normally and
    matches the oracle."""
    w = _staged_workload()
    sim = _sim(w, storage=F.STORE_FP16)
    sim.set_wait_limit(0)
    with pytest.raises(F.FslbmError) as e:
        sim.step(1)                # an even step: the staged kernel's first wait gives up
        sim.sync()
    assert e.value.code == -8
    with pytest.raises(F.FslbmError) as e:
        sim.step(1)                # the error word is sticky
    assert e.value.code == -8
    sim.close()
    sim = _sim(w, storage=F.STORE_FP16)
    o = oracle_from_workload(w)
    sim.step(2)
    o.step(2)
    to = o.get(O.F_TYPE)
    assert (sim.get(F.FIELD_TYPE) == to).all()
    fl = (to == 1) | (to == 2)
    dev = np.abs(sim.get(F.FIELD_PDF)[:, fl] - o.get(O.F_PDF)[:, fl]) / weights()[:, None]
    assert dev.max() < 2e-3
    sim.close()


def _staged_workload():
    """x extent 256 (a multiple of the 256-cell tile): with 16-bit storage the
    even steps run the staged pair kernel on every tile that holds liquid,
    face rows and x-edges included; the odd steps and FP32 run the pair
    kernel. Spheres sit on the periodic x seam and across tile borders."""
    w = W.Workload(name="staged", nx=256, ny=10, nz=20, tau=0.55, g=(5e-6, 0.0, -5e-5), liquid_height=14.0,
                   diameter=5.0, bed="none", seed=11).generate()
    w.xyz = np.array([[20.3, 5.1, 4.2], [60.7, 4.4, 6.1], [128.2, 5.5, 3.1], [255.5, 5.0, 5.0],
                      [190.4, 4.6, 12.8]])
    w.radius = np.array([2.6, 2.2, 2.9, 2.4, 2.5])
    w.fixed = np.array([0, 0, 1, 0, 0], np.uint8)
    return w


def test_staged_sweep_matches_oracle():
    w = _staged_workload()
    sim = _sim(w)
    o = oracle_from_workload(w)
    h = 14.0 + 2.0 * np.cos(2 * np.pi * (np.arange(w.nx) + 0.5) / w.nx)[None, :] + np.zeros((w.ny, 1))
    sim.init_surface(h)
    o.init_surface(h)
    for k in (1, 1, 9, 30):
        sim.step(k)
        o.step(k)
        _compare(sim, o, 1e-5 if k == 1 else 1e-4)
    assert sim.violations == 0
    sim.close()


@pytest.mark.parametrize("storage,tol", [(F.STORE_FP16, 2e-3), (F.STORE_BF16, 2e-2)])
def test_staged_sweep_16bit(storage, tol):
    """16-bit storage through the staged even step and the pair odd step:
    types exact, PDFs of fluid cells within the storage's rounding after one
    and after four steps (two of each parity)."""
    w = _staged_workload()
    sim = _sim(w, storage=storage)
    o = oracle_from_workload(w)
    for k in (1, 3):
        sim.step(k)
        o.step(k)
        to = o.get(O.F_TYPE)
        assert (sim.get(F.FIELD_TYPE) == to).all()
        fl = (to == 1) | (to == 2)
        dev = np.abs(sim.get(F.FIELD_PDF)[:, fl] - o.get(O.F_PDF)[:, fl]) / weights()[:, None]
        assert dev.max() < tol, (k, dev.max())
    sim.close()


@pytest.mark.parametrize("storage,tol", [(F.STORE_FP16, 1e-2), (F.STORE_BF16, 2e-2)])
def test_16bit_storage_keeps_a_slow_flow_under_a_deep_head(storage, tol):
    """A 110-cell deep liquid at rest starts to flow under a slope force of
    3e-8 (the laminar force of the large flume's Froude target): after 300
    steps its bulk velocity is about 1e-5, a PDF signal 3 w u of 3e-5 w
    beside the hydrostatic head 3 |g_z| h = 3.3e-3 w. The 16-bit stores hold
    deviations from the hydrostatic reference of the flat surface, so the
    rounding acts on the flow: bulk velocity within 1% (FP16) / 2% (BF16) of
    FP32, and the liquid mass kept to 1e-6."""
    w = W.Workload(name="deep", nx=64, ny=16, nz=128, g=(3e-8, 0.0, -1e-5), liquid_height=110.0,
                   bed="none").generate()
    out = {}
    for st in (F.STORE_FP32, storage):
        sim = _sim(w, storage=st, spheres=False)
        m0 = sim.reduce()[0]
        sim.step(300)
        r = sim.reduce()
        assert abs(r[0] / m0 - 1) < 1e-6
        out[st] = r[4]
        sim.close()
    u32, u16 = out[F.STORE_FP32], out[storage]
    assert 5e-6 < u32 < 2e-5, u32
    assert abs(u16 - u32) <= tol * abs(u32), (u16, u32)


def _dry(L=40, **kw):
    # the dry contact law alone (no lubrication correction)
    kw.setdefault("lubrication", 0)
    w = W.Workload(name="dry", nx=L, ny=L, nz=L, periodic=(1, 1, 1), g=(0.0, 0.0, 0.0), liquid_height=0.0,
                   bed="none", **kw).generate()
    return w


@pytest.mark.parametrize("e,r2", [(0.88, 3.0), (0.5, 5.0)])
def test_dem_restitution_on_gpu(e, r2):
    """Head-on collision in a gas-filled box: the GPU's DEM returns the
    restitution coefficient and conserves momentum, like the oracle. The
    sub-steps run in FP32 on exactly antisymmetric pair forces; each velocity
    change rounds to FP32, so the pair's momentum holds to FP32 rounding of
    the collision impulse (1e-6 of m v; 2e-8 observed)."""
    v, r1 = 0.01, 3.0
    w = _dry(restitution=e, diameter=6.0)
    w.xyz = np.array([[10.0, 20, 20], [10.0 + r1 + r2 + 1.0, 20, 20]])
    w.radius = np.array([r1, r2])
    w.fixed = np.zeros(2, np.uint8)
    sim = _sim(w)
    sim.set(F.FIELD_P_U, np.array([[v, 0, 0], [-v, 0, 0]]))
    sim.step(int(1.0 / v + 3 * w.collision_time + 20))
    U = sim.get(F.FIELD_P_U)
    assert abs((U[1, 0] - U[0, 0]) / (2 * v) - e) < 0.01 * e
    m = np.array([r1 ** 3, r2 ** 3])
    assert abs(m @ U[:, 0] - (m[0] - m[1]) * v) < 1e-6 * m.sum() * v
    sim.close()


def test_dem_rolling_on_gpu():
    v0, r = 0.01, 3.0
    w = W.Workload(name="roll", nx=40, ny=16, nz=16, periodic=(1, 1, 0), g=(0.0, 0.0, -1e-3),
                   liquid_height=0.0, bed="none", diameter=6.0, lubrication=0).generate()
    w.xyz = np.array([[10.0, 8.0, r]])
    w.radius = np.array([r])
    w.fixed = np.zeros(1, np.uint8)
    sim = _sim(w)
    sim.set(F.FIELD_P_U, np.array([[v0, 0.0, 0.0]]))
    sim.step(1500)
    U = sim.get(F.FIELD_P_U)[0]
    Wy = sim.get(F.FIELD_P_OMEGA)[0, 1]
    assert abs(U[0] / v0 - 5 / 7) < 2e-3
    assert abs(Wy * r / v0 - 5 / 7) < 2e-3
    sim.close()


@pytest.mark.parametrize("motion", ["approach", "slide"])
def test_dem_lubrication_matches_the_oracle(motion):
    """Lubrication corrections (Section 2.2, reading R-23) near the floor of
    a gas-filled box (omega 1.9): a sphere entering the lubrication range at
    0.01 toward the wall, and a sphere sliding at 0.01 at a fixed gap of
    0.2. The GPU's FP32 contact and lubrication terms summed in FP64 follow
    the FP64 oracle's trajectory: position within 1e-6, velocities within
    1e-3 of the initial speed, after every 20 steps."""
    r, v0 = 3.0, 0.01
    w = W.Workload(name="lub", nx=16, ny=16, nz=16, periodic=(1, 1, 0), tau=1 / 1.9, g=(0.0, 0.0, 0.0),
                   liquid_height=0.0, bed="none", diameter=6.0).generate()
    h0 = 2.0 / 3.0 if motion == "approach" else 0.2
    w.xyz = np.array([[8.0, 8.0, r + h0]])
    w.radius = np.array([r])
    w.fixed = np.zeros(1, np.uint8)
    u0 = np.array([[0.0, 0.0, -v0]]) if motion == "approach" else np.array([[v0, 0.0, 0.0]])
    sim = _sim(w)
    o = oracle_from_workload(w)
    sim.set(F.FIELD_P_U, u0)
    o.set(O.P_U, u0)
    for _ in range(5):
        sim.step(20)
        o.step(20)
        assert np.abs(sim.get(F.FIELD_P_X) - o.get(O.P_X)).max() < 1e-6
        assert np.abs(sim.get(F.FIELD_P_U) - o.get(O.P_U)).max() < 1e-3 * v0
        assert np.abs(sim.get(F.FIELD_P_OMEGA) - o.get(O.P_W)).max() * r < 1e-3 * v0
    # the lubrication acted: the approach slowed, the sliding turned into rolling
    U, Wo = sim.get(F.FIELD_P_U)[0], sim.get(F.FIELD_P_OMEGA)[0]
    if motion == "approach":
        assert -U[2] < 0.9 * v0
    else:
        assert U[0] - r * Wo[1] < 0.8 * v0
    sim.close()


@pytest.mark.parametrize("storage", [F.STORE_FP32, F.STORE_FP16])
def test_mass_conservation_with_moving_bed(storage):
    """Moving spheres pressed against the floor and each other: with the
    moving bounce-back's net injection taken from the pool (R-12a), the
    liquid mass stays within round-off of the storage over 500 steps."""
    w = W.tiny().generate()
    sim = _sim(w, storage=storage)
    m0 = sim.reduce()[0]
    sim.step(500)
    m1 = sim.reduce()[0]
    assert abs(m1 - m0) / m0 < 1e-6, (m0, m1)
    assert np.abs(sim.get(F.FIELD_P_X) - w.xyz).max() > 1e-3
    assert sim.violations == 0
    sim.close()


def test_bed_height_matches_oracle():
    """Bed topography (Section 3.2) of a bed that has moved for a few steps:
    the library's phi_b(x, z) equals the oracle's definition applied to the
    same cell types exactly, and h_b(x) to rounding, at two thresholds."""
    from oracle import diagnostics as D
    w = W.tiny().generate()
    sim = _sim(w)
    sim.step(3)
    t = sim.get(F.FIELD_TYPE)
    for level in (0.3, 0.55):
        h, phi = sim.bed_height(level, with_fraction=True)
        assert np.array_equal(phi, D.solid_fraction(t))
        assert np.allclose(h, D.bed_height(t, level), rtol=0.0, atol=1e-12)
        # the sparse hexagonal bed: some columns reach the threshold near
        # the bed top, the others only at the wall
        assert h.max() > 5.0 and h.min() >= -0.5 and h.max() <= w.nz + 0.5
    with pytest.raises(F.FslbmError):
        sim.bed_height(0.0)
    sim.close()


def test_flow_rate_control_matches_oracle():
    """Flow-rate control (Section 3.1) of a laminar film started from rest:
    after every 500 steps the library's body force equals the oracle
    controller's on the same film (same law, same update points), and the
    bulk velocities agree."""
    from oracle import flow_control as FC
    w = W.Workload(name="film", nx=8, ny=4, nz=24, periodic=(1, 1, 0), tau=1.0, g=(0.0, 0.0, 0.0),
                   liquid_height=16.0, bed="none", seed=1).generate()
    sim = _sim(w, spheres=False)
    o = oracle_from_workload(w, spheres=False)
    nu = (1.0 - 0.5) / 3
    target, gain, interval = 2e-4, 0.15 * 3 * nu / 16.0 ** 2, 100
    sim.set_flow_control(target, gain, interval)
    for _ in range(6):
        sim.step(500)
        hist = FC.run_controlled(o, 500, target, gain, interval)
        assert sim.body_force()[0] == pytest.approx(hist[-1, 1], rel=2e-3)
    assert sim.reduce()[4] == pytest.approx(o.reduce()[4], rel=2e-3)
    with pytest.raises(F.FslbmError):
        sim.set_flow_control(target, -1.0, interval)
    sim.set_flow_control(0.0, 0.0, 0)
    g = sim.body_force()
    sim.step(100)
    assert np.array_equal(sim.body_force(), g)          # control off: the force stays
    sim.close()


def test_bed_spectrum_matches_the_oracle():
    """PSD of a bed-height series (Section 4.1) on the GPU against the
    oracle's numpy transform: two travelling sines and noise on a 40 x 96
    grid, PSD within 1e-9 of its largest value, and the same dominant bedform
    (wavelength, period, celerity, amplitude)."""
    import torch
    from oracle import diagnostics as D
    nt, nx, dx, dt = 40, 96, 1.0, 25.0
    rng = np.random.default_rng(5)
    x = np.arange(nx)
    t = np.arange(nt)[:, None]
    h = 140.0 + 1.3 * np.sin(2 * np.pi * (4 * x / nx - 3 * t / nt)) + 0.4 * np.cos(2 * np.pi * (9 * x / nx + 2 * t / nt)) \
        + 0.05 * rng.standard_normal((nt, nx))
    dh = torch.from_numpy(h).cuda()
    psd = torch.empty((nt, nx), dtype=torch.float64, device="cuda")
    rc, peak = F.fslbm_bed_spectrum(dh, nt, nx, dx, dt, psd)
    assert rc == 0
    ref, (lam, T, c, amp) = D.bed_spectrum(h, dx, dt)
    got = psd.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-9 * ref.max()
    assert np.allclose(peak, [lam, T, c, amp], rtol=1e-9, atol=0)
    assert peak[0] == pytest.approx(24.0) and peak[2] > 0
    assert F.fslbm_bed_spectrum(dh, 1, nx, dx, dt, psd)[0] == -1


def test_transport_numbers_match_their_definitions():
    """Mean water depth, slope, Shields and Einstein numbers (Section 4.2,
    Table 2) of the tiny flume after a few steps: the library's values equal
    the oracle's definitions applied to the same cell types and fill levels,
    and the bedload rate of Eq. (1) that fslbm_reduce returns."""
    from oracle import diagnostics as D
    w = W.tiny().generate()
    sim = _sim(w)
    sim.step(12)
    tn = sim.transport_numbers(w.diameter)
    t, phi = sim.get(F.FIELD_TYPE), sim.get(F.FIELD_PHI)
    depth = D.mean_water_depth(t, phi)
    assert tn["water_depth"] == pytest.approx(depth, rel=0, abs=1e-9)
    assert tn["bed_height"] == pytest.approx(D.bed_height(t, 0.3).mean(), rel=0, abs=1e-9)
    tp = w.g[0] / abs(w.g[2])
    assert tn["tan_psi"] == pytest.approx(tp, rel=1e-15)
    assert tn["shields"] == pytest.approx(D.shields(depth, tp, w.rho_p, w.diameter), rel=1e-9)
    qb = sim.reduce()[6]
    assert tn["q_b"] == pytest.approx(qb, rel=1e-12, abs=1e-300)
    assert tn["einstein"] == pytest.approx(D.einstein(qb, w.rho_p, float(np.linalg.norm(w.g)), w.diameter),
                                           rel=1e-9, abs=1e-300)
    assert 10.0 < tn["water_depth"] < 26.0
    sim.close()


def test_galilean_correction_matches_the_oracle():
    """Galilean-invariance correction of the second-order relaxation (R-3
    variant; one-cell kernels): a longitudinal wave riding on U = 0.1 in a
    periodic 64 x 2 x 2 box. PDFs on f - w within 1e-5 of the oracle's after
    60 steps; and on the GPU its fluctuation energy decays at the rate of the
    wave at rest to 0.3% (4.5% slower without the correction)."""
    nx, k, A = 64, 2 * np.pi / 64, 1e-3

    def start(U):
        x = np.arange(nx) + 0.5
        f = np.zeros((27, 2, 2, nx))
        for i in range(nx):
            f[:, :, :, i] = O.feq(1.0, [U + A * np.sin(k * x[i]), 0, 0])[:, None, None]
        return f

    def gpu_decay(U, gal, steps=300, every=10):
        w = W.Workload(name="wave", nx=nx, ny=2, nz=2, periodic=(1, 1, 1), tau=1.0, g=(0.0, 0.0, 0.0),
                       liquid_height=1e9, bed="none", galilean_correction=gal).generate()
        sim = _sim(w, spheres=False)
        sim.set(F.FIELD_PDF, start(U))
        E = []
        for _ in range(0, steps, every):
            sim.step(every)
            rho, u = sim.get(F.FIELD_RHO), sim.get(F.FIELD_U)[0]
            E.append(((rho - rho.mean()) ** 2 / 3 + (u - u.mean()) ** 2).sum())
        sim.close()
        t = np.arange(1, len(E) + 1) * every
        return -np.polyfit(t, np.log(E), 1)[0]

    w = W.Workload(name="wave", nx=nx, ny=2, nz=2, periodic=(1, 1, 1), tau=1.0, g=(0.0, 0.0, 0.0),
                   liquid_height=1e9, bed="none", galilean_correction=1).generate()
    sim = _sim(w, spheres=False)
    o = oracle_from_workload(w, spheres=False)
    f0 = start(0.1)
    sim.set(F.FIELD_PDF, f0)
    o.set(O.F_PDF, f0)
    sim.step(60)
    o.step(60)
    t = o.get(O.F_TYPE)
    assert pdf_dev_err(sim.get(F.FIELD_PDF), o.get(O.F_PDF), t) < 1e-5
    sim.close()
    g0 = gpu_decay(0.0, 1)
    assert abs(gpu_decay(0.1, 1) / g0 - 1) < 0.003
    assert gpu_decay(0.1, 0) / g0 - 1 < -0.04
