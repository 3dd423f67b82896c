"""Physics pins of the oracle's streaming, boundary conditions, free-surface
boundary condition and momentum exchange (Sections 2.1 and 2.2), each against
a closed form of the continuum problem."""
import numpy as np
import pytest

import oracle as O


def test_open_channel_half_poiseuille():
    """Gravity-driven film on a no-slip floor with a free surface on top:
    u(z) = (g_x / nu) (H z - z^2 / 2), H the liquid volume per column."""
    gx, om, nz = 1e-6, 1.0, 24
    o = O.Oracle(O.OracleParams(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), omega=om, g=(gx, 0, 0),
                                liquid_height=16.0))
    o.step(6000)
    u = o.get(O.F_U)[0, :, 0, 0]
    t = o.get(O.F_TYPE)[:, 0, 0]
    H = o.get(O.F_PHI)[:, 0, 0].sum()
    nu = (1 / om - 0.5) / 3
    z = np.arange(nz) + 0.5
    ua = gx / nu * (H * z - z * z / 2)
    liq = t == O.LIQUID
    err = np.sqrt(np.sum((u[liq] - ua[liq]) ** 2) / np.sum(ua[liq] ** 2))
    assert err < 0.005


def test_hydrostatic_column_under_flat_surface():
    """At rest, rho(z) = rho_gas exp(3 |g_z| (H - z)) (pressure c_s^2 rho equals
    the gas pressure at the surface), and spurious currents vanish."""
    gz, nz = -1e-5, 40
    o = O.Oracle(O.OracleParams(nx=2, ny=2, nz=nz, periodic=(1, 1, 0), omega=1.0, g=(0, 0, gz),
                                liquid_height=30.0))
    o.step(8000)
    rho = o.get(O.F_RHO)[:, 0, 0]
    t = o.get(O.F_TYPE)[:, 0, 0]
    u = o.get(O.F_U)
    liq = t == O.LIQUID
    z = np.arange(nz) + 0.5
    slope = np.polyfit(z[liq], np.log(rho[liq]), 1)[0]
    assert abs(slope / (-3 * abs(gz)) - 1) < 1e-3
    H = o.get(O.F_PHI)[:, 0, 0].sum()
    pred = np.exp(3 * abs(gz) * (H - z))
    assert np.abs(rho[liq] / pred[liq] - 1).max() < 1e-6
    assert np.abs(u[:, liq]).max() < 1e-6


def test_moving_boundary_couette_and_momentum_exchange():
    """A fixed particle with a prescribed surface velocity U (a huge sphere,
    locally a plane at z = 16) over a no-slip floor: linear Couette profile
    u = U z / 16, and the momentum-exchange force on the particle equals the
    wall shear stress times the area, F_x = -nu U / 16 * (n_x n_y)."""
    U, om, nz, Hs, R = 0.01, 1.0, 24, 16.0, 200.0
    o = O.Oracle(O.OracleParams(nx=4, ny=4, nz=nz, periodic=(1, 1, 0), omega=om, liquid_height=1e9))
    o.add_spheres([[2.0, 2.0, Hs + R]], [R], [1])
    o.set(O.P_U, np.array([[U, 0.0, 0.0]]))
    o.step(3000)
    u = o.get(O.F_U)[0, :, 0, 0]
    t = o.get(O.F_TYPE)[:, 0, 0]
    liq = t == O.LIQUID
    assert liq.sum() == 16 and (t[16:] == O.SOLID).all()
    z = np.arange(nz) + 0.5
    assert np.abs(u[liq] - U * z[liq] / Hs).max() < 1e-6 * U
    F = o.get(O.P_F)[0]
    nu = (1 / om - 0.5) / 3
    assert abs(F[0] / (-nu * U / Hs * 16) - 1) < 1e-6
    assert abs(F[1]) < 1e-12


def test_hasimoto_drag_of_periodic_sphere_array():
    """Stokes drag on a simple-cubic array of fixed spheres (Hasimoto 1959):
    F = 6 pi mu r U K(c), 1/K = 1 - 1.7601 c^(1/3) + c - 1.5593 c^2, with U the
    superficial velocity. The run starts from the expected terminal flow so
    that the drag is quasi-steady after a few hundred steps. At r = 4 cells
    (volume fraction 0.019) the voxelised sphere's drag is within 5% of the
    series (a radius of 3 cells still carries a 6% voxelisation offset)."""
    L, r, om, gx = 24, 4.0, 1.0, 1e-6
    o = O.Oracle(O.OracleParams(nx=L, ny=L, nz=L, periodic=(1, 1, 1), omega=om, g=(gx, 0, 0),
                                liquid_height=1e9))
    o.add_spheres([[L / 2, L / 2, L / 2]], [r], [1])
    nu = (1 / om - 0.5) / 3
    c = (4 / 3) * np.pi * r ** 3 / L ** 3
    K = 1 / (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2)
    fl = o.get(O.F_TYPE) == O.LIQUID
    U0 = gx * fl.sum() / (6 * np.pi * nu * r * K) * L ** 3 / fl.sum()
    f = np.broadcast_to(O.feq(1.0, [U0, 0, 0])[:, None, None, None], (27,) + o.shape).copy()
    o.set(O.F_PDF, f)
    o.step(400)
    F = o.get(O.P_F)[0, 0]
    u = o.get(O.F_U)[0]
    rho = o.get(O.F_RHO)
    Ubar = (rho[fl] * u[fl]).sum() / L ** 3
    ratio = F / (6 * np.pi * nu * r * Ubar) / K
    assert abs(ratio - 1) < 0.05, ratio


def _wave_period_ratio(lam, a_over_lam=0.01, periods=1.3):
    """Period of a standing wave of wavelength lam (depth lam / 8, amplitude
    a_over_lam * lam, gravity 2e-4 * 64 / lam) over the linear dispersion
    relation's, from the first three zero crossings of its cos(kx) mode."""
    h0, a, gz = 0.125 * lam, a_over_lam * lam, -2e-4 * 64 / lam
    nz = int(h0 + 3 * a + 6)
    o = O.Oracle(O.OracleParams(nx=lam, ny=1, nz=nz, periodic=(1, 1, 0), omega=1.97, g=(0, 0, gz),
                                liquid_height=h0))
    x = np.arange(lam) + 0.5
    k = 2 * np.pi / lam
    o.init_surface((h0 + a * np.cos(k * x))[None, :])
    T0 = 2 * np.pi / np.sqrt(abs(gz) * k * np.tanh(k * h0))
    every = max(1, int(T0 / 200))
    ts, eta = [], []
    for st in range(0, int(periods * T0), every):
        o.step(every)
        col = o.get(O.F_PHI)[:, 0, :].sum(axis=0)
        ts.append(st + every)
        eta.append(2 / lam * np.sum((col - col.mean()) * np.cos(k * x)))
    eta, ts = np.array(eta), np.array(ts)
    zc = [ts[i] + (ts[i + 1] - ts[i]) * eta[i] / (eta[i] - eta[i + 1])
          for i in range(len(eta) - 1) if eta[i] * eta[i + 1] < 0]
    assert len(zc) >= 3 and o.violations == 0
    T = 2 * np.mean(np.diff(zc[:3]))
    return T / T0


def test_standing_gravity_wave_dispersion():
    """Standing gravity wave of amplitude lam / 100, omega^2 = g k tanh(k h):
    the free-surface boundary condition holds the pressure at interface-cell
    centres, so the period error is first order in the cell size once the
    amplitude spans a few cells. At lam = 128 and 256 cells the error falls
    by about half (9.5% to 4.2%), and the first-order Richardson
    extrapolation of the pair lies within 2% of the dispersion relation
    (1.1%)."""
    r128 = _wave_period_ratio(128)
    r256 = _wave_period_ratio(256)
    e128, e256 = abs(r128 - 1), abs(r256 - 1)
    assert e256 < 0.05
    assert 1.6 < e128 / e256 < 2.6              # first order
    assert abs((2 * r256 - r128) - 1) < 0.02


def test_flow_rate_controller_settles_on_the_film_force():
    """The body-force controller (Section 3.1; law of the flow_control module)
    on a gravity-free start: it must reach the bulk velocity asked for, with
    g_x at the value the half-Poiseuille film needs for it, 3 nu U / H^2."""
    from oracle import flow_control as FC
    om, nz = 1.0, 24
    o = O.Oracle(O.OracleParams(nx=1, ny=1, nz=nz, periodic=(1, 1, 0), omega=om, g=(0.0, 0, 0),
                                liquid_height=16.0))
    nu = (1 / om - 0.5) / 3
    H = o.get(O.F_PHI)[:, 0, 0].sum()
    target = 2e-4
    gain = 0.15 * 3 * nu / H ** 2
    hist = FC.run_controlled(o, 12000, target, gain, 100)
    assert hist[0, 2] == 0.0 and hist[0, 1] == pytest.approx(gain * target, rel=1e-12)   # from rest
    g_film = 3 * nu * target / H ** 2
    assert abs(hist[-1, 1] / g_film - 1) < 5e-3
    assert abs(hist[-1, 2] / target - 1) < 1e-3
    assert np.all(np.abs(hist[-10:, 2] / target - 1) < 2e-3)
