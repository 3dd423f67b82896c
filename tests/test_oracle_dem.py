"""Pins of the oracle's DEM (Section 2.2: linear contact model parameterised
by the restitution coefficient, collision time, Poisson ratio and friction
coefficient) and of the bedload rate of Eq. (1)."""
import numpy as np
import pytest

import oracle as O


def _dry(L=40, **kw):
    # the dry contact law alone (no lubrication correction)
    p = O.OracleParams(nx=L, ny=L, nz=L, periodic=(1, 1, 1), liquid_height=0.0, lubrication=0, **kw)
    return O.Oracle(p)


@pytest.mark.parametrize("e,r2", [(0.88, 3.0), (0.5, 5.0), (0.97, 3.0)])
def test_two_sphere_restitution(e, r2):
    """A head-on binary collision leaves the normal relative velocity reduced
    by the coefficient of restitution (closed form of the damped oscillator
    whose stiffness and damping are set from e and T_c)."""
    v, r1, Tc = 0.01, 3.0, 24.0
    o = _dry(restitution=e, collision_time=Tc)
    o.add_spheres([[10.0, 20, 20], [10.0 + r1 + r2 + 1.0, 20, 20]], [r1, r2])
    o.set(O.P_U, np.array([[v, 0, 0], [-v, 0, 0]]))
    U0 = o.get(O.P_U)
    o.step(int(1.0 / v + 3 * Tc + 20))
    U = o.get(O.P_U)
    assert abs((U[1, 0] - U[0, 0]) / (2 * v) - e) < 0.01 * e
    m = np.array([r1 ** 3, r2 ** 3])
    assert abs(m @ U[:, 0] - m @ U0[:, 0]) < 1e-15      # momentum


def test_sliding_sphere_ends_rolling_at_five_sevenths():
    """A sphere launched sliding on a wall with Coulomb friction ends rolling
    at 5/7 of its initial speed (angular momentum about the contact point)."""
    v0, r = 0.01, 3.0
    o = O.Oracle(O.OracleParams(nx=40, ny=16, nz=16, periodic=(1, 1, 0), g=(0, 0, -1e-3),
                                liquid_height=0.0, friction=0.5, collision_time=24.0, lubrication=0))
    o.add_spheres([[10.0, 8, r]], [r])
    o.set(O.P_U, np.array([[v0, 0, 0]]))
    o.step(1500)
    U = o.get(O.P_U)[0]
    Wy = o.get(O.P_W)[0, 1]
    assert abs(U[0] / v0 - 5 / 7) < 1e-3
    assert abs(Wy * r / v0 - 5 / 7) < 1e-3


def test_bedload_rate_eq1():
    o = _dry(L=20)
    rng = np.random.default_rng(1)
    X = rng.uniform(4, 16, (5, 3))
    X[:, 2] = np.arange(5) * 3.0 + 2.0
    R = np.full(5, 1.0)
    o.add_spheres(X, R)
    U = rng.normal(0, 1e-3, (5, 3))
    o.set(O.P_U, U)
    qb = o.reduce()[6]
    assert abs(qb - np.sum(U[:, 0] * 4 / 3 * np.pi) / (20 * 20)) < 1e-18


# ---------------------------------------------------------------- lubrication
# Reading R-23 of Section 2.2: below the resolved gap h_c = 2/3 cell the DEM
# adds 6 pi mu R^2 (1/h - 1/h_c) against the approach speed and
# 6 pi mu R (8/15) ln(h_c / h) against the sliding speed (R = r at a wall).

def _lub_box(omega=1.9):
    return O.Oracle(O.OracleParams(nx=16, ny=16, nz=16, periodic=(1, 1, 0), omega=omega, g=(0, 0, 0),
                                   liquid_height=0.0))


def test_lubrication_slows_an_approach_to_the_wall_as_the_closed_form():
    """A sphere entering the lubrication range of the floor at speed s0: with
    m ds/dt = -zeta(h) s and dh/dt = -s, s(h) = s0 + (6 pi mu r^2 / m)
    (ln(h / h0) - (h - h0) / h_c), h0 = h_c; the sub-stepped DEM follows it
    to 1% down to a gap of 0.15."""
    r, s0, hc = 3.0, 0.01, 2.0 / 3.0
    o = _lub_box()
    o.add_spheres([[8.0, 8.0, r + hc]], [r])
    o.set(O.P_U, np.array([[0.0, 0.0, -s0]]))
    mu = (1 / 1.9 - 0.5) / 3
    m = 2.55 * 4 / 3 * np.pi * r ** 3
    k = 6 * np.pi * mu * r * r / m
    checked = 0
    for _ in range(200):
        o.step(1)
        h = o.get(O.P_X)[0, 2] - r
        s = -o.get(O.P_U)[0, 2]
        if h < 0.15:
            break
        want = s0 + k * (np.log(h / hc) - (h - hc) / hc)
        assert abs(s / want - 1) < 0.01, (h, s, want)
        checked += 1
    assert checked > 50 and s < 0.8 * s0


def test_lubrication_damps_sliding_at_a_fixed_gap_exponentially():
    """A sphere sliding parallel to the floor at a gap of 0.2 with no normal
    motion: the sliding speed v = U_x - r Omega_y decays as
    exp(-c_t (1/m + r^2/I) t) = exp(-3.5 c_t t / m), with
    c_t = 6 pi mu r (8/15) ln(h_c / h); the gap does not change."""
    r, v0, h, hc = 3.0, 0.01, 0.2, 2.0 / 3.0
    o = _lub_box()
    o.add_spheres([[8.0, 8.0, r + h]], [r])
    o.set(O.P_U, np.array([[v0, 0.0, 0.0]]))
    mu = (1 / 1.9 - 0.5) / 3
    m = 2.55 * 4 / 3 * np.pi * r ** 3
    ct = 6 * np.pi * mu * r * (8 / 15) * np.log(hc / h)
    o.step(300)
    U = o.get(O.P_U)[0]
    W = o.get(O.P_W)[0]
    v = U[0] - r * W[1]
    assert v / v0 == pytest.approx(np.exp(-3.5 * ct * 300 / m), rel=1e-3)
    assert abs(o.get(O.P_X)[0, 2] - (r + h)) < 1e-12 and abs(U[2]) < 1e-15
    # the angular momentum about the contact line is kept: m U_x + (I / r) Omega_y
    assert m * U[0] + 0.4 * m * r * W[1] == pytest.approx(m * v0, rel=1e-12)
