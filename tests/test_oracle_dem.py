"""Pins of the oracle's DEM (Section 2.2: linear contact model parameterised
by the restitution coefficient, collision time, Poisson ratio and friction
coefficient) and of the bedload rate of Eq. (1)."""
import numpy as np
import pytest

import oracle as O


def _dry(L=40, **kw):
    p = O.OracleParams(nx=L, ny=L, nz=L, periodic=(1, 1, 1), liquid_height=0.0, **kw)
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
                                liquid_height=0.0, friction=0.5, collision_time=24.0))
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
