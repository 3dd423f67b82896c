"""Hand-computed pins of the oracle's conversion heuristics (Section 2.1,
readings R-7 and R-8) and of the re-mapping of uncovered cells (Section 2.2,
reading R-11). The paper gives no formula for any of them, so the values
below are worked out by hand from the readings:

- the excess-mass shares of a converting cell for a known normal (weights
  max(0, +n.c) when it fills, max(0, -n.c) when it empties, evenly when all
  vanish, into the pool without receivers);
- the density and velocity a new interface cell starts from (means over the
  liquid and interface cells of its block, nothing else);
- the state of an uncovered cell (f_eq of the mean neighbour density and of
  the particle's surface velocity U + Omega x d at the cell centre);
- whole steps on a flat layer at rest (uniform density 1, no gravity), where
  streaming, mass exchange and collision change nothing, so the outcome of
  a conversion, and of spreading the pool, is known in closed form.

A sign slip in the weights, a wrong neighbour set or a wrong surface
velocity changes one of these numbers; mass conservation alone would not
notice."""
import numpy as np
import pytest

import oracle as O


def q(cx, cy, cz):
    return (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1)


def _receivers(*dirs):
    r = np.zeros(27, np.uint8)
    for d in dirs:
        r[q(*d)] = 1
    return r


def test_excess_of_a_filled_cell_follows_the_normal():
    n = (0.6, 0.0, 0.8)
    rec = _receivers((1, 0, 0), (0, 0, 1), (1, 0, 1), (-1, 0, 0), (0, 1, 0))
    pool, sh = O.excess_shares(True, 0.3, n, rec)
    assert not pool
    # weights 0.6, 0.8, 1.4, 0, 0 (sum 2.8): 0.3 * w / 2.8
    want = np.zeros(27)
    want[q(1, 0, 0)] = 9 / 140
    want[q(0, 0, 1)] = 3 / 35
    want[q(1, 0, 1)] = 0.15
    assert np.allclose(sh, want, rtol=0, atol=1e-15)
    assert abs(sh.sum() - 0.3) < 1e-15


def test_excess_of_an_emptied_cell_goes_against_the_normal():
    n = (0.6, 0.0, 0.8)
    rec = _receivers((-1, 0, 0), (0, 0, -1), (-1, 0, -1), (1, 0, 0), (0, -1, 0))
    pool, sh = O.excess_shares(False, -0.07, n, rec)
    assert not pool
    # weights max(0, -n.c): 0.6, 0.8, 1.4, 0, 0 (sum 2.8)
    want = np.zeros(27)
    want[q(-1, 0, 0)] = -0.015
    want[q(0, 0, -1)] = -0.02
    want[q(-1, 0, -1)] = -0.035
    assert np.allclose(sh, want, rtol=0, atol=1e-15)


def test_excess_is_even_when_every_weight_vanishes_or_when_asked():
    rec = _receivers((1, 0, 0), (0, 1, -1), (-1, -1, 0))
    pool, sh = O.excess_shares(True, 0.3, (0.0, 0.0, 1.0), rec)     # n.c = 0, -1, 0
    assert not pool
    assert np.allclose(sh[rec == 1], 0.1, rtol=0, atol=1e-15) and np.all(sh[rec == 0] == 0)
    rec = _receivers((1, 0, 0), (0, 0, 1), (1, 0, 1), (-1, 0, 0), (0, 1, 0))
    pool, sh = O.excess_shares(True, 0.3, (0.6, 0.0, 0.8), rec, even=True)
    assert np.allclose(sh[rec == 1], 0.06, rtol=0, atol=1e-15)


def test_excess_without_receivers_goes_to_the_pool():
    pool, sh = O.excess_shares(True, 0.3, (0.0, 0.0, 1.0), np.zeros(27, np.uint8))
    assert pool and np.all(sh == 0)
    rec = np.zeros(27, np.uint8)
    rec[13] = 1                        # the cell itself never receives
    pool, sh = O.excess_shares(False, 0.2, (0.0, 0.0, 1.0), rec)
    assert pool and np.all(sh == 0)


def test_new_interface_cell_averages_liquid_and_interface_neighbours_only():
    t = np.full(27, O.GAS, np.uint8)
    rho = np.zeros(27)
    u = np.zeros((27, 3))
    t[13], rho[13], u[13] = O.INTERFACE, 5.0, (1.0, 1.0, 1.0)          # the cell itself: excluded
    t[q(1, 0, 0)], rho[q(1, 0, 0)], u[q(1, 0, 0)] = O.LIQUID, 1.02, (0.01, 0.0, 0.0)
    t[q(0, 0, -1)], rho[q(0, 0, -1)], u[q(0, 0, -1)] = O.INTERFACE, 0.99, (0.0, 0.02, 0.0)
    t[q(-1, 1, -1)], rho[q(-1, 1, -1)], u[q(-1, 1, -1)] = O.LIQUID, 1.05, (0.0, 0.0, -0.03)
    rho[q(0, 0, 1)], u[q(0, 0, 1)] = 7.0, (0.5, 0.5, 0.5)               # gas: excluded
    t[q(1, 1, 1)], rho[q(1, 1, 1)] = O.SOLID, 9.0                       # solid: excluded
    t[q(0, -1, 0)], rho[q(0, -1, 0)] = O.WALL, 11.0                     # beyond a wall: excluded
    cnt, rb, ub = O.new_interface_mean(t, rho, u)
    assert cnt == 3
    assert abs(rb - 1.02) < 1e-15
    assert np.allclose(ub, (0.01 / 3, 0.02 / 3, -0.01), rtol=0, atol=1e-17)


def test_uncovered_cell_takes_the_particle_surface_velocity():
    t = np.full(27, O.SOLID, np.uint8)
    rho = np.full(27, 3.0)
    t[q(0, 0, -1)] = O.WALL
    # no liquid or interface neighbour: the cell turns gas
    t[q(0, 0, 1)] = O.GAS
    typ, *_ = O.uncovered_state(t, rho, (0.01, 0, 0), (0, 0, 0.002), (1.5, -0.5, 0.25))
    assert typ == O.GAS
    # two fluid neighbours (rho 1.02 and 0.98) and no gas: liquid, rho 1
    t[q(0, 0, 1)] = O.SOLID
    t[q(1, 0, 0)], rho[q(1, 0, 0)] = O.LIQUID, 1.02
    t[q(-1, 0, 0)], rho[q(-1, 0, 0)] = O.INTERFACE, 0.98
    typ, f, rb, ub, m = O.uncovered_state(t, rho, (0.01, 0, 0), (0, 0, 0.002), (1.5, -0.5, 0.25))
    assert typ == O.LIQUID and abs(rb - 1.0) < 1e-15 and abs(m - 1.0) < 1e-15
    # Omega x d = (0 * 0.25 - 0.002 * -0.5, 0.002 * 1.5 - 0 * 0.25, 0) = (0.001, 0.003, 0)
    assert np.allclose(ub, (0.011, 0.003, 0.0), rtol=0, atol=1e-17)
    assert np.allclose(f, O.feq(1.0, (0.011, 0.003, 0.0)), rtol=0, atol=1e-16)
    # every component of the cross product: W = (1, -2, 3) 1e-3, d = (0.5, 1, -1.5)
    typ, f, rb, ub, m = O.uncovered_state(t, rho, (0, 0, 0), (0.001, -0.002, 0.003), (0.5, 1.0, -1.5))
    assert np.allclose(ub, (0.0, 0.003, 0.002), rtol=0, atol=1e-17)
    # a gas neighbour: interface with mass 0 (its mass comes in from the pool)
    t[q(0, 1, 1)] = O.GAS
    typ, f, rb, ub, m = O.uncovered_state(t, rho, (0.01, 0, 0), (0, 0, 0.002), (1.5, -0.5, 0.25))
    assert typ == O.INTERFACE and m == 0.0 and abs(rb - 1.0) < 1e-15


def _flat_layer(nx=8, ny=8, nz=8, H=4.5):
    """Liquid in z < 4, interface layer z = 4 (fill 0.5), gas above; density
    1 everywhere, no gravity: a fixed point of streaming, mass exchange and
    collision."""
    o = O.Oracle(O.OracleParams(nx=nx, ny=ny, nz=nz, periodic=(1, 1, 0), omega=1.0, g=(0, 0, 0), rho_gas=1.0,
                                liquid_height=H))
    t = o.get(O.F_TYPE)
    assert (t[:4] == O.LIQUID).all() and (t[4] == O.INTERFACE).all() and (t[5:] == O.GAS).all()
    assert np.allclose(o.get(O.F_PHI)[4], 0.5)
    return o


def test_whole_step_filled_cell_gives_its_excess_to_the_new_cells_above():
    o = _flat_layer()
    m = o.get(O.F_MASS)
    m[4, 3, 3] = 1.5                    # fill level 1.5 > 1 + eps: turns liquid
    o.set(O.F_MASS, m)
    m0 = o.reduce()[0]
    o.step(1)
    t, m = o.get(O.F_TYPE), o.get(O.F_MASS)
    assert t[4, 3, 3] == O.LIQUID and abs(m[4, 3, 3] - 1.0) < 1e-12
    # its normal is (0, 0, 1): the excess 0.5 goes to the 9 gas cells above,
    # which turn interface, weight 1 each; the layer (n.c = 0) gets nothing
    new = np.zeros_like(t, bool)
    new[5, 2:5, 2:5] = True
    assert (t[new] == O.INTERFACE).all() and (t[5][~new[5]] == O.GAS).all()
    assert np.allclose(m[new], 0.5 / 9, rtol=0, atol=1e-12)
    layer = t[4] == O.INTERFACE
    assert layer.sum() == 63 and np.allclose(m[4][layer], 0.5, rtol=0, atol=1e-12)
    assert o.pool == 0.0 and abs(o.reduce()[0] - m0) < 1e-12
    # the new cells start from the mean of their fluid neighbours: rho 1, u 0
    f = o.get(O.F_PDF)
    assert np.allclose(f[:, new], O.feq(1.0, (0, 0, 0))[:, None], rtol=0, atol=1e-14)


def test_whole_step_emptied_cell_takes_its_deficit_from_the_liquid_below():
    o = _flat_layer()
    m = o.get(O.F_MASS)
    m[4, 3, 3] = -0.05                  # fill level below -eps: turns gas
    o.set(O.F_MASS, m)
    o.step(1)
    t, m = o.get(O.F_TYPE), o.get(O.F_MASS)
    assert t[4, 3, 3] == O.GAS and m[4, 3, 3] == 0.0
    # the 9 liquid cells below turn interface with m = rho = 1, and receive
    # the excess -0.05 with weight max(0, -n.c) = 1 each
    emp = np.zeros_like(t, bool)
    emp[3, 2:5, 2:5] = True
    assert (t[emp] == O.INTERFACE).all()
    assert np.allclose(m[emp], 1.0 - 0.05 / 9, rtol=0, atol=1e-12)
    layer = (t[4] == O.INTERFACE)
    assert layer.sum() == 63 and np.allclose(m[4][layer], 0.5, rtol=0, atol=1e-12)


def test_whole_step_film_without_liquid_empties_into_the_pool():
    """A film of interface cells (fill 0.5) on the floor with gas above: no
    cell has a liquid neighbour, so all turn gas, none can receive, and the
    whole mass goes to the pool, which stays there (no interface cell is
    left to spread it over)."""
    o = O.Oracle(O.OracleParams(nx=6, ny=6, nz=4, periodic=(1, 1, 0), omega=1.0, g=(0, 0, 0), rho_gas=1.0,
                                liquid_height=0.5))
    assert (o.get(O.F_TYPE)[0] == O.INTERFACE).all()
    o.step(1)
    assert (o.get(O.F_TYPE) == O.GAS).all()
    assert abs(o.pool - 0.5 * 36) < 1e-12
    assert abs(o.reduce()[0] - 18.0) < 1e-12


def test_whole_step_pool_is_spread_evenly_over_the_interface_cells():
    o = _flat_layer()
    o.set_pool(0.3)
    o.step(1)
    t, m = o.get(O.F_TYPE), o.get(O.F_MASS)
    ifc = t == O.INTERFACE
    assert ifc.sum() == 64 and (t[:4] == O.LIQUID).all()
    assert np.allclose(m[ifc], 0.5 + 0.3 / 64, rtol=0, atol=1e-12)
    assert o.pool == 0.0
