"""Pins of the oracle's Laplace pressure (Section 2.1: the free-surface
boundary condition carries the gas pressure plus 2 sigma kappa, here
rho_gas + 6 sigma kappa in lattice density). A hand-built learned-normal
network reproduces the finite-difference normal of a flat layer exactly and
reports a constant curvature kappa0; without gravity the liquid then settles
at the density the boundary condition imposes, in closed form."""
import numpy as np
import pytest

import oracle as O

from helpers import py_network as _network


def _layer(sigma):
    # a flat layer in a box periodic in x and y, walls far from the surface
    return O.Oracle(O.OracleParams(nx=4, ny=4, nz=16, periodic=(1, 1, 0), omega=1.0, g=(0.0, 0.0, 0.0),
                                   liquid_height=8.4, sigma=sigma))


def _liquid_density(o):
    t = o.get(O.F_TYPE)
    return float(o.get(O.F_RHO)[t == O.LIQUID].mean())


def test_laplace_pressure_sets_the_liquid_density():
    sigma, kappa0 = 1e-3, 1.0 / 6.0                 # 6 sigma kappa0 = 1e-3
    o = _layer(sigma)
    o.set_mlp(_network(1.0 / 16.0, kappa0), bf16=False)
    t = o.get(O.F_TYPE)
    k = o.get(O.F_CURV)
    assert np.all(k[t == O.INTERFACE] == kappa0) and np.all(k[t != O.INTERFACE] == 0.0)
    o.step(3000)
    rho = _liquid_density(o)
    assert rho - 1.0 == pytest.approx(6 * sigma * kappa0, rel=1e-5)
    # total liquid mass is kept: the layer gives up the volume the density gained
    assert abs(o.reduce()[0] / (4 * 4 * 8.4) - 1.0) < 1e-12


def test_no_tension_without_curvature_or_sigma():
    # sigma = 0 with the network's curvature, and sigma > 0 with the
    # finite-difference normal (which carries no curvature): rho stays 1
    for sigma, net in ((0.0, _network(1.0 / 16.0, 1.0 / 6.0)), (1e-3, None)):
        o = _layer(sigma)
        if net is not None:
            o.set_mlp(net, bf16=False)
        o.step(600)
        assert abs(_liquid_density(o) - 1.0) < 1e-9
        assert np.all(o.get(O.F_CURV) == 0.0) == (net is None)
