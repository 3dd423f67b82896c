"""Oracle of the flow-rate control of Section 3.1: the streamwise body force
F_x is adjusted during the run so that the bulk liquid velocity holds a
prescribed value.

TEST INFRASTRUCTURE ONLY (tests). The paper states the goal, not the
controller, so the law is a reading: after every `interval` completed
steps, with U the fill-weighted bulk velocity sum(phi rho u_x) /
sum(phi rho) of the current state (the quantity the reductions report),

    g_x <- g_x + gain (U_target - U),

an integral controller on the body-force acceleration. The new g_x drives
the fluid and weighs the particles from the next step on. In a steady
laminar film of depth H it settles at g_x = 3 nu U_target / H^2 (the mean of
the half-Poiseuille profile (g_x / nu)(H z - z^2 / 2) over the depth).
"""
from __future__ import annotations

import numpy as np


def run_controlled(o, steps: int, target: float, gain: float, interval: int):
    """Advance the oracle `o` by `steps` steps under the controller; returns
    the (steps done, g_x, U) after every update."""
    hist = []
    done = 0
    g = list(o.params.g)
    while done + interval <= steps:
        o.step(interval)
        done += interval
        u = float(o.reduce()[4])
        g[0] = g[0] + gain * (target - u)
        o.set_gravity(g)
        hist.append((done, g[0], u))
    if done < steps:
        o.step(steps - done)
    return np.array(hist)
