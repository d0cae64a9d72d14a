"""Pins of the oracle's voxel wall-shear-stress proxy (oracle_wss).

In steady plane Poiseuille flow driven by a body force G per unit mass the
shear stress is linear across the channel, sigma_xy = -rho G (y - y_c), so at
the first fluid cell, half a cell from a half-way bounce-back wall, |tau| is
rho G (h - 1/2) for the half-width h.  The LBM reproduces that stress exactly
(the non-equilibrium second moment carries the viscous stress of a quadratic
profile without truncation error), for any relaxation rate, and whichever
tangential direction the flow takes.
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, channel_problem
from oracle.oracle import Oracle

TAU_EXACT = 0.5 + np.sqrt(3.0 / 16.0)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("tau", [TAU_EXACT, 0.8])
@pytest.mark.parametrize("axis", [0, 2])
def test_wall_shear_of_plane_poiseuille(q, tau, axis):
    ny, G = 18, 1e-6
    nu = (tau - 0.5) / 3.0
    prob = channel_problem(ny, q=q, nu=nu, body_force=G)
    force = [0.0, 0.0, 0.0]
    force[axis] = G
    prob.bc["body_force"] = tuple(force)
    o = Oracle(prob)
    o.step(20000)
    w = o.wall_shear()
    rho = o.moments()["rho"]
    h = (ny - 2) / 2.0
    for y in (1, ny - 2):
        expect = rho[:, y, :] * G * (h - 0.5)
        assert np.abs(w[:, y, :] - expect).max() <= 1e-9 * G * h
    assert np.all(w[:, 2:ny - 2, :] == 0.0)  # no wall links away from the walls
    assert np.all(w[:, [0, ny - 1], :] == 0.0)  # solid rows


def test_wall_shear_zero_off_the_wall_and_on_open_boundaries():
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    o = Oracle(prob)
    o.step(60)
    w = o.wall_shear()
    assert np.all(w[prob.flags == 0] == 0.0)
    assert np.all(w[prob.flags >= 2] == 0.0)  # inlet and outlet cells
    assert (w > 0).sum() > 100 and np.isfinite(w).all()
