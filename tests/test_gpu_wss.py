"""The wall-shear-stress proxy (lbm_wall_shear, through the C ABI) against the
FP64 oracle's (oracle_wss) and against the plane Poiseuille stress.

Error metric: max |tau_gpu - tau_ref| over the box divided by max |tau_ref|.
The proxy is built from the non-equilibrium second moment, like the shear
rate, so it takes the shear rate's bounds: 1e-4 for FP32 storage, 1e-2 for
FP16 deviation storage.
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, channel_problem, pipe_problem
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu


def wss_error(lbm, prob, steps, storage="f32"):
    sim = lbm.Simulation(prob, storage=storage)
    sim.step(steps)
    g = sim.wall_shear().astype(np.float64)
    o = Oracle(prob)
    o.step(steps)
    r = o.wall_shear()
    assert np.array_equal(g == 0.0, r == 0.0)  # the same wall cells
    return np.abs(g - r).max() / np.abs(r).max(), sim, g


@pytest.mark.parametrize("q", [19, 27])
def test_small_aneurysm_fp32(lbm, q):
    e, _, _ = wss_error(lbm, aneurysm_problem(24, q=q, small=True, u0=0.05, period=100.0), 200)
    assert e <= 1e-4, e


def test_small_aneurysm_fp16(lbm):
    e, _, _ = wss_error(lbm, aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0), 200, "f16dev")
    assert e <= 1e-2, e


def test_pipe_with_periodic_faces(lbm):
    """Walls of the porous-plug pipe, including the cells on its periodic faces
    (general path)."""
    e, _, _ = wss_error(lbm, pipe_problem(q=19), 200)
    assert e <= 1e-4, e


def test_plane_poiseuille_stress(lbm):
    ny, G, tau = 18, 1e-6, 0.8
    prob = channel_problem(ny, q=27, nu=(tau - 0.5) / 3.0, body_force=G)
    sim = lbm.Simulation(prob)
    sim.step(20000)
    w = sim.wall_shear().astype(np.float64)
    rho = sim.moments()["rho"].astype(np.float64)
    h = (ny - 2) / 2.0
    for y in (1, ny - 2):
        assert np.abs(w[:, y, :] - rho[:, y, :] * G * (h - 0.5)).max() <= 1e-4 * G * h
    assert np.all(w[:, 2:ny - 2, :] == 0.0)


def test_device_output_equals_host_output(lbm):
    prob = aneurysm_problem(24, q=19, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob)
    sim.step(50)
    assert np.array_equal(sim.wall_shear(), sim.wall_shear(on_device=True).cpu().numpy())
