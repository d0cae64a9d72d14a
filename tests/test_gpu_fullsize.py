"""Parity at the full sizes of the workloads, against the FP64 oracle run to
the same time (minutes of host time; marked slow).

* 256^3 aneurysm, FP32 storage, 2000 steps: velocity, shear rate, density, mass drift.
* 384^3 aneurysm, FP32 / FP16 / BF16 deviation storage, 1000 steps (FP32 also
  at 200 steps): velocity, shear rate, density, mass drift.
* 128^3 adjoint, T = 500, K = 50: J and d J / d phi at 16 random sac voxels
  (rng seed 1) against central differences (eps = 1e-4) of the FP64 oracle's J.
* 24^3 adjoint, T = 100, K = 10, against the FP64 autograd gradient.

Error metric as in test_gpu_parity.py: max over fluid cells of |a - b| over
max |b|.  Stated bounds: FP32 1e-5 at 200 steps (the FP32 target); after 1000 or
2000 steps of the pulsatile Carreau-Yasuda flow the FP32 rounding of the
stored state accumulates to about 1.2e-5 (measured), bound 2e-5.  FP16
deviations 1e-3 (velocity) and 2e-3 (shear rate); BF16 (8-bit significand)
1e-2 and 2e-2.  Mass drift: the GPU's relative change of total mass agrees
with the oracle's within 1e-5 (FP32, FP16) and 1e-4 (BF16).  Adjoint: relative
gradient error 1e-3 per voxel.
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem
from oracle.oracle import Oracle
from oracle.torch_ref import TorchLBM

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def field_errors(g, r, fluid):
    den = np.abs(r["u"][:, fluid]).max()
    gd = np.abs(r["gdot"][fluid]).max()
    return dict(u=np.abs(g["u"][:, fluid].astype(np.float64) - r["u"][:, fluid]).max() / den,
                gdot=np.abs(g["gdot"][fluid].astype(np.float64) - r["gdot"][fluid]).max() / gd,
                rho=np.abs(g["rho"][fluid].astype(np.float64) - r["rho"][fluid]).max())


def test_aneurysm256_fp32_2000_steps(lbm):
    prob = aneurysm_problem(256, q=27)
    fluid = prob.flags > 0
    o = Oracle(prob)
    m0 = o.diag()[0]
    o.step(2000)
    r = o.moments()
    drift_ref = (o.diag()[0] - m0) / m0
    o.close()
    sim = lbm.Simulation(prob)
    d0 = sim.diag()[0]
    sim.step(2000)
    e = field_errors(sim.moments(), r, fluid)
    drift = (sim.diag()[0] - d0) / d0
    assert e["u"] <= 2e-5 and e["gdot"] <= 2e-5 and e["rho"] <= 1e-5, e
    assert abs(drift - drift_ref) <= 1e-5, (drift, drift_ref)


def test_aneurysm384_storage_types_1000_steps(lbm):
    prob = aneurysm_problem(384, q=27)
    fluid = prob.flags > 0
    o = Oracle(prob)
    m0 = o.diag()[0]
    o.step(200)
    r200 = o.moments()
    o.step(800)
    r = o.moments()
    drift_ref = (o.diag()[0] - m0) / m0
    o.close()
    bounds = {"f32": (2e-5, 2e-5, 1e-5), "f16dev": (1e-3, 2e-3, 1e-5), "bf16dev": (1e-2, 2e-2, 1e-4)}
    for storage, (bu, bg, bm) in bounds.items():
        sim = lbm.Simulation(prob, storage=storage)
        d0 = sim.diag()[0]
        sim.step(200)
        if storage == "f32":
            e200 = field_errors(sim.moments(), r200, fluid)
            assert e200["u"] <= 1e-5 and e200["gdot"] <= 1e-5, e200
        sim.step(800)
        e = field_errors(sim.moments(), r, fluid)
        drift = (sim.diag()[0] - d0) / d0
        sim.close()
        assert e["u"] <= bu and e["gdot"] <= bg, (storage, e)
        assert abs(drift - drift_ref) <= bm, (storage, drift, drift_ref)


def test_adjoint128_against_oracle_finite_differences(lbm):
    prob = aneurysm_problem(128, q=27)
    T, K = 500, 50
    sim = lbm.Simulation(prob)
    J, g = sim.adjoint(T, K, prob.region)
    g = g.cpu().numpy()
    sim.close()
    J0 = Oracle(prob).run_objective(T, prob.region)
    assert abs(J - J0) <= 1e-4 * abs(J0), (J, J0)
    rng = np.random.default_rng(1)
    cand = np.argwhere((prob.region > 0) & (prob.flags > 0) & (prob.phi < 0.99) & (prob.phi > 0.61))
    eps = 1e-4
    for z, y, x in cand[rng.choice(len(cand), 16, replace=False)]:
        ph = prob.phi.astype(np.float64).copy()
        ph[z, y, x] += eps
        jp = Oracle(prob, phi=ph).run_objective(T, prob.region)
        ph[z, y, x] -= 2 * eps
        jm = Oracle(prob, phi=ph).run_objective(T, prob.region)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - g[z, y, x]) <= 1e-3 * abs(fd), (z, y, x, fd, g[z, y, x])


def test_adjoint24_T100_K10_against_reference_gradient(lbm):
    prob = aneurysm_problem(24, q=27, small=True)
    Jr, gr = TorchLBM(prob).gradient(prob.phi, 100, prob.region)
    sim = lbm.Simulation(prob)
    J, g = sim.adjoint(100, 10, prob.region)
    g = g.cpu().numpy()
    assert abs(J - Jr) <= 1e-5 * abs(Jr)
    assert np.abs(g - gr).max() <= 1e-3 * np.abs(gr).max()
