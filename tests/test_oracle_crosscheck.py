"""The two FP64 oracles (C push form, torch pull form) against each other, the
Zou-He inlet against its defining momentum identity, and the torch reference
gradient against central finite differences of the C oracle."""

import math

import numpy as np
import pytest
import torch

from lbm_inputs import aneurysm_problem, periodic_box_problem, pipe_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle
from oracle.torch_ref import TorchLBM


def _compare(prob, steps, shape_tensor=None):
    o = Oracle(prob, shape_tensor=shape_tensor)
    o.step(steps)
    m = o.moments()
    tl = TorchLBM(prob, shape_tensor=shape_tensor)
    phi = torch.tensor(prob.phi.astype(np.float64))
    f, om = tl.run(phi, steps)
    fl = tl.fields(f, om, phi)
    umax = max(np.abs(m["u"]).max(), 1e-30)
    assert np.abs(fl["u"].numpy() - m["u"]).max() < 1e-12 * umax + 1e-15  # f ~ w: absolute round-off of sum f c
    assert np.abs(fl["rho"].numpy() - m["rho"]).max() < 1e-13
    gmax = max(m["gdot"].max(), 1e-30)
    assert np.abs(fl["gdot"].numpy() - m["gdot"]).max() < 1e-10 * gmax
    assert np.abs(fl["omega"].numpy() - m["omega"]).max() < 1e-9


@pytest.mark.parametrize("q", [19, 27])
def test_c_and_torch_oracles_agree_on_small_aneurysm(q):
    """Porous sac, Carreau-Yasuda, pulsatile Zou-He inlet, extrapolation outlet."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=40.0)
    _compare(prob, 25)


def test_c_and_torch_oracles_agree_with_anisotropic_permeability():
    """The fixed-point velocity solve with a per-cell shape tensor: Gaussian
    elimination and an eigendecomposition square root in C + numpy against
    batched torch solves and torch's own eigendecomposition."""
    from lbm_inputs import coil_shape_tensor

    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=40.0)
    _compare(prob, 25, shape_tensor=coil_shape_tensor(prob.flags.shape, ratio=4.0, seed=1))


def test_c_and_torch_oracles_agree_on_pipe():
    _compare(pipe_problem(q=19), 15)


def test_c_and_torch_oracles_agree_periodic_random_porosity():
    rng = np.random.default_rng(3)
    phi = (0.65 + 0.35 * rng.random((5, 4, 6))).astype(np.float32)
    rheo = lattice_rheology(0.1, 0.01, 50.0, 0.4, 2.0)
    prob = periodic_box_problem(6, 4, 5, q=27, rheology=rheo, body_force=(2e-4, -1e-4, 5e-5),
                                obstacles=8, phi=phi, d_p=2.0)
    _compare(prob, 20)


@pytest.mark.parametrize("q", [19, 27])
def test_zou_he_momentum_identity(q):
    """After the inlet reconstruction (non-equilibrium bounce-back of the
    unknown populations, Sec. 4) every inlet cell carries rho = sum_i f_i (phi
    = 1), the normal momentum rho u_in.n of the Hagen-Poiseuille profile
    u_in = 2 v(t) (1 - r^2/R^2) n exactly, and the tangential momentum
    rho ub_t + N_t with N_t = sum_{c.n=0} (f - f^eq(rho, ub)) c_t, the residual
    of the populations that stream along the inlet plane (no tangential
    correction), from arbitrary (perturbed) incoming populations."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.04, amp=0.5, period=30.0)
    o = Oracle(prob)
    rng = np.random.default_rng(q)
    f, om = o.get_state()
    o.set_state(f * (1 + 0.1 * rng.standard_normal(f.shape)), om, 0)
    t = 7
    o.apply_boundaries(t)
    f, _ = o.get_state()
    c, w, _ = o.lattice()
    cells = o.cells()
    nx, ny, nz = prob.dims
    b = prob.bc
    v = b["u0"] * (1 + b["amp"] * math.sin(2 * math.pi * t / b["period"]))
    n_in = 0
    largest_residual = 0.0
    inplane = c[:, 2] == 0
    for k, idx in enumerate(cells):
        if prob.flags.reshape(-1)[idx] != 2:
            continue
        n_in += 1
        x, y = idx % nx, (idx // nx) % ny
        r2 = (x + 0.5 - b["inlet_center"][0]) ** 2 + (y + 0.5 - b["inlet_center"][1]) ** 2
        ub = np.array([0.0, 0.0, 2 * v * max(0.0, 1 - r2 / b["inlet_radius"] ** 2)])
        rho = f[k].sum()
        mom = f[k] @ c
        cu = c @ ub
        feq = w * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * ub @ ub)
        resid = ((f[k] - feq)[inplane, None] * c[inplane]).sum(0)
        assert abs(mom[2] - rho * ub[2]) < 1e-15
        assert np.abs(mom[:2] - resid[:2]).max() < 1e-15
        largest_residual = max(largest_residual, np.abs(resid[:2]).max())
    assert n_in > 20
    assert largest_residual > 1e-4  # the tangential residual is genuinely left in place


def test_reference_gradient_matches_finite_differences():
    """d J / d phi from torch autograd (pull form) against central differences
    (eps = 1e-4) of the C oracle's objective, J = time-and-sac mean of
    rho |u|^2 / 2, at sac voxels with porosity strictly inside (0.6, 1)."""
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    T = 16
    J, grad = TorchLBM(prob).gradient(prob.phi, T, prob.region)
    J0 = Oracle(prob).run_objective(T, prob.region)
    assert abs(J - J0) < 1e-12 * abs(J0)  # FP64 rounding of two summation orders (1.3e-13 seen)
    rng = np.random.default_rng(1)
    cand = np.argwhere((prob.region > 0) & (prob.flags > 0) & (prob.phi < 0.99) & (prob.phi > 0.61))
    scale = np.abs(grad).max()
    eps = 1e-4
    for z, y, x in cand[rng.choice(len(cand), 5, replace=False)]:
        ph = prob.phi.astype(np.float64).copy()
        ph[z, y, x] += eps
        jp = Oracle(prob, phi=ph).run_objective(T, prob.region)
        ph[z, y, x] -= 2 * eps
        jm = Oracle(prob, phi=ph).run_objective(T, prob.region)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - grad[z, y, x]) < 1e-4 * scale + 1e-6 * abs(fd)


@pytest.mark.parametrize("q", [19, 27])
def test_c_and_torch_wall_shear_agree(q):
    """The voxel wall-shear-stress proxy of the two FP64 restatements."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=100.0)
    tl = TorchLBM(prob)
    phi = torch.tensor(prob.phi.astype(np.float64))
    f, om = tl.run(phi, 30)
    wt = tl.wall_shear(f, om, phi).numpy()
    o = Oracle(prob)
    o.step(30)
    wo = o.wall_shear()
    assert np.array_equal(wt > 0, wo > 0)
    assert np.abs(wt - wo).max() <= 1e-12 * np.abs(wo).max()


def test_wall_shear_objective_gradient_matches_differences():
    """Autograd of the torch wall-shear objective against its own central
    differences (eps = 1e-5) at the two sac voxels of largest gradient, once
    the inflow has reached the sac wall (T = 30)."""
    prob = aneurysm_problem(24, q=19, small=True, u0=0.05, period=50.0)
    T = 30
    tl = TorchLBM(prob)
    J, grad = tl.gradient(prob.phi, T, prob.region, kind="wss")
    cand = np.argwhere((prob.region > 0) & (prob.flags > 0) & (prob.phi < 0.99) & (prob.phi > 0.61))
    order = np.argsort(-np.abs(grad[tuple(cand.T)]))
    scale = np.abs(grad).max()
    for z, y, x in cand[order[:2]]:
        vals = []
        for sgn in (1, -1):
            ph = prob.phi.astype(np.float64).copy()
            ph[z, y, x] += sgn * 1e-5
            vals.append(float(tl.objective(torch.tensor(ph), T, prob.region, checkpoint=False, kind="wss")))
        fd = (vals[0] - vals[1]) / 2e-5
        assert abs(fd - grad[z, y, x]) <= 1e-4 * scale, (fd, grad[z, y, x])


def test_anisotropic_reference_gradient_matches_finite_differences():
    """With a shape tensor: d J / d phi from autograd of the torch restatement
    (the fixed-point iteration unrolled to FP64 convergence) against central
    differences (eps = 1e-4) of the C oracle's objective, at sac voxels of the
    porous medium and at the largest-gradient voxel."""
    from lbm_inputs import coil_shape_tensor

    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    S = coil_shape_tensor(prob.flags.shape, ratio=4.0, seed=1)
    T = 16
    J, grad = TorchLBM(prob, shape_tensor=S).gradient(prob.phi, T, prob.region)
    J0 = Oracle(prob, shape_tensor=S).run_objective(T, prob.region)
    assert abs(J - J0) < 1e-12 * abs(J0)
    rng = np.random.default_rng(2)
    cand = np.argwhere((prob.region > 0) & (prob.flags > 0) & (prob.phi < 0.99) & (prob.phi > 0.61))
    pts = list(cand[rng.choice(len(cand), 4, replace=False)])
    big = np.unravel_index(np.argmax(np.abs(np.where(prob.phi < 0.99, grad, 0.0))), grad.shape)
    pts.append(np.array(big))
    scale = np.abs(grad).max()
    eps = 1e-4
    for z, y, x in pts:
        ph = prob.phi.astype(np.float64).copy()
        ph[z, y, x] += eps
        jp = Oracle(prob, phi=ph, shape_tensor=S).run_objective(T, prob.region)
        ph[z, y, x] -= 2 * eps
        jm = Oracle(prob, phi=ph, shape_tensor=S).run_objective(T, prob.region)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - grad[z, y, x]) < 1e-4 * scale + 1e-6 * abs(fd), (z, y, x, fd, grad[z, y, x])


def test_c_and_torch_wall_shear_agree_with_anisotropic_permeability():
    from lbm_inputs import coil_shape_tensor

    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    S = coil_shape_tensor(prob.flags.shape, ratio=4.0, seed=1)
    tl = TorchLBM(prob, shape_tensor=S)
    phi = torch.tensor(prob.phi.astype(np.float64))
    f, om = tl.run(phi, 30)
    wt = tl.wall_shear(f, om, phi).numpy()
    o = Oracle(prob, shape_tensor=S)
    o.step(30)
    wo = o.wall_shear()
    assert np.array_equal(wt > 0, wo > 0)
    assert np.abs(wt - wo).max() <= 1e-12 * np.abs(wo).max()
