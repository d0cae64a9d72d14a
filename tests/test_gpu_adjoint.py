"""The hand-written discrete adjoint (lbm_adjoint, through the C ABI) against
the FP64 reference gradient (autograd of the torch pull-form restatement),
against central differences of the FP64 C oracle, and its own invariants.

Objective: J = time-and-region mean of rho |u|^2 / 2 over steps 1..T.  Error
metric: max |dJ/dphi_gpu - dJ/dphi_ref| over the box divided by max
|dJ/dphi_ref| (the gradient spans orders of magnitude, so a pointwise relative
error is dominated by cells where it vanishes).  Tolerance 1e-3 for FP32
storage; J itself to 1e-5.
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, periodic_box_problem, pipe_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle
from oracle.torch_ref import TorchLBM

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3
TOL_J = 1e-5


def grad_err(g, ref):
    return np.abs(g - ref).max() / np.abs(ref).max()


def gpu_adjoint(lbm, prob, T, K, region, storage="f32"):
    sim = lbm.Simulation(prob, storage=storage)
    try:
        J, g = sim.adjoint(T, K, region)
        return J, g.cpu().numpy()
    finally:
        sim.close()


def check_against_reference(lbm, prob, T, K, region, storage="f32", tol=TOL_GRAD, tol_j=TOL_J):
    Jr, gr = TorchLBM(prob).gradient(prob.phi, T, region)
    J, g = gpu_adjoint(lbm, prob, T, K, region, storage)
    assert abs(J - Jr) <= tol_j * abs(Jr), (J, Jr)
    e = grad_err(g, gr)
    assert e <= tol, e
    assert np.all(g[prob.flags == 0] == 0.0)
    return g, gr


@pytest.mark.parametrize("q", [27, 19])
def test_small_aneurysm_matches_reference_gradient(lbm, q):
    """24^3 aneurysm with the random porous sac: Zou-He inlet, extrapolation
    outlet, bounce-back walls, Kozeny-Carman drag, Carreau-Yasuda; T = 40,
    checkpoint every 8 steps."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=50.0)
    check_against_reference(lbm, prob, 40, 8, prob.region)


def test_periodic_random_porosity_matches_reference_gradient(lbm):
    """Fully periodic box (every cell on the wrapping path next to a face),
    random porosity everywhere, solid obstacles, body force, constant
    permeability drag with Forchheimer term."""
    rng = np.random.default_rng(3)
    shape = (8, 10, 12)
    phi = (0.7 + 0.3 * rng.random(shape)).astype(np.float32)
    prob = periodic_box_problem(12, 10, 8, q=27, phi=phi, body_force=(2e-5, -1e-5, 5e-6), obstacles=6, seed=2,
                                rheology=lattice_rheology(0.08, 0.01, 50.0, 0.4, 2.0), k_const=0.5,
                                forchheimer=1, d_p=1.0)
    prob.phi[prob.flags == 0] = 1.0
    region = np.zeros(shape, np.uint8)
    region[2:6, 3:8, 2:9] = 1
    check_against_reference(lbm, prob, 25, 25, region)


def test_pipe_body_force_kozeny_carman_matches_reference_gradient(lbm):
    """32x32x64 pipe (periodic along z, D3Q19) with the porous plug and body
    force; region = a slab downstream of the plug."""
    prob = pipe_problem(q=19)
    region = np.zeros(prob.flags.shape, np.uint8)
    region[40:48] = 1
    check_against_reference(lbm, prob, 12, 5, region)


def test_gradient_is_independent_of_the_checkpoint_interval(lbm):
    """Replays reproduce the forward states bit for bit, so every K gives the
    same J and the same gradient."""
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    T = 23
    J0, g0 = gpu_adjoint(lbm, prob, T, T, prob.region)
    for K in (1, 4, 7, 100):
        J, g = gpu_adjoint(lbm, prob, T, K, prob.region)
        assert J == J0
        assert np.array_equal(g, g0), K


def test_gradient_matches_oracle_finite_differences(lbm):
    """Central differences (eps = 1e-4) of the FP64 C oracle's objective at
    sac voxels with porosity strictly inside (0.6, 1)."""
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    T = 16
    J, g = gpu_adjoint(lbm, prob, T, 4, prob.region)
    J0 = Oracle(prob).run_objective(T, prob.region)
    assert abs(J - J0) <= TOL_J * abs(J0)
    rng = np.random.default_rng(1)
    cand = np.argwhere((prob.region > 0) & (prob.flags > 0) & (prob.phi < 0.99) & (prob.phi > 0.61))
    scale = np.abs(g).max()
    eps = 1e-4
    for z, y, x in cand[rng.choice(len(cand), 6, replace=False)]:
        ph = prob.phi.astype(np.float64).copy()
        ph[z, y, x] += eps
        jp = Oracle(prob, phi=ph).run_objective(T, prob.region)
        ph[z, y, x] -= 2 * eps
        jm = Oracle(prob, phi=ph).run_objective(T, prob.region)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - g[z, y, x]) <= TOL_GRAD * scale, (z, y, x, fd, g[z, y, x])


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
def test_reduced_precision_storage_gradient(lbm, storage):
    """With FP16 / BF16 deviation storage the forward trajectory carries the
    storage rounding, and the gradient inherits it: stated tolerances 1e-2
    (FP16) and 5e-2 (BF16) against the FP64 reference."""
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    tol = 1e-2 if storage == "f16dev" else 5e-2
    check_against_reference(lbm, prob, 40, 10, prob.region, storage, tol=tol, tol_j=tol)


def test_autograd_function(lbm):
    """sac_kinetic_energy is a torch function of phi whose backward is the
    adjoint."""
    import torch

    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    phi = torch.tensor(prob.phi, dtype=torch.float64, requires_grad=True)
    J = lbm.sac_kinetic_energy(prob, phi, 10, 3, prob.region)
    (2.0 * J).backward()
    J2, g = gpu_adjoint(lbm, prob, 10, 3, prob.region)
    assert float(J) == J2
    assert np.array_equal(phi.grad.numpy(), 2.0 * g)


def test_context_state_is_untouched(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    sim = lbm.Simulation(prob)
    sim.step(7)
    before = sim.save()
    sim.adjoint(9, 4, prob.region)
    assert sim.t == 7
    assert np.array_equal(sim.save(), before)
    sim.step(3)
    ref = lbm.Simulation(prob)
    ref.step(10)
    assert np.array_equal(sim.moments()["u"], ref.moments()["u"])


def test_adjoint_rejects_bad_arguments(lbm):
    import torch

    prob = aneurysm_problem(24, q=27, small=True)
    sim = lbm.Simulation(prob)
    assert lbm.lbm_adjoint_workspace_size(sim.ctx, 0, 4) == 0
    assert lbm.lbm_adjoint_workspace_size(sim.ctx, 4, 0) == 0
    with pytest.raises(lbm.LBMError) as e:
        sim.adjoint(5, 2, np.zeros(prob.flags.shape, np.uint8))  # region without fluid cells
    assert e.value.status == lbm.LBM_EINVAL
    nbytes = lbm.lbm_adjoint_workspace_size(sim.ctx, 5, 2)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    grad = torch.empty(prob.flags.shape, dtype=torch.float64, device="cuda")
    reg = np.ascontiguousarray(prob.region, dtype=np.uint8)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_adjoint(sim.ctx, 5, 2, 0, reg.ctypes.data, 0, ws.data_ptr(), nbytes - 256, grad.data_ptr())
    assert e.value.status == lbm.LBM_ENOMEM
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_adjoint(sim.ctx, 5, 2, 0, reg.ctypes.data, 0, ws.data_ptr() + 8, nbytes - 256, grad.data_ptr())
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:  # no such objective
        lbm.lbm_adjoint(sim.ctx, 5, 2, 2, reg.ctypes.data, 0, ws.data_ptr(), nbytes, grad.data_ptr())
    assert e.value.status == lbm.LBM_EINVAL


@pytest.mark.parametrize("q", [27, 19])
def test_wall_shear_objective_matches_reference_gradient(lbm, q):
    """Objective 1: time-and-sac-wall mean of the wall-shear-stress proxy,
    against autograd of the torch restatement (whose proxy equals the C
    oracle's, see test_oracle_crosscheck)."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=50.0)
    T = 40
    Jr, gr = TorchLBM(prob).gradient(prob.phi, T, prob.region, kind="wss")
    sim = lbm.Simulation(prob)
    J, g = sim.adjoint(T, 8, prob.region, "wss")
    g = g.cpu().numpy()
    assert abs(J - Jr) <= TOL_J * abs(Jr), (J, Jr)
    e = grad_err(g, gr)
    assert e <= TOL_GRAD, e


def test_wall_shear_objective_independent_of_checkpoint_interval(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    sim = lbm.Simulation(prob)
    J0, g0 = sim.adjoint(17, 17, prob.region, "wss")
    J1, g1 = sim.adjoint(17, 3, prob.region, "wss")
    assert J0 == J1 and np.array_equal(g0.cpu().numpy(), g1.cpu().numpy())


@pytest.mark.parametrize("objective", ["ke", "wss"])
def test_anisotropic_permeability_matches_reference_gradient(lbm, objective):
    """The adjoint through the fixed-point velocity solve of an anisotropic
    permeability (lbm_set_anisotropy): implicit-function reverse of the
    converged velocity against autograd of the torch restatement, which
    unrolls the same iteration to FP64 convergence (measured: 7e-7)."""
    from lbm_inputs import coil_shape_tensor

    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=50.0)
    S = coil_shape_tensor(prob.flags.shape, ratio=4.0, seed=1)
    T, K = 30, 6
    Jr, gr = TorchLBM(prob, shape_tensor=S).gradient(prob.phi, T, prob.region, kind=objective)
    sim = lbm.Simulation(prob)
    try:
        sim.set_anisotropy(S)
        J, g = sim.adjoint(T, K, prob.region, objective=objective)
        g = g.cpu().numpy()
    finally:
        sim.close()
    assert abs(J - Jr) <= TOL_J * abs(Jr), (J, Jr)
    assert grad_err(g, gr) <= TOL_GRAD, grad_err(g, gr)
    # the anisotropy changes the gradient measurably
    _, gi = TorchLBM(prob).gradient(prob.phi, T, prob.region, kind=objective)
    assert grad_err(gi, gr) > 5 * TOL_GRAD
