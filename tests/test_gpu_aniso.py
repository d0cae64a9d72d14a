"""The anisotropic velocity solve (lbm_set_anisotropy, the fixed-point
iteration of the Sec. 3 remark) against the FP64 oracle.

Error metric as in test_gpu_parity.py: max over fluid cells of |a - b| over
max |b|.  Bounds: velocity 1e-5 and shear rate 1e-4 with FP32 storage, 1e-3 /
2e-3 with FP16 deviations, 1e-2 / 2e-2 with BF16 (as for the isotropic path); the identity shape tensor reproduces the explicit isotropic
GPU solution within 1e-6 (the same kernels up to the FP32 solve); the uniform
periodic medium reaches the exact Darcy-Forchheimer fixed point within 1e-5.
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, coil_shape_tensor, periodic_box_problem, pipe_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu


def rel_err(a, b, fluid):
    return np.abs(a[..., fluid].astype(np.float64) - b[..., fluid]).max() / np.abs(b[..., fluid]).max()


@pytest.mark.parametrize("q,storage", [(19, "f32"), (27, "f32"), (27, "f16dev"), (27, "bf16dev")])
def test_aneurysm_against_oracle(lbm, q, storage):
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=100.0)
    S = coil_shape_tensor(prob.flags.shape, ratio=4.0, seed=1)
    sim = lbm.Simulation(prob, storage=storage)
    sim.set_anisotropy(S)
    sim.step(200)
    g = sim.moments()
    o = Oracle(prob, shape_tensor=S)
    o.step(200)
    r = o.moments()
    fluid = prob.flags > 0
    eu, eg = rel_err(g["u"], r["u"], fluid), rel_err(g["gdot"], r["gdot"], fluid)
    bu, bg = {"f32": (1e-5, 1e-4), "f16dev": (1e-3, 2e-3), "bf16dev": (1e-2, 2e-2)}[storage]
    assert eu <= bu and eg <= bg, (eu, eg)
    # the anisotropy changes the flow measurably
    iso = Oracle(prob)
    iso.step(200)
    assert rel_err(iso.moments()["u"], r["u"], fluid) > 1e-3


def test_pipe_with_periodic_faces_and_wall_shear(lbm):
    """General-path cells (periodic faces) inside the porous plug, and the
    wall-shear-stress proxy with the anisotropic solve."""
    prob = pipe_problem(q=19)
    S = coil_shape_tensor(prob.flags.shape, ratio=0.3, seed=2)
    sim = lbm.Simulation(prob)
    sim.set_anisotropy(S)
    sim.step(200)
    o = Oracle(prob, shape_tensor=S)
    o.step(200)
    fluid = prob.flags > 0
    assert rel_err(sim.moments()["u"], o.moments()["u"], fluid) <= 1e-5
    w, wr = sim.wall_shear().astype(np.float64), o.wall_shear()
    assert np.abs(w - wr).max() <= 1e-4 * np.abs(wr).max()


def test_identity_shape_tensor_matches_the_explicit_path(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    S = np.zeros((6,) + prob.flags.shape, np.float32)
    S[:3] = 1.0
    a = lbm.Simulation(prob)
    b = lbm.Simulation(prob)
    b.set_anisotropy(S)
    a.step(200)
    b.step(200)
    fluid = prob.flags > 0
    ua, ub = a.moments()["u"], b.moments()["u"]
    assert np.abs(ua[:, fluid] - ub[:, fluid]).max() <= 1e-6 * np.abs(ua[:, fluid]).max()
    b.set_anisotropy(None)  # back to the explicit path
    b.step(1)


def test_uniform_medium_fixed_point(lbm):
    rng = np.random.default_rng(9)
    R, rr = np.linalg.qr(rng.standard_normal((3, 3)))
    R = R * np.sign(np.diag(rr))
    lam = np.array([0.25, 1.0, 4.0])
    Sm = R @ np.diag(lam) @ R.T
    Sh = R @ np.diag(np.sqrt(lam)) @ R.T
    rheo = lattice_rheology(0.1, 0.02, 20.0, 0.5, 2.0)
    phi, d, g = 0.7, 3.0, np.array([4e-3, 2e-3, -1e-3])
    prob = periodic_box_problem(4, 3, 5, q=27, phi_value=phi, rheology=rheo, body_force=tuple(g), d_p=d)
    comp = np.array([Sm[0, 0], Sm[1, 1], Sm[2, 2], Sm[0, 1], Sm[0, 2], Sm[1, 2]])
    S = np.broadcast_to(comp[:, None, None, None], (6,) + prob.flags.shape).astype(np.float32)
    sim = lbm.Simulation(prob)
    sim.set_anisotropy(S)
    sim.step(4000)
    u = sim.moments()["u"][:, 1, 1, 1].astype(np.float64)
    ph = float(np.float32(phi))
    k = ph ** 3 * d * d / (150 * (1 - ph) ** 2)
    A = ph ** 2 * 0.1 * Sm / k
    B = ph ** 3 * 1.75 / np.sqrt(150 * ph ** 3) / np.sqrt(k) * Sh
    x = np.linalg.solve(A, g)
    for _ in range(50):
        n = np.linalg.norm(x)
        x = x - np.linalg.solve(A + n * B + np.outer(B @ x, x) / n, A @ x + n * (B @ x) - g)
    assert np.abs(u - x).max() <= 1e-5 * np.linalg.norm(x)


def test_errors(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob)
    bad = np.zeros((6,) + prob.flags.shape, np.float32)
    bad[:3] = 1.0
    bad[2][prob.phi < 1] = -1.0  # not positive definite where the medium is
    with pytest.raises(lbm.LBMError) as e:
        sim.set_anisotropy(bad)
    assert e.value.status == lbm.LBM_EINVAL
    S = np.zeros_like(bad)
    S[:3] = 1.0
    with pytest.raises(lbm.LBMError) as e:
        sim.set_anisotropy(S, max_iter=0)
    assert e.value.status == lbm.LBM_EINVAL
    sim.set_anisotropy(S)
    sim.set_anisotropy(None)  # back to the isotropic closure
    sim.step(1)
