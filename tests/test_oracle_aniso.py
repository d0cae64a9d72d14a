"""Pins of the oracle's anisotropic velocity solve (the fixed-point iteration
of the Sec. 3 remark, with K = k(phi) S^{-1} for a per-cell shape tensor S).

* S = Id reproduces the explicit isotropic solution of Sec. 3 (the iteration
  converges to the closed form) on a porous aneurysm, to round-off.
* Uniform medium, fully periodic, body force g: each step adds exactly
  rho (g + f(u)) of momentum, so the steady velocity solves
  g = phi^2 nu K^{-1} u + phi^3 C_F |u| K^{-1/2} u, solved here by Newton's
  method with K^{-1/2} built from the rotation that defines S (independent of
  the oracle's eigendecomposition).  The Forchheimer term is a few percent of
  the drag, so dropping it, a transposed tensor or a wrong square root fails.
* The square root of the shape tensor squares back to S and equals
  R diag(sqrt(l)) R^T for S = R diag(l) R^T.
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, periodic_box_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle, shape_tensor_sqrt


def rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def pack(M):
    return np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])


def test_shape_tensor_square_root():
    rng = np.random.default_rng(4)
    S, H = [], []
    for _ in range(20):
        R = rotation(rng)
        lam = rng.uniform(0.1, 10.0, 3)
        S.append(pack(R @ np.diag(lam) @ R.T))
        H.append(pack(R @ np.diag(np.sqrt(lam)) @ R.T))
    S = np.array(S).T.reshape(6, 4, 5, 1)
    got = shape_tensor_sqrt(S)
    assert np.abs(got - np.array(H).T.reshape(6, 4, 5, 1)).max() < 1e-13
    with pytest.raises(ValueError):
        shape_tensor_sqrt(np.stack([np.ones(3), -np.ones(3), np.ones(3), np.zeros(3), np.zeros(3), np.zeros(3)]))


@pytest.mark.parametrize("q", [19, 27])
def test_identity_shape_tensor_gives_the_explicit_solution(q):
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=100.0)
    iso = Oracle(prob)
    S = np.zeros((6,) + prob.flags.shape)
    S[:3] = 1.0
    ani = Oracle(prob, shape_tensor=S)
    iso.step(60)
    ani.step(60)
    a, b = iso.moments(), ani.moments()
    fluid = prob.flags > 0
    assert np.abs(a["u"][:, fluid] - b["u"][:, fluid]).max() <= 1e-12 * np.abs(a["u"][:, fluid]).max()
    assert np.abs(a["rho"] - b["rho"]).max() <= 1e-13
    assert (prob.phi[fluid] < 1).sum() > 100  # the porous sac takes the iteration


@pytest.mark.parametrize("q", [19, 27])
def test_uniform_anisotropic_darcy_forchheimer_fixed_point(q):
    rng = np.random.default_rng(9)
    R = rotation(rng)
    lam = np.array([0.25, 1.0, 4.0])
    S = R @ np.diag(lam) @ R.T
    Sh = R @ np.diag(np.sqrt(lam)) @ R.T
    rheo = lattice_rheology(0.1, 0.02, 20.0, 0.5, 2.0)
    phi_set, d = 0.7, 3.0
    g = np.array([4e-3, 2e-3, -1e-3])
    prob = periodic_box_problem(4, 3, 5, q=q, phi_value=phi_set, rheology=rheo, body_force=tuple(g), d_p=d)
    St = np.broadcast_to(pack(S)[:, None, None, None], (6,) + prob.flags.shape).copy()
    o = Oracle(prob, shape_tensor=St)
    o.step(4000)
    m = o.moments()
    u = m["u"][:, 1, 1, 1]
    phi = float(np.float32(phi_set))
    nu = 0.1
    k = phi ** 3 * d * d / (150 * (1 - phi) ** 2)
    cf = 1.75 / np.sqrt(150 * phi ** 3)
    A = phi ** 2 * nu * S / k
    b = phi ** 3 * cf / np.sqrt(k)
    B = b * Sh
    x = np.linalg.solve(A, g)
    for _ in range(50):  # Newton on A x + |x| B x - g = 0
        n = np.linalg.norm(x)
        r = A @ x + n * (B @ x) - g
        J = A + n * B + np.outer(B @ x, x) / n
        x = x - np.linalg.solve(J, r)
    assert np.linalg.norm(A @ x + np.linalg.norm(x) * (B @ x) - g) < 1e-17
    forch = np.linalg.norm(np.linalg.norm(x) * (B @ x)) / np.linalg.norm(g)
    assert forch > 0.02  # the Forchheimer share is not negligible
    assert np.abs(u - x).max() < 1e-11 * np.linalg.norm(x)
    cosang = u @ g / (np.linalg.norm(u) * np.linalg.norm(g))
    assert cosang < np.cos(np.radians(5.0))  # anisotropy turns the flow off the force
    assert np.ptp(m["u"][0]) < 1e-15
