"""Local identities of one collision of the FP64 oracle (Sec. 3), on random
admissible populations.  Each check uses a relation that is not the formula
the oracle evaluates, so that a dropped term, a wrong sign or a wrong index in
the oracle fails it."""

import numpy as np
import pytest

from lbm_inputs import periodic_box_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle

CS2 = 1.0 / 3.0


def _random_cell(o, rng, amp=0.05):
    f, _ = o.get_state()
    f0 = f[0] * (1.0 + amp * rng.standard_normal(o.q))
    return f0


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("forch", [0, 1])
def test_velocity_solves_implicit_definition(q, forch):
    """u must satisfy phi rho u = sum f c + F/2 with F = rho (g + f_d(u)):
    the explicit formula of Sec. 3 is the solution of this implicit definition."""
    rng = np.random.default_rng(q + 10 * forch)
    rheo = lattice_rheology(0.1, 0.01, 30.0, 0.4, 2.0)
    for phi in (0.62, 0.8, 0.97, 1.0):
        prob = periodic_box_problem(3, 3, 3, q=q, phi_value=phi, rheology=rheo,
                                    body_force=(3e-4, -2e-4, 1e-4), d_p=2.0, forchheimer=forch)
        o = Oracle(prob)
        c, w, _ = o.lattice()
        for _ in range(5):
            f = _random_cell(o, rng, 0.2)
            _, info = o.collide_cell(0, f, 1.2)
            ph = float(np.float32(phi))
            lhs = ph * info["rho"] * info["u"]
            rhs = f @ c + 0.5 * info["F"]
            assert np.abs(lhs - rhs).max() < 1e-15 * max(1.0, np.abs(rhs).max()) + 1e-17
            assert abs(info["rho"] - f.sum() / ph) < 1e-14
        o.close()


@pytest.mark.parametrize("q", [19, 27])
def test_collision_mass_and_momentum(q):
    """With uniform porosity (Omega^phi = 0), the collision conserves mass and
    adds exactly F to the momentum: sum Omega^f = sum Omega^SRT = 0,
    sum Omega^f c = (1 - omega/2) F and sum Omega^SRT c = omega F / 2."""
    rng = np.random.default_rng(q)
    rheo = lattice_rheology(0.12, 0.01, 40.0, 0.35, 2.0)
    prob = periodic_box_problem(3, 3, 3, q=q, phi_value=0.75, rheology=rheo,
                                body_force=(1e-4, 2e-4, -3e-4), d_p=1.5, forchheimer=1)
    o = Oracle(prob)
    c, w, _ = o.lattice()
    for _ in range(10):
        f = _random_cell(o, rng, 0.3)
        fpost, info = o.collide_cell(0, f, 1.5)
        assert abs(fpost.sum() - f.sum()) < 1e-15
        assert np.abs(fpost @ c - (f @ c + info["F"])).max() < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_shear_rate_from_raw_second_moment(q):
    """gdot = omega_prev ||Pi||_F / (c_s^2 rho) with Pi written through the raw
    second moment: sum f^eq c c = phi rho (c_s^2 I + u u) for these second-order
    equilibria, so Pi = sum f c c - phi rho (c_s^2 I + u u) + (F u + u F)/2."""
    rng = np.random.default_rng(3 + q)
    rheo = lattice_rheology(0.12, 0.01, 40.0, 0.35, 2.0)
    for phi in (0.7, 1.0):
        prob = periodic_box_problem(3, 3, 3, q=q, phi_value=phi, rheology=rheo,
                                    body_force=(1e-4, 0, 0), d_p=1.5, forchheimer=1)
        o = Oracle(prob)
        c, w, _ = o.lattice()
        ph = float(np.float32(phi))
        for _ in range(5):
            f = _random_cell(o, rng, 0.1)
            om_prev = 1.3
            _, info = o.collide_cell(0, f, om_prev)
            rho, u, F = info["rho"], info["u"], info["F"]
            S = np.einsum("i,ia,ib->ab", f, c, c)
            P = S - ph * rho * (CS2 * np.eye(3) + np.outer(u, u)) + 0.5 * (np.outer(F, u) + np.outer(u, F))
            g = om_prev * np.sqrt((P * P).sum()) / (CS2 * rho)
            assert abs(g - info["gdot"]) < 1e-12 * abs(g)


def test_carreau_yasuda_limits():
    """Eq. (3): n = 1 or mu0 = mu_inf give a Newtonian rate omega = 1/(3 nu/rho + 1/2);
    a huge shear rate gives mu_inf; zero shear gives mu0."""
    rng = np.random.default_rng(7)
    cases = [
        (lattice_rheology(0.1, 0.01, 10.0, 1.0, 2.0), lambda g: 0.1),
        (lattice_rheology(0.05, 0.05, 10.0, 0.3, 2.0), lambda g: 0.05),
        (lattice_rheology(0.1, 0.01, 1e40, 0.3, 2.0), lambda g: 0.01),
        (lattice_rheology(0.1, 0.01, 1e-12, 0.3, 2.0), lambda g: 0.1),
    ]
    for rheo, mu in cases:
        prob = periodic_box_problem(2, 2, 2, q=19, rheology=rheo)
        o = Oracle(prob)
        f = _random_cell(o, rng, 0.2)
        _, info = o.collide_cell(0, f, 1.0)
        rho = info["rho"]
        expect = 1.0 / (mu(info["gdot"]) / (rho * CS2) + 0.5)
        assert abs(info["omega"] - expect) < 1e-9 * expect


def test_lattice_units_of_table1():
    """Table 1 (tests/golden/table1.json): the lattice scales dx = 43.95 um,
    dt = 5.42 us and rho0 = 1060 kg/m^3 map a dynamic viscosity mu to the lattice
    kinematic viscosity (mu / rho0) dt / dx^2, lambda to lambda / dt and the grain
    size to d_p / dx; the drag uses nu = mu0 / rho0 (Sec. 4)."""
    import json
    import os

    from lbm_inputs.configs import Problem, _no_inlet

    with open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")) as fh:
        t1 = json.load(fh)
    dx, dt, rho0 = t1["dx_um"] * 1e-6, t1["dt_us"] * 1e-6, t1["rho0_kg_m3"]
    rheo = dict(mu0=t1["mu0_read_kg_m_s"], mu_inf=t1["mu_inf_read_kg_m_s"], lam=t1["lambda_s"],
                n=t1["n"], a=t1["a"], rho0=rho0, dx=dx, dt=dt)
    porous = dict(d_p=t1["d_P_um"] * 1e-6, k_const=0.0, nu_darcy=0.0, forchheimer=1)
    bc = _no_inlet()
    bc["body_force"] = (0.0, 0.0, 0.0)
    prob = Problem("t1", np.ones((2, 2, 2), np.uint8), np.ones((2, 2, 2), np.float32), 27, (1, 1, 1),
                   rheo, porous, bc, None)
    lp = Oracle(prob).lattice_params()
    # dt / dx^2 = 5.42e-6 / (43.95e-6)^2 = 2805.96 s/m^2
    assert abs(dt / dx ** 2 - 2805.96) < 0.01
    assert abs(lp["mu0"] - 0.16 / 1060 * 2805.96) < 1e-5
    assert abs(lp["mu_inf"] - 0.0035 / 1060 * 2805.96) < 1e-6
    assert abs(lp["lam"] - 8.2 / 5.42e-6) < 1.0
    assert abs(lp["d_p"] - 600 / 43.95) < 1e-9
    assert lp["nu_d"] == lp["mu0"]
    # relaxation times of the limit viscosities, tau = 3 nu + 1/2
    assert 0.5 < 3 * lp["mu_inf"] + 0.5 < 3 * lp["mu0"] + 0.5
