"""Pins of the FP64 oracle against closed-form flows and exact invariants."""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, channel_problem, periodic_box_problem, pipe_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle

TAU_EXACT = 0.5 + np.sqrt(3.0 / 16.0)


def _channel_profile(o, ny):
    m = o.moments()
    return m["u"][0][0, :, 0], m


@pytest.mark.parametrize("q", [19, 27])
def test_poiseuille_exact_at_magic_tau(q):
    """Plane Poiseuille flow u = G (h^2 - y^2) / (2 nu) between half-way
    bounce-back walls (Sec. 4) is reproduced to round-off by BGK when
    tau = 1/2 + sqrt(3/16) (Krueger et al. 2017, Sec. 5.3): checks the viscosity
    to relaxation relation, the Guo force and the wall treatment at once."""
    ny, G = 18, 1e-6
    nu = (TAU_EXACT - 0.5) / 3.0
    o = Oracle(channel_problem(ny, q=q, nu=nu, body_force=G))
    o.step(20000)
    u, _ = _channel_profile(o, ny)
    h = (ny - 2) / 2.0
    y = np.arange(ny) + 0.5 - ny / 2.0
    exact = G * (h * h - y * y) / (2.0 * nu)
    err = np.abs(u[1:-1] - exact[1:-1]).max() / exact.max()
    assert err < 1e-10


@pytest.mark.parametrize("q", [19, 27])
def test_poiseuille_slip_is_uniform(q):
    """Away from the magic tau the BGK / bounce-back error of Poiseuille flow is
    a uniform slip: the profile is still an exact parabola of curvature -G/nu."""
    ny, G, tau = 18, 1e-6, 0.8
    nu = (tau - 0.5) / 3.0
    o = Oracle(channel_problem(ny, q=q, nu=nu, body_force=G))
    o.step(20000)
    u, _ = _channel_profile(o, ny)
    h = (ny - 2) / 2.0
    y = np.arange(ny) + 0.5 - ny / 2.0
    diff = u[1:-1] - G * (h * h - y[1:-1] ** 2) / (2.0 * nu)
    assert np.ptp(diff) < 1e-9 * u.max()
    assert abs(diff.mean()) > 1e-4 * u.max()  # a genuine slip, not zero


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("mode", ["kc", "kc_darcy_only", "k_const"])
def test_uniform_darcy_forchheimer_fixed_point(q, mode):
    """Uniform porous medium, fully periodic, body force g: each step adds
    exactly rho (g + f_d(u)) of momentum, so the steady velocity solves
    g = phi^2 nu u / k + phi^3 C_F |u| u / sqrt(k) (Sec. 2) for any viscosity
    law: |u| = (-a + sqrt(a^2 + 4 b |g|)) / (2 b), a = phi^2 nu / k,
    b = phi^3 C_F / sqrt(k).  Kozeny-Carman k = phi^3 d^2 / (150 (1-phi)^2),
    Ergun C_F = 1.75 / sqrt(150 phi^3)."""
    rheo = lattice_rheology(0.1, 0.02, 20.0, 0.5, 2.0)
    phi_set, d, g = 0.7, 3.0, np.array([2e-4, 1e-4, -0.5e-4])
    forch = 0 if mode == "kc_darcy_only" else 1
    kc = 0.6 if mode == "k_const" else 0.0
    prob = periodic_box_problem(4, 3, 5, q=q, phi_value=phi_set, rheology=rheo, body_force=tuple(g),
                                d_p=d, k_const=kc, forchheimer=forch)
    o = Oracle(prob)
    o.step(3000)
    m = o.moments()
    u = m["u"][:, 1, 1, 1]
    phi = float(np.float32(phi_set))
    nu = 0.1
    k = kc if kc > 0 else phi ** 3 * d * d / (150 * (1 - phi) ** 2)
    cf = 1.75 / np.sqrt(150 * phi ** 3) if forch else 0.0
    a = phi ** 2 * nu / k
    b = phi ** 3 * cf / np.sqrt(k)
    gn = np.linalg.norm(g)
    un = gn / a if b == 0 else (-a + np.sqrt(a * a + 4 * b * gn)) / (2 * b)
    assert abs(np.linalg.norm(u) - un) < 1e-11 * un
    assert np.abs(u / np.linalg.norm(u) - g / gn).max() < 1e-10
    assert np.ptp(m["u"][0]) < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_mass_conserved_uniform_porosity(q):
    """Uniform porosity, walls and periodic axes only: the collision conserves
    mass and streaming / bounce-back moves it, so sum f stays constant to
    round-off over 2000 perturbed, forced, non-Newtonian steps."""
    rheo = lattice_rheology(0.1, 0.02, 20.0, 0.5, 2.0)
    prob = periodic_box_problem(8, 6, 5, q=q, phi_value=0.8, rheology=rheo, body_force=(1e-5, 0, 2e-6),
                                obstacles=25, d_p=3.0)
    o = Oracle(prob)
    f, om = o.get_state()
    rng = np.random.default_rng(1)
    o.set_state(f * (1 + 0.05 * rng.standard_normal(f.shape)), om, 0)
    m0 = o.diag()[0]
    o.step(2000)
    m1 = o.diag()[0]
    assert abs(m1 - m0) < 2e-12 * m0  # round-off accumulated over 2000 steps


@pytest.mark.parametrize("q", [19, 27])
def test_mass_change_equals_porosity_source(q):
    """With varying porosity the only mass source is Omega^phi:
    Delta M = sum_x rho(x) sum_i w_i (phi(x + c_i) - phi(x)), with phi(x + c_i)
    replaced by phi(x) across solid links (Sec. 3, porosity collision term)."""
    rheo = lattice_rheology(0.1, 0.02, 20.0, 0.5, 2.0)
    rng = np.random.default_rng(5)
    phi = (0.6 + 0.4 * rng.random((5, 6, 7))).astype(np.float32)
    prob = periodic_box_problem(7, 6, 5, q=q, rheology=rheo, body_force=(1e-5, 0, 0), obstacles=10, phi=phi)
    o = Oracle(prob)
    f, om = o.get_state()
    o.set_state(f * (1 + 0.02 * rng.standard_normal(f.shape)), om, 0)
    o.step(3)
    c, w, _ = o.lattice()
    m = o.moments()
    rho = m["rho"]
    flags = prob.flags
    ph = prob.phi.astype(np.float64)
    fluid = flags > 0
    src = np.zeros_like(ph)
    for i in range(o.q):
        sh = (-c[i][2], -c[i][1], -c[i][0])
        nb_phi = np.roll(ph, shift=sh, axis=(0, 1, 2))
        nb_fluid = np.roll(fluid, shift=sh, axis=(0, 1, 2))
        src += w[i] * np.where(nb_fluid, nb_phi - ph, 0.0)
    expect = (rho * src)[fluid].sum()
    M0 = o.diag()[0]
    o.step(1)
    dM = o.diag()[0] - M0
    assert abs(dM - expect) < 1e-13 * M0
    assert abs(expect) > 1e-6  # the source term is genuinely active


@pytest.mark.parametrize("q", [19, 27])
def test_rest_state_is_fixed_point_with_porosity(q):
    """At rest, f = w_i phi: the collision gives f* = w_i phi(x + c_i) through
    Omega^phi, which streams onto the rest equilibrium of the neighbour, and the
    bounce-back links carry no porosity jump.  With zero inflow and rho_out = 1
    the state must stay at rest exactly, in a porous aneurysm with both open
    boundaries."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.0)
    o = Oracle(prob)
    o.step(50)
    m = o.moments()
    fl = prob.flags > 0
    assert np.abs(m["u"]).max() < 1e-13  # round-off; a wrong porosity link gives ~1e-2
    assert np.abs(m["rho"][fl] - 1.0).max() < 1e-14
    assert np.ptp(prob.phi[fl]) > 0.15  # porosity really varies


def test_pipe_symmetry():
    """The pipe is symmetric under x -> 31 - x, y -> 31 - y and x <-> y; the
    FP64 solution must keep these symmetries to round-off."""
    prob = pipe_problem(q=19)
    o = Oracle(prob)
    o.step(200)
    uz = o.moments()["u"][2]
    s = np.abs(uz).max()
    assert s > 1e-5
    assert np.abs(uz - uz[:, :, ::-1]).max() < 1e-10 * s
    assert np.abs(uz - uz[:, ::-1, :]).max() < 1e-10 * s
    assert np.abs(uz - uz.transpose(0, 2, 1)).max() < 1e-10 * s


def _brinkman_error(q, h):
    """Max error of the oracle against the Brinkman profile (Sec. 2 with
    uniform phi and no Forchheimer term): nu phi u'' - phi^2 nu_D u / k + g = 0,
    u = u_D (1 - cosh(beta y) / cosh(beta h)), u_D = g k / (phi^2 nu_D),
    beta^2 = phi nu_D / (k nu).  beta h = 2 is kept fixed as h grows."""
    ny = 2 * h + 2
    phi_set, nu, g = 0.8, 0.1, 1e-6
    phi = float(np.float32(phi_set))
    beta = 2.0 / h
    k = phi * nu / (beta * beta * nu)  # nu_D = nu (Newtonian, nu = mu0)
    d = np.sqrt(k * 150 * (1 - phi) ** 2 / phi ** 3)
    rheo = lattice_rheology(nu, nu, 0.0, 1.0, 2.0)
    prob = channel_problem(ny, q=q, rheology=rheo, body_force=g, phi_value=phi_set, d_p=d, forchheimer=0)
    o = Oracle(prob)
    o.step(int(40 * h * h / nu) + 2000)
    u = o.moments()["u"][0][0, :, 0]
    y = np.arange(ny) + 0.5 - ny / 2.0
    ud = g * k / (phi * phi * nu)
    exact = ud * (1 - np.cosh(beta * y) / np.cosh(beta * h))
    return np.abs(u[1:-1] - exact[1:-1]).max() / exact.max()


@pytest.mark.parametrize("q", [19])
def test_brinkman_channel_converges_second_order(q):
    e1 = _brinkman_error(q, 4)
    e2 = _brinkman_error(q, 8)
    assert e2 < 0.02
    assert e1 / e2 > 3.0  # second order: the error falls ~4x per halving of dx


def _cy_reference(y, h, g, mu):
    """1-D quadrature reference of steady Carreau-Yasuda plane Poiseuille flow:
    the shear stress is exact, mu(sqrt(2) |u'|) |u'| = g |y| (rho = 1), since
    ||gdot||_F = sqrt(2) |u'| for a shear flow (Sec. 2); |u'| is found by
    bisection and integrated from the wall at y = h.  Returns (u, |u'|)."""

    def dudy(yy):
        tau = g * abs(yy)
        lo, hi = 0.0, 1.0
        while mu(np.sqrt(2) * hi) * hi < tau:
            hi *= 2
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if mu(np.sqrt(2) * mid) * mid < tau:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    u, du = [], []
    for yy in y:
        xs = np.linspace(abs(yy), h, 801)
        vals = np.array([dudy(x) for x in xs])
        u.append(np.trapezoid(vals, xs))
        du.append(dudy(yy))
    return np.array(u), np.array(du)


def _cy_channel_error(h):
    """Steady Carreau-Yasuda channel at half-width h (lambda and g scaled so the
    dimensionless problem is the same at every h): max relative errors of the
    velocity and of the recovered shear rate gdot (from Pi, with
    omega(t-1) = omega(t) at steady state) against the quadrature reference."""
    g = 2e-5 * (8.0 / h) ** 3
    ny = 2 * h + 2
    mu0, mui, lam, n, a = 0.12, 0.02, 2000.0 * (h / 8.0) ** 2, 0.5, 2.0
    rheo = lattice_rheology(mu0, mui, lam, n, a)

    def mu(gd):
        return mui + (mu0 - mui) * (1 + (lam * gd) ** a) ** ((n - 1) / a)

    o = Oracle(channel_problem(ny, q=19, rheology=rheo, body_force=g))
    o.step(int(40000 * (h / 8.0) ** 2))
    m = o.moments()
    u = m["u"][0][0, 1:-1, 0]
    y = (np.arange(ny) + 0.5 - ny / 2.0)[1:-1]
    ref, dref = _cy_reference(y, h, g, mu)
    gref = np.sqrt(2) * dref
    sel = np.abs(y) > 2  # away from the centre line, where gdot -> 0
    eu = np.abs(u - ref).max() / ref.max()
    eg = np.abs(m["gdot"][0, 1:-1, 0] - gref)[sel].max() / gref.max()
    return eu, eg, np.ptp(m["omega"][0, 1:-1, 0])


def test_carreau_yasuda_poiseuille():
    """Shear-thinning channel flow converges at second order to the quadrature
    reference, and gdot from Pi equals sqrt(2) |u'| of that reference."""
    e8, g8, om8 = _cy_channel_error(8)
    e16, g16, _ = _cy_channel_error(16)
    assert e16 < 2e-3
    assert e8 / e16 > 3.0
    assert g16 < 1e-5 and g8 < 1e-4
    assert om8 > 0.05  # the viscosity genuinely varies across the channel
