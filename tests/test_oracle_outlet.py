"""Pins of the oracle's extrapolation outlet (Sec. 4: outflow by extrapolation,
with the prescribed outlet density of the pressure outlet) against closed-form
open-channel flows, with planted mistakes that each must fail them.

Geometry: a plane channel one cell wide in x (periodic), walls normal to y at
half-links (half-width h = (ny - 2) / 2), a Zou-He velocity inlet on z = 0 and
the extrapolation outlet on z = nz - 1 with rho_out = 1.  Newtonian BGK at
tau = 1/2 + sqrt(3/16), the relaxation time at which half-way bounce-back
carries plane Poiseuille flow exactly (Krueger et al. 2017, Sec. 5.3).  The
inlet's disk profile 2 v (1 - r^2 / R^2) with R = h and the centre on the cell
centre in x is the plane parabola u_max (1 - y^2 / h^2), u_max = 2 v.

* Body-force driven: with g = G e_z and u_max = G h^2 / (2 nu) the fully
  developed Poiseuille flow at uniform density rho_out is a z-invariant steady
  state that the outlet must leave undisturbed: downstream of the inlet's
  developing region the profile is the parabola and rho = rho_out.
* Pressure driven (g = 0): the outlet alone sets the density level.  Plane
  Poiseuille flow needs dp/dz = -2 nu rho u_max / h^2, i.e. with p = rho / 3
  a linear density of slope -6 nu u_max / h^2 (the -3 G of the equivalent
  body force G = 2 nu u_max / h^2), uniform across y, reaching rho_out at the
  outlet cells.  The weak compressibility of the scheme (rho u_z, not u_z, is
  constant along z) perturbs this at the order of the density drop, 3e-5 here.

Planted mistakes (compiled from a copy of the oracle source with one line
changed): rho_nb for rho_out in the first equilibrium (the outlet degenerates
to a zero-gradient copy), the non-equilibrium part dropped, a zero velocity in
the first equilibrium, and the unknown populations selected with the wrong
sign of the normal.  The third slip named for this boundary, the cell's own
porosity for the neighbour's, cannot act: the oracle and the library both
require porosity 1 on outlet cells and on their interior neighbours.
"""

import os

import numpy as np
import pytest

from lbm_inputs.configs import Problem, lattice_rheology
from oracle import oracle as oracle_mod
from oracle.oracle import Oracle

TAU_EXACT = 0.5 + np.sqrt(3.0 / 16.0)
NU = (TAU_EXACT - 0.5) / 3.0
NY, NZ, STEPS = 18, 24, 30000
H = (NY - 2) / 2.0


def open_channel(q, G=0.0, u_max=None):
    flags = np.ones((NZ, NY, 1), np.uint8)
    flags[:, 0, :] = 0
    flags[:, NY - 1, :] = 0
    flags[0, 1:NY - 1, :] = 2
    flags[NZ - 1, 1:NY - 1, :] = 3
    phi = np.ones(flags.shape, np.float32)
    if u_max is None:
        u_max = G * H * H / (2.0 * NU)
    bc = dict(body_force=(0.0, 0.0, G), inlet_axis=2, inlet_side=0, inlet_center=(0.5, NY / 2.0, 0.0),
              inlet_radius=H, u0=u_max / 2.0, amp=0.0, period=1.0, ramp_steps=0.0,
              outlet_axis=2, outlet_side=1, rho_out=1.0)
    porous = dict(d_p=1.0, k_const=0.0, nu_darcy=0.0, forchheimer=0)
    prob = Problem("open_channel", flags, phi, q, (1, 0, 0), lattice_rheology(NU, NU, 0.0, 1.0, 2.0), porous, bc,
                   None)
    return prob, u_max


def run(q, mode, library=None):
    """Steady fields of the open channel: u_z and rho on the (z, y) plane."""
    if mode == "force":
        prob, u_max = open_channel(q, G=1e-6)
    else:
        prob, u_max = open_channel(q, u_max=1e-4)
    o = Oracle(prob, library=library)
    o.step(STEPS)
    m = o.moments()
    o.close()
    return m["u"][2][:, :, 0], m["rho"][:, :, 0], u_max


def parabola(u_max):
    y = np.arange(NY) + 0.5 - NY / 2.0
    return u_max * (1.0 - y * y / (H * H))


def force_pins(u, rho, u_max):
    """Relative profile error at the outlet slice, largest |rho - rho_out|
    over the downstream half, and the spread of the mass flux over z."""
    err = np.abs(u[NZ - 1, 1:-1] - parabola(u_max)[1:-1]).max() / u_max
    drho = np.abs(rho[NZ // 2:, 1:-1] - 1.0).max()
    flux = (rho[:, 1:-1] * u[:, 1:-1]).sum(axis=1)
    return err, drho, np.ptp(flux) / flux.mean()


def pressure_pins(u, rho, u_max):
    """Density slope against -6 nu u_max / h^2 (relative), the outlet density
    against rho_out and the residual of the linear fit (both relative to the
    density drop along the channel), and the spread across y over the
    downstream half (the inlet's developing region is not the outlet's)."""
    z = np.arange(NZ)
    r = rho[:, 1:-1].mean(axis=1)
    slope, icpt = np.polyfit(z[2:-2], r[2:-2], 1)
    expect = -6.0 * NU * u_max / (H * H)
    drop = abs(expect) * (NZ - 1)
    fit = np.abs(r[2:-2] - (slope * z[2:-2] + icpt)).max() / drop
    out = np.abs(rho[NZ - 1, 1:-1] - 1.0).max() / drop
    across = max(np.ptp(rho[k, 1:-1]) for k in range(NZ // 2, NZ)) / drop
    return abs(slope / expect - 1.0), out, fit, across


@pytest.mark.parametrize("q", [19, 27])
def test_body_force_poiseuille_leaves_the_outlet_undisturbed(q):
    u, rho, u_max = run(q, "force")
    err, drho, flux = force_pins(u, rho, u_max)
    assert err < 1e-7  # measured 4.6e-9
    assert drho < 1e-10  # measured 5.0e-12
    assert flux < 1e-10  # steady: the mass flux is the same through every slice


@pytest.mark.parametrize("q", [19, 27])
def test_pressure_driven_channel_has_the_poiseuille_pressure_drop(q):
    u, rho, u_max = run(q, "pressure")
    slope, out, fit, across = pressure_pins(u, rho, u_max)
    assert slope < 1e-4  # measured 1.8e-5 (weak compressibility)
    assert out < 1e-4  # measured 1.0e-5 of the drop
    assert fit < 1e-4  # measured 2.8e-6
    assert across < 1e-4  # measured 4.1e-6
    # the profile stays the parabola up to the compressibility of the scheme
    assert np.abs(u[NZ - 1, 1:-1] - parabola(u_max)[1:-1]).max() / u_max < 1e-4


OUTLET_LINE = ("            f[i] = equilibrium(o, i, o->phi[idx], o->p.rho_out, u_nb) + fn[i] - "
               "equilibrium(o, i, o->phi[nbi], rho_nb, u_nb);")
SELECT = "        if (o->c[i][ax] * sgn > 0)\n" + OUTLET_LINE.split(" + fn[i]")[0]
PLANTS = {
    "rho_nb_for_rho_out": (OUTLET_LINE, OUTLET_LINE.replace("o->p.rho_out, u_nb", "rho_nb, u_nb")),
    "non_equilibrium_dropped": (OUTLET_LINE, OUTLET_LINE.split(" + fn[i]")[0] + ";"),
    "zero_velocity_in_first_equilibrium": (
        OUTLET_LINE, "            { double u0_[3] = {0.0, 0.0, 0.0}; "
                     + OUTLET_LINE.strip().replace("o->p.rho_out, u_nb", "o->p.rho_out, u0_") + " }"),
    "normal_sign_of_the_unknowns": (SELECT, SELECT.replace("* sgn > 0", "* sgn < 0")),
}


@pytest.fixture(scope="module")
def planted(tmp_path_factory):
    with open(os.path.join(os.path.dirname(oracle_mod.__file__), "lbm_oracle.c")) as fh:
        src = fh.read()
    d = tmp_path_factory.mktemp("planted_oracle")
    libs = {}
    for name, (a, b) in PLANTS.items():
        assert src.count(a) == 1, f"planted line of {name} not found exactly once"
        path = os.path.join(d, name + ".c")
        with open(path, "w") as fh:
            fh.write(src.replace(a, b))
        libs[name] = oracle_mod.load_library(oracle_mod.compile_library(path, os.path.join(d, name + ".so")))
    return libs


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_outlet_mistakes_fail_the_pins(planted, name):
    u, rho, u_max = run(19, "force", planted[name])
    err, drho, flux = force_pins(u, rho, u_max)
    assert err > 1e-5 or drho > 1e-6 or flux > 1e-6, f"{name} passes the body-force pins"
    u, rho, u_max = run(19, "pressure", planted[name])
    slope, out, fit, across = pressure_pins(u, rho, u_max)
    assert slope > 1e-3, f"{name} passes the pressure-drop pin"
