"""Workload definitions: geometry + porosity + physical parameters.

Parameters are given as the user states them: rheology in SI units together
with the grid spacing, time step and reference density that map them to the
lattice (Table 1 of the paper), inlet/body-force values in lattice units.
Converting them is each consumer's own job.
"""

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import geometry as geo
from . import porosity as por

# Table 1 of the paper: reference density, grid spacing, time step, grain size.
PAPER_TABLE1 = dict(rho0=1060.0, dx=43.95e-6, dt=5.42e-6, d_p=600e-6)

# Carreau-Yasuda blood parameters of the synthetic workloads (SI).
WORKLOAD_CY = dict(mu0=0.056, mu_inf=0.00345, lam=3.313, n=0.3568, a=2.0)

# Viscosity relaxation time of the aneurysm workloads [s]: the stated 3.313 s
# (611 255 time steps at the Table 1 spacing), with which any shear takes the
# viscosity to mu_inf (relaxation time tau = 0.527).  The inlet's
# non-equilibrium bounce-back stays stable there; with the tangential
# correction of the D2Q9 / D3Q19 literature added to it, the same workloads
# lost finiteness within 200-400 steps.
ANEURYSM_LAMBDA = WORKLOAD_CY["lam"]

# Body force (lattice units) driving the 32x32x64 pipe: the Newtonian estimate
# G = 4 Re nu_inf^2 / R^3 for Re = 10, R = 14 and nu_inf = 0.0091326 (mu_inf of
# WORKLOAD_CY at the Table 1 spacing).
PIPE_BODY_FORCE = 1.2158e-6


@dataclass
class Problem:
    """One complete problem statement for the VANSE LBM."""

    name: str
    flags: np.ndarray            # uint8 (nz, ny, nx)
    phi: np.ndarray              # float32 (nz, ny, nx)
    q: int = 27
    periodic: tuple = (0, 0, 0)
    rheology: dict = field(default_factory=dict)   # mu0, mu_inf, lam, n, a (SI); rho0, dx, dt
    porous: dict = field(default_factory=dict)     # d_p [m], k_const [m^2] (0: Kozeny-Carman), nu_darcy [m^2/s] (<=0: mu0/rho0), forchheimer
    bc: dict = field(default_factory=dict)         # body_force, inlet_*, outlet_*, rho_out (lattice units)
    region: Optional[np.ndarray] = None            # uint8 (nz, ny, nx) objective / diagnostic region

    @property
    def dims(self):
        nz, ny, nx = self.flags.shape
        return nx, ny, nz

    @property
    def n_fluid(self):
        return int((self.flags != geo.SOLID).sum())


def _no_inlet():
    return dict(inlet_axis=-1, inlet_side=0, inlet_center=(0.0, 0.0, 0.0), inlet_radius=1.0,
                u0=0.0, amp=0.0, period=1.0, ramp_steps=0.0,
                outlet_axis=-1, outlet_side=1, rho_out=1.0)


def pipe_problem(q=19, storage="f32"):
    """32x32x64 pipe of radius 14 along z, periodic in z, driven by a body force;
    porosity 0.75 in the plug z=24..40, 1 elsewhere.  Carreau-Yasuda blood."""
    flags = geo.pipe_flags()
    phi = por.plug_porosity(flags)
    bc = _no_inlet()
    bc["body_force"] = (0.0, 0.0, PIPE_BODY_FORCE)
    rheo = dict(WORKLOAD_CY, rho0=PAPER_TABLE1["rho0"], dx=PAPER_TABLE1["dx"], dt=PAPER_TABLE1["dt"])
    porous = dict(d_p=PAPER_TABLE1["d_p"], k_const=0.0, nu_darcy=0.0, forchheimer=1)
    return Problem("pipe32x32x64", flags, phi, q, (0, 0, 1), rheo, porous, bc, None)


def aneurysm_problem(n, q=27, seed=0, small=False, porous_sac=True, u0=0.05, amp=0.5,
                     period=1000.0, ramp_steps=0.0, coil=None, lam=None):
    """Synthetic aneurysm in an n^3 box with a pulsatile Poiseuille inlet on z=0
    and a pressure outlet on x=n-1; sac porosity from the seeded random field.

    ``coil``: None (random porous field), or a uint8 wire mask; then
    ``porous_sac`` picks the box-filtered porosity (True) or solid wire voxels
    (False, fully resolved).  ``lam``: viscosity relaxation time [s]
    (default ANEURYSM_LAMBDA).
    """
    flags = geo.aneurysm_flags(n, small)
    region = geo.sac_mask(n, small)
    if coil is None:
        phi = por.sac_random_porosity(n, small, seed) if porous_sac else np.ones((n, n, n), np.float32)
    else:
        raise NotImplementedError("wire coils are built by coil_problem")
    cx, cy, r = geo.aneurysm_inlet(n, small)
    bc = dict(body_force=(0.0, 0.0, 0.0), inlet_axis=2, inlet_side=0,
              inlet_center=(cx, cy, 0.0), inlet_radius=r, u0=u0, amp=amp, period=period,
              ramp_steps=ramp_steps, outlet_axis=0, outlet_side=1, rho_out=1.0)
    rheo = dict(WORKLOAD_CY, rho0=PAPER_TABLE1["rho0"], dx=PAPER_TABLE1["dx"], dt=PAPER_TABLE1["dt"])
    rheo["lam"] = ANEURYSM_LAMBDA if lam is None else lam
    porous = dict(d_p=PAPER_TABLE1["d_p"], k_const=0.0, nu_darcy=0.0, forchheimer=1)
    name = f"aneurysm{n}" + ("s" if small else "")
    return Problem(name, flags, phi, q, (0, 0, 0), rheo, porous, bc, region)


# The paper's porosity averaging window (Table 1: 1.23 mm, 28 cells at the
# Table 1 spacing) and the lower clamp of the averaged porosity.  With an 8^3
# window the 2-voxel wire gives porosities down to the clamp and steps of an
# eighth between neighbouring cells; the 512^3 workload then loses finiteness
# at 20 and 25 % packing (measured over 5000 steps; 15 % stays finite).
COIL_WINDOW = 28
COIL_PHI_MIN = 0.05


def coil_problem(n, resolved, packing=0.25, seed=0, q=27, wire=None, phi=None, base=None, **kw):
    """The aneurysm of :func:`aneurysm_problem` with a wire coil in the sac
    (Sec. 4): a seeded random-walk helical wire, 2 voxels thick, filling
    ``packing`` of the sac (:func:`porosity.wire_coil`).

    ``resolved``: the wire voxels are solid (half-way bounce-back), porosity 1
    elsewhere.  Otherwise (volume averaged): every cell stays fluid and the
    porosity is ``phi``, the volume average of the wire over the
    COIL_WINDOW^3 box clamped at COIL_PHI_MIN, which the caller computes
    (lbm.porosity_average on the GPU; the oracle's porosity_average in tests);
    it may be a CUDA tensor.  ``wire``: a precomputed wire mask (else it is
    generated from ``packing`` and ``seed``).  ``base``: the uncoiled problem,
    if already built.  Other keywords go to aneurysm_problem.
    """
    base = base if base is not None else aneurysm_problem(n, q=q, porous_sac=False, **kw)
    if not resolved:
        if phi is None:
            raise ValueError("the averaged coil takes its averaged porosity field as phi")
        return dataclasses.replace(base, name=f"coil{n}a", phi=phi)
    wire = (por.wire_coil(n, packing=packing, seed=seed) if wire is None else wire) > 0
    flags = base.flags.copy()
    flags[wire] = 0
    return dataclasses.replace(base, name=f"coil{n}r", flags=flags)


def lattice_rheology(mu0, mu_inf, lam, n, a):
    """Rheology stated directly in lattice units (dx = dt = rho0 = 1)."""
    return dict(mu0=mu0, mu_inf=mu_inf, lam=lam, n=n, a=a, rho0=1.0, dx=1.0, dt=1.0)


def channel_problem(ny, q=19, nu=None, rheology=None, body_force=1e-6, phi_value=1.0,
                    d_p=None, k_const=0.0, forchheimer=0, nx=2, nz=2):
    """Plane channel (walls normal to y, periodic in x and z) driven along x.

    Lattice units throughout.  ``nu`` gives a Newtonian fluid (mu0 = mu_inf);
    ``rheology`` a Carreau-Yasuda dict from :func:`lattice_rheology`.
    """
    flags = geo.channel_flags(ny, nx, nz)
    phi = np.full(flags.shape, np.float32(phi_value), dtype=np.float32)
    if rheology is None:
        rheology = lattice_rheology(nu, nu, 0.0, 1.0, 2.0)
    bc = _no_inlet()
    bc["body_force"] = (body_force, 0.0, 0.0)
    porous = dict(d_p=d_p if d_p is not None else 1.0, k_const=k_const, nu_darcy=0.0,
                  forchheimer=forchheimer)
    return Problem(f"channel{ny}", flags, phi, q, (1, 0, 1), rheology, porous, bc, None)


def periodic_box_problem(nx, ny, nz, q=27, phi_value=1.0, rheology=None, body_force=(0.0, 0.0, 0.0),
                         d_p=1.0, k_const=0.0, forchheimer=1, nu_darcy=0.0, obstacles=0, seed=0,
                         phi=None):
    """Fully periodic box in lattice units, optional random solid voxels and an
    optional explicit porosity field."""
    flags = geo.periodic_box_flags(nx, ny, nz, obstacles, seed)
    if phi is None:
        phi = np.full(flags.shape, np.float32(phi_value), dtype=np.float32)
    if rheology is None:
        rheology = lattice_rheology(0.1, 0.1, 0.0, 1.0, 2.0)
    bc = _no_inlet()
    bc["body_force"] = tuple(body_force)
    porous = dict(d_p=d_p, k_const=k_const, nu_darcy=nu_darcy, forchheimer=forchheimer)
    return Problem(f"box{nx}x{ny}x{nz}", flags, phi.astype(np.float32), q, (1, 1, 1), rheology,
                   porous, bc, None)
