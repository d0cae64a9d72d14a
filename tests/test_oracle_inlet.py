"""Stability pin of the Zou-He inlet (Sec. 4) at the lowest relaxation time
the Carreau-Yasuda law of the blood workloads reaches (tau = 0.527 at mu_inf
at the Table 1 spacing).

An open pipe (Zou-He inlet on z = 0 with zero inflow, extrapolation outlet on
z = nz - 1, Newtonian BGK at tau = 0.527) starts from the rest state with a
1e-4 perturbation of every population.  The oracle's inlet, non-equilibrium
bounce-back of the unknown populations, lets the perturbation decay.  A
planted copy of the oracle that adds the tangential correction of the D2Q9 /
D3Q19 literature (the residual N_t = sum_{c.n=0} (f - f^eq) c_t removed from
the unknowns with c_t != 0) must let it grow: that correction is what made the
aneurysm workloads lose finiteness with the stated relaxation time lambda of
the Carreau-Yasuda law.
"""

import os

import numpy as np
import pytest

from lbm_inputs import geometry as geo
from lbm_inputs.configs import Problem, lattice_rheology
from oracle import oracle as oracle_mod
from oracle.oracle import Oracle

TAU = 0.527
R, L = 10, 24
STEPS = 600


def open_pipe(q):
    n = 2 * R + 6
    flags = geo.pipe_flags(n, n, L, radius=R, cx=n / 2, cy=n / 2)
    flags[0][flags[0] == 1] = 2
    flags[L - 1][flags[L - 1] == 1] = 3
    phi = np.ones(flags.shape, np.float32)
    nu = (TAU - 0.5) / 3.0
    bc = dict(body_force=(0.0, 0.0, 0.0), inlet_axis=2, inlet_side=0, inlet_center=(n / 2, n / 2, 0.0),
              inlet_radius=R, u0=0.0, amp=0.0, period=1.0, ramp_steps=0.0, outlet_axis=2, outlet_side=1,
              rho_out=1.0)
    porous = dict(d_p=1.0, k_const=0.0, nu_darcy=0.0, forchheimer=0)
    return Problem("open_pipe", flags, phi, q, (0, 0, 0), lattice_rheology(nu, nu, 0.0, 1.0, 2.0), porous, bc, None)


def perturbation_growth(q, library=None):
    """max |rho - 1| after STEPS steps over its value after 20 steps."""
    prob = open_pipe(q)
    o = Oracle(prob, library=library)
    f, om = o.get_state()
    rng = np.random.default_rng(0)
    o.set_state(f * (1 + 1e-4 * rng.standard_normal(f.shape)), om, 0)
    fluid = prob.flags > 0
    o.step(20)
    a0 = np.abs(o.moments()["rho"][fluid] - 1).max()
    o.step(STEPS - 20)
    a1 = np.abs(o.moments()["rho"][fluid] - 1).max()
    o.close()
    return a1 / a0 if np.isfinite(a1) else np.inf


@pytest.mark.parametrize("q", [19, 27])
def test_inlet_rest_state_perturbation_decays_at_lowest_relaxation_time(q):
    assert perturbation_growth(q) < 0.5


RECONSTRUCTION = ("            f[i] = f[o->opp[i]] + equilibrium(o, i, phi, rho, ub) - "
                  "equilibrium(o, o->opp[i], phi, rho, ub);\n}")
TANGENTIAL_CORRECTION = """
    for (int tng = 0; tng < 3; ++tng) {
        if (tng == ax) continue;
        double nres = 0.0, ncnt = 0.0;
        for (int i = 0; i < o->q; ++i) {
            int cn = o->c[i][ax] * sgn;
            if (cn == 0) nres += (f[i] - equilibrium(o, i, phi, rho, ub)) * o->c[i][tng];
            if (cn > 0) ncnt += o->c[i][tng] * o->c[i][tng];
        }
        for (int i = 0; i < o->q; ++i)
            if (o->c[i][ax] * sgn > 0) f[i] -= o->c[i][tng] * nres / ncnt;
    }
}"""


def test_planted_tangential_correction_makes_the_inlet_unstable(tmp_path):
    with open(os.path.join(os.path.dirname(oracle_mod.__file__), "lbm_oracle.c")) as fh:
        src = fh.read()
    assert src.count(RECONSTRUCTION) == 1
    path = os.path.join(tmp_path, "corrected.c")
    with open(path, "w") as fh:
        fh.write(src.replace(RECONSTRUCTION, RECONSTRUCTION[:-1] + TANGENTIAL_CORRECTION))
    lib = oracle_mod.load_library(oracle_mod.compile_library(path, os.path.join(tmp_path, "corrected.so")))
    assert perturbation_growth(27, lib) > 100.0
