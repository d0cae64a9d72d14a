"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error metric: max over fluid cells of |u_gpu - u_ref| divided by max |u_ref|
(pointwise relative error is undefined where u = 0); the same for the shear
rate.  Tolerances: FP32 storage 1e-5 (velocity), FP16 deviation storage 1e-3,
BF16 deviation storage 1e-2 (reported; 8-bit significand).
"""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, periodic_box_problem, pipe_problem
from lbm_inputs.configs import lattice_rheology
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu

TOL_U = {"f32": 1e-5, "f16dev": 1e-3, "bf16dev": 1e-2}


def rel_err(a, b, fluid):
    den = np.abs(b[..., fluid]).max()
    return np.abs(a[..., fluid] - b[..., fluid]).max() / max(den, 1e-300)


def run_both(lbm, prob, steps, storage="f32"):
    sim = lbm.Simulation(prob, storage=storage)
    sim.step(steps)
    g = sim.moments()
    o = Oracle(prob)
    o.step(steps)
    r = o.moments()
    fluid = prob.flags > 0
    errs = dict(
        u=rel_err(g["u"].astype(np.float64), r["u"], fluid),
        rho=np.abs(g["rho"][fluid] - r["rho"][fluid]).max(),
        gdot=rel_err(g["gdot"].astype(np.float64), r["gdot"], fluid),
        omega=np.abs(g["omega"][fluid] - r["omega"][fluid]).max(),
    )
    assert sim.t == steps
    return sim, o, errs


@pytest.mark.parametrize("q", [19, 27])
def test_pipe_fp32_200_steps(lbm, q):
    """32x32x64 pipe, Carreau-Yasuda, porous plug, body force, periodic z."""
    _, _, e = run_both(lbm, pipe_problem(q=q), 200)
    assert e["u"] <= 1e-5, e
    assert e["rho"] <= 1e-6, e
    assert e["gdot"] <= 1e-4, e


def test_small_aneurysm_short_relaxation_time(lbm):
    """The 24^3 aneurysm with a hundred times shorter Carreau-Yasuda relaxation
    time than the workload's 3.313 s: the viscosity stays between mu_0 and
    mu_inf over the flow instead of sitting at mu_inf, so the whole law (and
    the omega(t-1) feedback of the shear rate) is exercised."""
    from lbm_inputs.configs import WORKLOAD_CY

    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0, lam=WORKLOAD_CY["lam"] / 100)
    _, _, e = run_both(lbm, prob, 200)
    assert e["u"] <= 1e-5, e


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("storage", ["f32", "f16dev", "bf16dev"])
def test_small_aneurysm(lbm, q, storage):
    """24^3 aneurysm: porous sac, pulsatile Zou-He inlet, extrapolation outlet."""
    prob = aneurysm_problem(24, q=q, small=True, u0=0.05, period=100.0)
    _, _, e = run_both(lbm, prob, 200, storage)
    assert e["u"] <= TOL_U[storage], e


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_aneurysm_64(lbm, storage):
    """64^3 aneurysm family member: many blocks and a ragged last block."""
    prob = aneurysm_problem(64, q=27, u0=0.05, period=200.0)
    assert prob.n_fluid % 256 != 0
    _, _, e = run_both(lbm, prob, 300, storage)
    assert e["u"] <= TOL_U[storage], e


def test_full_size_aneurysm_256_fp32(lbm):
    """The 256^3 aneurysm workload in the benchmark's launch configuration,
    compared over its first 100 steps (the oracle is too slow for all 2000)."""
    prob = aneurysm_problem(256, q=27)
    _, _, e = run_both(lbm, prob, 100, "f32")
    assert e["u"] <= 1e-5, e


def test_full_size_aneurysm_384_f16(lbm):
    """The 384^3 aneurysm with FP16 deviation storage, first 60 steps."""
    prob = aneurysm_problem(384, q=27)
    _, _, e = run_both(lbm, prob, 60, "f16dev")
    assert e["u"] <= 1e-3, e


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("storage", ["f32"])
def test_periodic_random_porosity(lbm, q, storage):
    """Porosity gradients everywhere, including cells on the periodic faces
    (whose porosity neighbours wrap around), obstacles and a body force.
    FP32 only: in a closed box the porosity mass source drives rho away from 1,
    so the stored deviation is dominated by rho - 1 and 16-bit rounding of it is
    large against the small velocity of this case."""
    rng = np.random.default_rng(11)
    phi = (0.62 + 0.36 * rng.random((10, 11, 12))).astype(np.float32)
    rheo = lattice_rheology(0.08, 0.01, 60.0, 0.4, 2.0)
    prob = periodic_box_problem(12, 11, 10, q=q, rheology=rheo, body_force=(3e-5, -1e-5, 2e-5),
                                obstacles=40, phi=phi, d_p=2.5)
    _, _, e = run_both(lbm, prob, 150, storage)
    assert e["u"] <= TOL_U[storage], e


def test_mass_conservation_periodic(lbm):
    """Uniform porosity, periodic box with obstacles: sum f is conserved; the
    FP32 drift stays at round-off level."""
    rheo = lattice_rheology(0.1, 0.02, 20.0, 0.5, 2.0)
    prob = periodic_box_problem(40, 24, 20, q=27, phi_value=0.8, rheology=rheo, body_force=(2e-5, 0, 1e-5),
                                obstacles=300, d_p=3.0)
    sim = lbm.Simulation(prob)
    m0 = sim.diag()[0]
    sim.step(500)
    d = sim.diag()
    assert abs(d[0] - m0) < 1e-6 * m0
    assert d[7] == 0


def test_diag_matches_oracle(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob)
    sim.step(150)
    g = sim.diag(prob.region)
    o = Oracle(prob)
    o.step(150)
    r = o.diag(prob.region)
    assert abs(g[0] - r[0]) < 1e-6 * r[0]
    assert abs(g[1] - r[1]) < 1e-4 * r[1]
    assert abs(g[2] - r[2]) < 1e-4 * r[2]
    assert g[3] == r[3]
    assert abs(g[4] - r[4]) < 1e-5 * r[4]
    assert abs(g[5] - r[5]) < 1e-5 and abs(g[6] - r[6]) < 1e-5
    assert g[7] == 0


def test_moments_device_equals_host(lbm):
    prob = aneurysm_problem(24, q=19, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob)
    sim.step(37)
    h = sim.moments()
    d = sim.moments(on_device=True)
    for k in ("rho", "gdot", "omega"):
        assert np.array_equal(h[k], d[k].cpu().numpy())
    assert np.array_equal(h["u"], d["u"].cpu().numpy())


def test_inputs_on_device_and_determinism(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    a = lbm.Simulation(prob)
    b = lbm.Simulation(prob, inputs_on_device=True)
    a.step(80)
    b.step(80)
    ma, mb = a.moments(), b.moments()
    assert np.array_equal(ma["u"], mb["u"]) and np.array_equal(ma["rho"], mb["rho"])


def test_save_load_roundtrip(lbm):
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob, storage="f16dev")
    sim.step(40)
    buf = sim.save()
    sim.step(30)
    ref = sim.moments()
    sim.load_state(buf)
    assert sim.t == 40
    sim.step(30)
    again = sim.moments()
    assert np.array_equal(ref["u"], again["u"])
    assert np.array_equal(ref["omega"], again["omega"])


def test_empty_and_tiny_domains(lbm):
    prob = periodic_box_problem(4, 4, 4, q=27)
    prob.flags[:] = 0
    sim = lbm.Simulation(prob)
    assert sim.n_fluid == 0
    sim.step(3)
    assert np.all(sim.diag() == 0)
    prob = periodic_box_problem(4, 4, 4, q=19)
    prob.flags[:] = 0
    prob.flags[1, 2, 3] = 1
    sim = lbm.Simulation(prob)
    assert sim.n_fluid == 1
    sim.step(10)
    m = sim.moments()
    assert np.abs(m["u"]).max() == 0.0  # a single walled cell at rest stays at rest
    assert abs(sim.diag()[0] - 1.0) < 1e-6


def test_invalid_inputs_rejected(lbm):
    from lbm_inputs import aneurysm_problem as ap

    prob = ap(24, small=True)
    bad = prob.phi.copy()
    bad[prob.flags == 1] = 1.5
    prob2 = ap(24, small=True)
    prob2.phi = bad
    with pytest.raises(lbm.LBMError) as e:
        lbm.Simulation(prob2)
    assert e.value.status == lbm.LBM_EINVAL
    prob3 = ap(24, small=True)
    prob3.flags[5, 5, 5] = 3  # an outlet cell away from its face
    with pytest.raises(lbm.LBMError) as e:
        lbm.Simulation(prob3)
    assert e.value.status == lbm.LBM_EINVAL


def test_workspace_too_small(lbm):
    import torch

    prob = pipe_problem()
    g = lbm.make_grid(prob.dims, 19, "f32", prob.periodic)
    r, p, b = lbm.make_params(prob.rheology, prob.porous, prob.bc)
    need = lbm.lbm_workspace_size(g, lbm.lbm_list_length(g, np.ascontiguousarray(prob.flags).ctypes.data))
    ws = torch.empty(need - 4096, dtype=torch.uint8, device="cuda")
    flags = np.ascontiguousarray(prob.flags)
    phi = np.ascontiguousarray(prob.phi)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(g, flags.ctypes.data, phi.ctypes.data, 0, r, p, b, ws.data_ptr(), need - 4096,
                     torch.cuda.current_stream().cuda_stream)
    assert e.value.status == lbm.LBM_ENOMEM


def test_instability_check_from_host_injected_state(lbm):
    """A NaN written into a checkpoint on the host is caught by the periodic
    non-finite check (failure injected on the host, not on the device)."""
    prob = aneurysm_problem(24, q=27, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob)
    sim.step(5)
    buf = sim.save()
    f = buf[256:256 + 4 * 27 * 64].view(np.float32)
    f[:64] = np.nan  # rest populations of the first 64 packed slots
    sim.load_state(buf)
    lbm.lbm_set_check(sim.ctx, 2)
    with pytest.raises(lbm.LBMError) as e:
        sim.step(4)
    assert e.value.status == lbm.LBM_EUNSTABLE


def test_l2_window_leaves_results_unchanged(lbm):
    """The L2 residency window of the step launches changes where the per-slot
    words live, not what is computed: with and without it the fields agree
    bit for bit."""
    prob = aneurysm_problem(48, q=27, u0=0.05, period=100.0)
    a = lbm.Simulation(prob)
    b = lbm.Simulation(prob)
    assert lbm.lbm_l2_window_bytes(a.ctx) > 0
    lbm.lbm_set_l2_window(b.ctx, 0)
    assert lbm.lbm_l2_window_bytes(b.ctx) == 0
    a.step(50)
    b.step(50)
    lbm.lbm_set_l2_window(b.ctx, 1 << 20)
    assert 0 < lbm.lbm_l2_window_bytes(b.ctx) <= 1 << 20
    a.step(10)
    b.step(10)
    ma, mb = a.moments(), b.moments()
    for k in ("rho", "u", "gdot", "omega"):
        assert np.array_equal(ma[k], mb[k]), k
    a.close()
    b.close()
