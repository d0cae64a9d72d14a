"""Benchmark of the fused VANSE LBM step on GB300.

Workload: the synthetic 384^3 aneurysm (D3Q27, Carreau-Yasuda blood, porous
coil in the sac, pulsatile Zou-He inlet, pressure outlet), 1000 time steps per
benchmark step, distributions stored as FP32; the FP16 and BF16 deviation
storage variants are timed the same way and reported beside it with their
velocity error against the FP64 oracle.

One benchmark step = one 1000-time-step run of the workload.  The metric is
fluid-cell lattice updates per second (MLUPS) and the fraction of the measured
HBM copy bandwidth the step kernel reaches with its algorithmic bytes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica on its own GPU (independent
problems, no collective on the data path): weak scaling.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="aneurysm384", n=384, q=27, lbm_steps=1000, seed=0)
METRIC = "fluid MLUPS and % of HBM roofline, FP32 vs FP16-stored at stated error"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0  # the ~8 TB/s the workload states as the HBM roofline


def bytes_per_update(q, storage):
    """Algorithmic bytes per fluid-cell update: read and write every
    distribution once (2 Q s), read and write omega (8), read phi (4) and the
    link mask (4)."""
    s = 4 if storage == "f32" else 2
    return 2 * q * s + 16


def kernel_source_hash():
    """Hash of the sources and build flags the step kernel is compiled from (a
    stored traffic figure is only reported while they are unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2402_10809_gb300", "csrc")
    for fn in ("kernels.cuh", "lattice.cuh", "step.cu", os.path.join("..", "build.py")):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def load_traffic(name, storage):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary,
    only if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("kernel_hash") != kernel_source_hash():
        return None
    v = d.get("per_launch_bytes", {}).get(f"{name}_{storage}")
    return v


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    """(world size, rank, local rank, torch.distributed or None) from the
    launcher's environment; NCCL with GPUs, gloo without (host-side tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return ws, rank, local, dist
    return 1, 0, 0, None


def max_over_ranks(dist, value, device):
    """The largest value over all ranks, on every rank (the value itself
    without a process group): the timed region of the slowest replica."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size, fluid_cells, time_steps, seconds):
    """Whole-job fluid MLUPS: every rank advances its own replica of the
    workload (weak scaling), timed by the slowest rank."""
    return world_size * fluid_cells * time_steps / seconds / 1e6


def flush_l2(torch, buf):
    buf.fill_(1.0)


def time_variant(torch, lbm, prob, storage, steps, warmup, lbm_steps, flush, setup=None):
    sim = lbm.Simulation(prob, storage=storage)
    if setup is not None:
        setup(sim)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush_l2(torch, flush)
        sim.step(lbm_steps)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush_l2(torch, flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(lbm_steps)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return sim, times


def run_ours(args):
    import torch

    ws, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    from lbm_inputs import aneurysm_problem
    from paper_2402_10809_gb300 import lbm

    lbm.load()
    n = args.n
    name = f"aneurysm{n}"
    prob = aneurysm_problem(n, q=WORKLOAD["q"], seed=WORKLOAD["seed"])
    nf = prob.n_fluid
    L = args.lbm_steps
    st0 = args.storage
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    peak, peak_kind = load_peaks()

    # ---- timed region: FP32 storage (the headline), barrier + sync on both sides
    sim, _ = time_variant(torch, lbm, prob, st0, 0, args.warmup, L, flush)
    for _ in range(args.warmup):
        flush_l2(torch, flush)
        sim.step(L)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    per = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(torch, flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(L)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total = max_over_ranks(dist, sum(per), "cuda")
    clocks = clk.summary()
    launch_s = total / (args.steps * L)  # average step-kernel launch duration (back-to-back launches)
    mlups = job_throughput(ws, nf, L * args.steps, total)
    bpu = bytes_per_update(WORKLOAD["q"], st0)
    achieved = bpu * nf / launch_s / 1e9
    traffic = load_traffic(name, st0)

    # ---- storage variants, same protocol
    variants = {}
    for st in () if args.no_variants else [v for v in ("f32", "f16dev", "bf16dev") if v != st0]:
        s2, tv = time_variant(torch, lbm, prob, st, max(3, args.steps // 2), args.warmup, L, flush)
        tv_mean = sum(tv) / len(tv)
        b2 = bytes_per_update(WORKLOAD["q"], st)
        variants[st] = {"value": nf * L / tv_mean / 1e6, "unit": UNIT,
                        "roofline_frac": b2 * nf / (tv_mean / L) / 1e9 / peak,
                        "roofline_frac_nominal": b2 * nf / (tv_mean / L) / 1e9 / NOMINAL_HBM_GBS,
                        "bytes_per_update": b2, "traffic": load_traffic(name, st)}
        s2.close()

    # ---- end to end through the C ABI with host buffers (pinned), per step:
    # H2D of flags + porosity + region, set-up, L time steps, D2H of diagnostics
    e2e = None
    if not args.no_e2e:
        pin_flags = torch.from_numpy(np.ascontiguousarray(prob.flags)).pin_memory()
        pin_phi = torch.from_numpy(np.ascontiguousarray(prob.phi)).pin_memory()
        pin_reg = torch.from_numpy(np.ascontiguousarray(prob.region)).pin_memory()
        grid = lbm.make_grid(prob.dims, prob.q, st0, prob.periodic)
        r, p, b = lbm.make_params(prob.rheology, prob.porous, prob.bc)
        nbytes = lbm.lbm_workspace_size(grid, lbm.lbm_list_length(grid, pin_flags.data_ptr()))
        wsb = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        sh = stream.cuda_stream

        def e2e_step():
            ctx = lbm.lbm_init(grid, pin_flags.data_ptr(), pin_phi.data_ptr(), 0, r, p, b, wsb.data_ptr(), nbytes, sh)
            lbm.lbm_step(ctx, L)
            d = lbm.lbm_diag(ctx, pin_reg.data_ptr(), 0)
            lbm.lbm_destroy(ctx)
            return d

        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ne = max(2, args.steps // 2)
        for _ in range(ne):
            flush_l2(torch, flush)
            e2e_step()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": nf * L * ne / te / 1e6 * ws, "unit": UNIT,
               "h2d_bytes_per_step": int(prob.flags.nbytes + prob.phi.nbytes + prob.region.nbytes),
               "d2h_bytes_per_step": 64}

    line = {
        "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{name} D3Q27 {st0}-stored, {L} time steps per step, "
                               f"{nf} fluid cells, Carreau-Yasuda (lambda {prob.rheology['lam'] * 1e3:g} ms), "
                               f"porous sac, pulsatile inlet",
                   "box": [n] * 3, "fluid_cells": nf, "time_steps_per_step": L,
                   "q": WORKLOAD["q"], "storage": st0, "parallelism": f"replicas{ws}",
                   "l2": f"{bpu * nf / 1e6:.0f} MB touched per time step and a 256 MB L2 flush "
                         "before each timed step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "nominal_peak": NOMINAL_HBM_GBS, "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_update": bpu,
                     "kernel": f"lbm_kernel<27,{st0},step> average over back-to-back launches"},
        "storage_variants": variants,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": args.steps * L,
    }
    if rank == 0:
        line["wall_shear"] = wall_shear_pass(torch, lbm, sim, prob, stream)
    if rank == 0 and not args.no_aniso:
        line["anisotropic"] = aniso_cost(torch, lbm, prob, args, flush, mlups / ws)
    if rank == 0 and not args.no_slabs:
        line["slabs_one_gpu"] = slab_overhead(torch, lbm, prob, args, flush, mlups / ws)
    if rank == 0 and not args.no_config2:
        line["config1"] = config1_throughput(torch, lbm, args, flush)
        line["config2"] = config2_throughput(torch, lbm, args, flush)
    if rank == 0 and not args.no_adjoint:
        line["adjoint"] = adjoint_cost(torch, lbm, args, args.adjoint_n)
        if args.adjoint_n2 > 0:
            line["adjoint_large"] = adjoint_cost(torch, lbm, args, args.adjoint_n2)
    if rank == 0 and not args.no_coil:
        line["coil"] = coil_study(torch, lbm, args)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(prob, sim_factory=lambda st: lbm.Simulation(prob, storage=st),
                                            sample_steps=args.cpu_sample_steps, error_steps=args.error_steps)
    sim.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


ADJOINT = dict(name="aneurysm128", n=128, q=27, T=500, K=50, seed=0)
# Algorithmic bytes of one reverse fluid-cell update (D3Q27, FP32): pull of
# S(t-1), lambda(t) read, lambda(t-1) write (3 x 108), omega 4, mu read + write
# 8, phi 4, mask 4, rho - 1 gather 4, dJ/dphi read-modify-write 16.
ADJOINT_BYTES_PER_UPDATE = 364
L2_BYTES = 129e6  # GB300 L2 cache


def adjoint_cost(torch, lbm, args, n):
    """Cost of lbm_adjoint (forward with checkpoints, segment replays, reverse
    sweep) on the n^3 aneurysm, T = 500 steps, checkpoint every K = 50 steps,
    against T forward steps of the same problem; both timed with CUDA events on
    the launching stream.  A second figure keeps the whole trajectory (K = T,
    no replay) when the device has room for it; from it, the reverse step
    alone.  Its HBM fraction is reported only where the reverse step's bytes
    exceed the L2 cache (at 128^3 its working set stays in L2)."""
    from lbm_inputs import aneurysm_problem

    prob = aneurysm_problem(n, q=ADJOINT["q"], seed=ADJOINT["seed"])
    T, K = args.adjoint_T, args.adjoint_K
    sim = lbm.Simulation(prob)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        out = None
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return min(ts), out

    for _ in range(args.warmup):
        sim.step(T)
    t_fwd, _ = timed(lambda: sim.step(T), 3)
    reg = np.ascontiguousarray(prob.region, dtype=np.uint8)
    grad = torch.empty(prob.flags.shape, dtype=torch.float64, device="cuda")
    res = {"workload": f"aneurysm{n} D3Q27 FP32, {prob.n_fluid} fluid cells, J = time-and-sac mean of "
                       f"rho|u|^2/2 over steps 1..{T}, gradient w.r.t. porosity",
           "T": T, "forward_s": t_fwd, "forward_step_us": 1e6 * t_fwd / T}
    variants = [("checkpointed", K)] + ([] if args.no_full_history else [("full_history", T)])
    for name, k in variants:
        nbytes = lbm.lbm_adjoint_workspace_size(sim.ctx, T, k)
        free, _ = torch.cuda.mem_get_info()
        if nbytes > 0.8 * free:
            res[name] = {"K": k, "skipped": f"needs {nbytes / 1e9:.1f} GB"}
            continue
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        run = lambda: lbm.lbm_adjoint(sim.ctx, T, k, 0, reg.ctypes.data, 0, ws.data_ptr(), nbytes, grad.data_ptr())
        run()
        t_adj, J = timed(run, 3)
        res[name] = {"K": k, "seconds": t_adj, "cost_vs_forward": t_adj / t_fwd, "J": J,
                     "workspace_gb": nbytes / 1e9}
        if k >= T:
            # no replay: the reverse sweep is the adjoint time minus the T forward steps
            t_rev = (t_adj - t_fwd) / (T + 1)
            peak, _ = load_peaks()
            bytes_rev = ADJOINT_BYTES_PER_UPDATE * prob.n_fluid
            res[name].update({"reverse_step_us": 1e6 * t_rev, "reverse_vs_forward_step": t_rev / (t_fwd / T),
                              "reverse_bytes_per_update": ADJOINT_BYTES_PER_UPDATE,
                              "reverse_bytes_per_step": bytes_rev})
            if bytes_rev > L2_BYTES:
                res[name]["reverse_roofline_frac"] = bytes_rev / t_rev / 1e9 / peak
        del ws
    sim.close()
    return res


def aniso_cost(torch, lbm, prob, args, flush, iso_value):
    """Cost of the anisotropic velocity solve (Sec. 3 remark: fixed-point
    iteration with a 3x3 solve per step) against the explicit solve of the
    headline, on the same workload and protocol (warm-up, L2 flush, CUDA
    events): the porous sac gets a seeded coil shape tensor (wire direction
    field, 4 times more permeable along the wire; lbm_inputs.coil_shape_tensor),
    the rest of the box S = Id.  Algorithmic bytes per porous cell update rise
    by 48 (A - Id and B, 12 floats)."""
    from lbm_inputs import coil_shape_tensor

    por = (prob.phi < 1) & (prob.flags > 0)
    idx = np.nonzero(por)
    lo = [int(a.min()) for a in idx]
    hi = [int(a.max()) + 1 for a in idx]
    S = np.zeros((6,) + prob.flags.shape, np.float32)
    S[:3] = 1.0
    S[:, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = coil_shape_tensor(tuple(h - l for l, h in zip(lo, hi)),
                                                                      ratio=4.0, seed=0)
    iters, tol = 16, 1e-6
    L = args.lbm_steps
    sim, tv = time_variant(torch, lbm, prob, "f32", max(3, args.steps // 2), args.warmup, L, flush,
                           setup=lambda s: s.set_anisotropy(S, max_iter=iters, tol=tol))
    finite = bool(sim.diag()[7] == 0)
    sim.close()
    nf, npor = prob.n_fluid, int(por.sum())
    t = sum(tv) / len(tv)
    value = nf * L / t / 1e6
    bpu = bytes_per_update(WORKLOAD["q"], "f32") + 48.0 * npor / nf
    peak, _ = load_peaks()
    return {"value": value, "unit": UNIT, "vs_explicit": value / iso_value, "porous_cells": npor,
            "max_iter": iters, "tol": tol, "bytes_per_update": bpu,
            "roofline_frac": bpu * nf * L / t / 1e9 / peak, "finite": finite}


def wall_shear_pass(torch, lbm, sim, prob, stream):
    """One pass of the voxel wall-shear-stress proxy (lbm_wall_shear, device
    output) on the benchmark state: CUDA events around 5 passes, best taken.
    Algorithmic bytes: the dense output (4 N, cleared and written), the slot
    masks (4 n_store) and, per wall cell, its populations plus porosity, rate
    and row id (Q s + 12)."""
    out = torch.empty(prob.flags.shape, dtype=torch.float32, device="cuda")
    lbm.lbm_wall_shear(sim.ctx, out.data_ptr(), 1)
    best = 1e9
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lbm.lbm_wall_shear(sim.ctx, out.data_ptr(), 1)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    n_wall = int((out > 0).sum().item())
    n_store = lbm.lbm_list_length(sim.grid, np.ascontiguousarray(prob.flags).ctypes.data)
    nbytes = 4 * prob.flags.size + 4 * n_store + n_wall * (prob.q * 4 + 12)
    peak, _ = load_peaks()
    return {"pass_us": 1e6 * best, "wall_cells": n_wall, "algorithmic_bytes": nbytes,
            "roofline_frac": nbytes / best / 1e9 / peak, "unit": "lattice stress |tau|",
            "max_wss": float(out.max().item())}


COIL_PACKINGS = (0.15, 0.20, 0.25)


def porosity_average_cost(torch, lbm, wire_t, flags_t, stream, reps=5):
    """The volume averaging of a coil on the GPU (lbm_porosity_average, three
    sliding-window passes) at the coil study's box: median CUDA-event time over
    `reps` calls after 3 warm-up calls on the launching stream (wire, flags and
    porosity together exceed L2).  Algorithmic bytes: wire + flags read, FP32
    porosity written = 6 B per cell."""
    from lbm_inputs import COIL_PHI_MIN, COIL_WINDOW

    nz, ny, nx = wire_t.shape
    nbytes = lbm.lbm_porosity_workspace_size(nx, ny, nz)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    phi = torch.empty(tuple(wire_t.shape), dtype=torch.float32, device="cuda")

    def call():
        lbm.lbm_porosity_average(nx, ny, nz, wire_t.data_ptr(), flags_t.data_ptr(), COIL_WINDOW, COIL_PHI_MIN,
                                 phi.data_ptr(), ws.data_ptr(), nbytes, stream.cuda_stream)

    for _ in range(3):
        call()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e3)
    us = float(np.median(times))
    alg = 6 * wire_t.numel()
    peak, kind = load_peaks()
    return {"cells": int(wire_t.numel()), "window": COIL_WINDOW, "us": us, "kernel_launches": 3,
            "algorithmic_bytes": int(alg), "achieved_gbs": alg / us / 1e3, "peak_gbs": peak,
            "roofline_frac": (alg / us / 1e3) / peak, "peak_kind": kind}


def coil_study(torch, lbm, args):
    """The fully resolved vs volume-averaged coil (Sec. 4) at the largest size:
    the n^3 aneurysm without coil, then for each packing density of the paper
    (15, 20, 25 % of the sac) a seeded random-walk wire (2 voxels thick; the
    lower packings are the first part of the same walk) as solid voxels, and the
    same wire averaged into porosity over the paper's window (28^3 cells) on the
    GPU (lbm_porosity_average), and over the 8^3 window of the workload
    statement as written (`averaged_window8`).  FP32, pulsatile inflow.  Throughput from CUDA
    events around the time steps (the diagnostic launches are outside the timed
    chunks); the sac-mean |u| over the fluid cells of the sac and over its whole
    volume (wire voxels count as u = 0), and the mean wall shear stress
    (lbm_wall_shear) over the sac wall (the fluid cells of the sac next to the
    vessel wall of the uncoiled geometry, so that the coil's own surface is left
    out), each averaged over the last 1000 steps; their ratios to the uncoiled
    case and of averaged to resolved."""
    from scipy.ndimage import binary_dilation

    from lbm_inputs import COIL_PHI_MIN, COIL_WINDOW, aneurysm_problem, coil_packings, coil_problem

    n, steps, every, last = args.coil_n, args.coil_steps, 100, 1000
    base = aneurysm_problem(n, porous_sac=False)
    wires = coil_packings(n, COIL_PACKINGS)
    sac_wall = (base.region > 0) & (base.flags > 0) & binary_dilation(base.flags == 0, np.ones((3, 3, 3), bool))
    sac_wall_t = torch.from_numpy(sac_wall).to("cuda")
    flags_t = torch.from_numpy(np.ascontiguousarray(base.flags)).to("cuda")
    n_region = float((base.region > 0).sum())
    wss = torch.empty(sac_wall.shape, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {"workload": f"aneurysm{n} D3Q27 FP32, {steps} pulsatile steps; wire coils at "
                       + "/".join(f"{round(100 * p)}" for p in COIL_PACKINGS)
                       + f" % of the sac, fully resolved and volume averaged over {COIL_WINDOW}^3 cells",
           "steps": steps}

    def run(prob):
        sim = lbm.Simulation(prob)
        sim.step(every)  # warm-up chunk, not timed
        t_run, u_sum, v_sum, w_sum, k, bad = 0.0, 0.0, 0.0, 0.0, 0, 0.0
        wall = sac_wall_t & (flags_t > 0) if prob.flags is base.flags else \
            sac_wall_t & torch.from_numpy(prob.flags > 0).to("cuda")
        for _ in range(steps // every - 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(every)
            e1.record(stream)
            e1.synchronize()
            t_run += e0.elapsed_time(e1) / 1e3
            if sim.t > steps - last:
                d = sim.diag(prob.region)
                u_sum += d[2] / max(d[3], 1.0)
                v_sum += d[2] / n_region
                lbm.lbm_wall_shear(sim.ctx, wss.data_ptr(), 1)
                w_sum += float(wss[wall].mean().item())
                bad = max(bad, d[7])
                k += 1
        timed_steps = (steps // every - 1) * every
        n_fluid = sim.n_fluid
        sim.close()
        def fin(v):  # a state that lost finiteness has no averages (JSON has no NaN)
            v = float(v)
            return v if np.isfinite(v) and bad == 0 else None

        return {"fluid_cells": int(n_fluid),
                "value": float(n_fluid * timed_steps / t_run / 1e6) if t_run > 0 else None, "unit": UNIT,
                "sac_mean_u": fin(u_sum / max(k, 1)), "sac_volume_mean_u": fin(v_sum / max(k, 1)),
                "sac_wall_mean_wss": fin(w_sum / max(k, 1)), "sac_wall_cells": int(wall.sum().item()),
                "finite": bool(bad == 0)}

    keys = ("sac_mean_u", "sac_volume_mean_u", "sac_wall_mean_wss")
    res["uncoiled"] = run(base)
    res["porosity_average"] = porosity_average_cost(
        torch, lbm, torch.from_numpy(wires[max(COIL_PACKINGS)]).to("cuda"), flags_t, stream)
    for p in COIL_PACKINGS:
        wire_t = torch.from_numpy(wires[p]).to("cuda")
        phi_t = lbm.porosity_average(wire_t, COIL_WINDOW, COIL_PHI_MIN, flags_t)
        r = {"packing": p, "wire_voxels": int(wires[p].sum()),
             "resolved": run(coil_problem(n, True, wire=wires[p], base=base)),
             "averaged": run(coil_problem(n, False, phi=phi_t, base=base))}
        r["averaged"]["min_porosity"] = float(phi_t[flags_t > 0].min().item())
        # the 8^3 window of the workload statement, as written (steps of an
        # eighth of the porosity between neighbouring cells; see `finite`)
        phi8 = lbm.porosity_average(wire_t, 8, COIL_PHI_MIN, flags_t)
        r["averaged_window8"] = run(coil_problem(n, False, phi=phi8, base=base))
        r["averaged_window8"]["min_porosity"] = float(phi8[flags_t > 0].min().item())
        del phi8
        def ratio(a, b):
            return a / b if a is not None and b else None

        for case in ("resolved", "averaged", "averaged_window8"):
            for key in keys:
                r[case][key + "_ratio"] = ratio(r[case][key], res["uncoiled"][key])
        r["averaged_over_resolved"] = {key: ratio(r["averaged"][key], r["resolved"][key]) for key in keys}
        res[f"packing_{round(100 * p)}"] = r
        del wire_t, phi_t
    return res


def cpu_baseline(prob, sim_factory=None, sample_steps=30, error_steps=1000):
    """The FP64 oracle timed on the host cores on a bounded sample (the first
    sample_steps time steps of the same workload).  When a GPU factory is
    given, the same oracle run continues to error_steps and every storage
    type is compared with it after the same number of steps: the largest
    velocity and shear-rate deviation over the fluid cells relative to the
    oracle's largest value, the relative L2 velocity deviation, and the mass
    drift (M(T) - M(0)) / M(0) of the GPU run beside the oracle's (the porosity
    term of Sec. 3 and the open boundaries make the mass change; both sides
    must change it alike)."""
    from oracle.oracle import Oracle, num_threads

    o = Oracle(prob)
    m0_ref = o.diag()[0]
    t0 = time.perf_counter()
    o.step(sample_steps)
    dt = time.perf_counter() - t0
    out = {"value": prob.n_fluid * sample_steps / dt / 1e6, "unit": UNIT, "cores": num_threads(),
           "kind": "oracle",
           "sample": f"first {sample_steps} time steps of {WORKLOAD['name']} (D3Q27), FP64, OpenMP"}
    if sim_factory is not None:
        steps = max(error_steps, sample_steps)
        o.step(steps - sample_steps)
        r = o.moments()
        drift_ref = (o.diag()[0] - m0_ref) / m0_ref
        o.close()
        fl = prob.flags > 0
        den = np.abs(r["u"][:, fl]).max()
        gd = np.abs(r["gdot"][fl]).max()
        l2 = np.sqrt((r["u"][:, fl] ** 2).sum())
        errs = {}
        for st in ("f32", "f16dev", "bf16dev"):
            s = sim_factory(st)
            m0 = s.diag()[0]
            s.step(steps)
            drift = (s.diag()[0] - m0) / m0
            g = s.moments()
            errs[st] = {"u_max_rel": float(np.abs(g["u"][:, fl] - r["u"][:, fl]).max() / den),
                        "u_l2_rel": float(np.sqrt(((g["u"][:, fl] - r["u"][:, fl]) ** 2).sum()) / l2),
                        "gdot_max_rel": float(np.abs(g["gdot"][fl] - r["gdot"][fl]).max() / gd),
                        "mass_drift": float(drift), "mass_drift_oracle": float(drift_ref),
                        "after_steps": steps}
            s.close()
        out["error_vs_oracle"] = errs
        out["error_vs_oracle_pipe"] = pipe_error()
    return out


def pipe_error(steps=200):
    """The 32x32x64 D3Q19 pipe (Carreau-Yasuda, porous plug, body force,
    periodic in z) after its 200 steps on the GPU (FP32 storage) against the
    oracle: largest velocity and shear-rate deviation over the fluid cells
    relative to the oracle's largest value."""
    from lbm_inputs import pipe_problem
    from oracle.oracle import Oracle
    from paper_2402_10809_gb300 import lbm

    prob = pipe_problem(q=19)
    o = Oracle(prob)
    o.step(steps)
    r = o.moments()
    o.close()
    s = lbm.Simulation(prob, storage="f32")
    s.step(steps)
    g = s.moments()
    s.close()
    fl = prob.flags > 0
    return {"workload": f"pipe 32x32x64 D3Q19 f32-stored, {steps} steps",
            "u_max_rel": float(np.abs(g["u"][:, fl] - r["u"][:, fl]).max() / np.abs(r["u"][:, fl]).max()),
            "gdot_max_rel": float(np.abs(g["gdot"][fl] - r["gdot"][fl]).max() / np.abs(r["gdot"][fl]).max())}


def slab_overhead(torch, lbm, prob, args, flush, unsharded):
    """The headline workload split into z-slabs on this one GPU (the
    decomposition a box too large for one GPU would use across GPUs): the
    slabs' step kernels plus one face-exchange launch per face and time step;
    CUDA events around args.lbm_steps time steps after a warm-up run."""
    from paper_2402_10809_gb300 import slabs

    res = {}
    stream = torch.cuda.current_stream()
    for ns in (2, 4):
        sl = slabs.SlabSimulation(prob, ns, storage="f32")
        sl.step(args.lbm_steps)
        ts = []
        for _ in range(3):
            flush_l2(torch, flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sl.step(args.lbm_steps)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        finite = bool(sl.diag()[7] == 0)
        sl.close()
        v = prob.n_fluid * args.lbm_steps / min(ts) / 1e6
        res[f"slabs{ns}"] = {"value": v, "unit": UNIT, "vs_unsharded": v / unsharded, "bounds": sl.bounds,
                             "finite": finite}
    return res


def config1_throughput(torch, lbm, args, flush):
    """The 32x32x64 D3Q19 pipe (FP32) over its 200 time steps as one timed
    run after a warm-up run, L2 flushed before each; a box this small is
    bound by the launches, not by HBM."""
    from lbm_inputs import pipe_problem

    prob = pipe_problem(q=19)
    L = 200
    sim, tv = time_variant(torch, lbm, prob, "f32", 3, 1, L, flush)
    finite = bool(sim.diag()[7] == 0)
    sim.close()
    t = min(tv)
    return {"workload": f"pipe 32x32x64 D3Q19 f32-stored, {L} time steps, {prob.n_fluid} fluid cells",
            "value": prob.n_fluid * L / t / 1e6, "unit": UNIT, "seconds": t, "us_per_step": 1e6 * t / L,
            "finite": finite}


def config2_throughput(torch, lbm, args, flush):
    """The 256^3 aneurysm (FP32, D3Q27) over its 2000 time steps as one timed
    run after a warm-up run, L2 flushed before each (CUDA events on the
    launching stream)."""
    from lbm_inputs import aneurysm_problem

    prob = aneurysm_problem(256, q=27, seed=0)
    L = 2000
    sim, tv = time_variant(torch, lbm, prob, "f32", 2, 1, L, flush)
    finite = bool(sim.diag()[7] == 0)
    sim.close()
    t = min(tv)
    peak, _ = load_peaks()
    bpu = bytes_per_update(27, "f32")
    return {"workload": f"aneurysm256 D3Q27 f32-stored, {L} time steps, {prob.n_fluid} fluid cells",
            "value": prob.n_fluid * L / t / 1e6, "unit": UNIT, "seconds": t,
            "roofline_frac": bpu * prob.n_fluid * L / t / 1e9 / peak,
            "roofline_frac_nominal": bpu * prob.n_fluid * L / t / 1e9 / NOMINAL_HBM_GBS, "finite": finite}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from lbm_inputs import aneurysm_problem
    from oracle.oracle import Oracle, num_threads

    prob = aneurysm_problem(WORKLOAD["n"], q=WORKLOAD["q"], seed=WORKLOAD["seed"])
    nf = prob.n_fluid
    o = Oracle(prob)
    per = args.ref_sample_steps
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per)
    dt = time.perf_counter() - t0
    v = nf * per * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD['name']} D3Q27, each step a bounded sample of {per} time steps",
                       "box": [WORKLOAD["n"]] * 3, "fluid_cells": nf, "q": WORKLOAD["q"],
                       "time_steps_per_step": per,
                       "note": f"the oracle advances {per} time steps per bench step where the GPU arm advances "
                               f"{WORKLOAD['lbm_steps']}; both report fluid-cell updates per second"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": num_threads(), "kind": "oracle",
                             "sample": f"{per} time steps per step of {WORKLOAD['name']}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lbm-steps", type=int, default=WORKLOAD["lbm_steps"])
    ap.add_argument("--cpu-sample-steps", type=int, default=30)
    ap.add_argument("--error-steps", type=int, default=WORKLOAD["lbm_steps"],
                    help="time steps after which every storage type is compared with the oracle")
    ap.add_argument("--no-config2", action="store_true", help="skip the pipe (200 steps) and 256^3 (2000 steps) throughputs")
    ap.add_argument("--no-slabs", action="store_true", help="skip the z-slab split on one GPU")
    ap.add_argument("--adjoint-n2", type=int, default=256, help="second adjoint box (0: none)")
    ap.add_argument("--ref-sample-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the other storage types")
    ap.add_argument("--no-full-history", action="store_true", help="skip the adjoint with K = T")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"], help="aneurysm box edge")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16dev", "bf16dev"])
    ap.add_argument("--no-coil", action="store_true", help="skip the resolved / averaged coil study")
    ap.add_argument("--no-aniso", action="store_true", help="skip the anisotropic-permeability cost")
    ap.add_argument("--coil-n", type=int, default=512)
    ap.add_argument("--coil-steps", type=int, default=5000)
    ap.add_argument("--adjoint-n", type=int, default=ADJOINT["n"])
    ap.add_argument("--adjoint-T", type=int, default=ADJOINT["T"])
    ap.add_argument("--adjoint-K", type=int, default=ADJOINT["K"])
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: warm-up raised to 3 (timing rule)", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
