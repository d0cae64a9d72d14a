"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

Every compute step runs in the CUDA kernels of liblbm.so.  PyTorch provides the
device workspace and the stream.  The binding fails loudly when the library is
missing or cannot be loaded; there is no CPU fallback.
"""

import ctypes as C
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE = range(6)
LBM_SOLID, LBM_FLUID, LBM_INLET, LBM_OUTLET = range(4)
LBM_F32, LBM_F16DEV, LBM_BF16DEV = range(3)
STORAGE = {"f32": LBM_F32, "f16dev": LBM_F16DEV, "bf16dev": LBM_BF16DEV}
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EUNSTABLE", 5: "LBM_ESTATE"}

# Symbols include/lbm.h declares (checked by the tests).
SYMBOLS = ["lbm_list_length", "lbm_workspace_size", "lbm_init", "lbm_step", "lbm_moments", "lbm_diag", "lbm_diag_noalloc",
           "lbm_set_check",
           "lbm_state_size", "lbm_save", "lbm_load", "lbm_time", "lbm_fluid_count", "lbm_last_error",
           "lbm_destroy", "lbm_adjoint_workspace_size", "lbm_adjoint", "lbm_wall_shear",
           "lbm_porosity_workspace_size", "lbm_porosity_average", "lbm_anisotropy_buffer_size",
           "lbm_set_anisotropy", "lbm_slab_bounds", "lbm_plane_slots", "lbm_set_halo", "lbm_halo_message_size",
           "lbm_halo_pack", "lbm_halo_unpack", "lbm_halo_exchange", "lbm_set_l2_window",
           "lbm_l2_window_bytes", "lbm_set_l2_group", "lbm_step_slabs"]


class lbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("q", C.c_int32),
                ("storage", C.c_int32), ("periodic", C.c_int32 * 3)]


class lbm_rheology(C.Structure):
    _fields_ = [("mu0", C.c_double), ("mu_inf", C.c_double), ("lambda_", C.c_double), ("n", C.c_double),
                ("a", C.c_double), ("rho0", C.c_double), ("dx", C.c_double), ("dt", C.c_double)]


class lbm_porous(C.Structure):
    _fields_ = [("d_p", C.c_double), ("k_const", C.c_double), ("nu_darcy", C.c_double),
                ("forchheimer", C.c_int32)]


class lbm_bc(C.Structure):
    _fields_ = [("body_force", C.c_double * 3), ("inlet_axis", C.c_int32), ("inlet_side", C.c_int32),
                ("inlet_center", C.c_double * 3), ("inlet_radius", C.c_double), ("u0", C.c_double),
                ("amp", C.c_double), ("period", C.c_double), ("ramp_steps", C.c_double),
                ("outlet_axis", C.c_int32), ("outlet_side", C.c_int32), ("rho_out", C.c_double)]


_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Loads liblbm.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build()")
    L = C.CDLL(path)
    P, vp = C.POINTER, C.c_void_p
    L.lbm_list_length.restype = C.c_int64
    L.lbm_list_length.argtypes = [P(lbm_grid), vp]
    L.lbm_workspace_size.restype = C.c_size_t
    L.lbm_workspace_size.argtypes = [P(lbm_grid), C.c_int64]
    L.lbm_init.restype = C.c_int
    L.lbm_init.argtypes = [P(vp), P(lbm_grid), vp, vp, C.c_int32, P(lbm_rheology), P(lbm_porous), P(lbm_bc),
                           vp, C.c_size_t, vp]
    L.lbm_step.restype = C.c_int
    L.lbm_step.argtypes = [vp, C.c_int32]
    L.lbm_moments.restype = C.c_int
    L.lbm_moments.argtypes = [vp, vp, vp, vp, vp, C.c_int32]
    L.lbm_diag.restype = C.c_int
    L.lbm_diag.argtypes = [vp, vp, C.c_int32, P(C.c_double)]
    L.lbm_diag_noalloc.restype = C.c_int
    L.lbm_diag_noalloc.argtypes = [vp, vp, P(C.c_double)]
    L.lbm_set_check.restype = C.c_int
    L.lbm_set_check.argtypes = [vp, C.c_int32]
    L.lbm_state_size.restype = C.c_size_t
    L.lbm_state_size.argtypes = [vp]
    L.lbm_save.restype = C.c_int
    L.lbm_save.argtypes = [vp, vp, C.c_size_t, C.c_int32]
    L.lbm_load.restype = C.c_int
    L.lbm_load.argtypes = [vp, vp, C.c_size_t, C.c_int32]
    L.lbm_time.restype = C.c_int64
    L.lbm_time.argtypes = [vp]
    L.lbm_fluid_count.restype = C.c_int64
    L.lbm_fluid_count.argtypes = [vp]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_last_error.argtypes = [vp]
    L.lbm_wall_shear.restype = C.c_int
    L.lbm_wall_shear.argtypes = [vp, vp, C.c_int32]
    L.lbm_adjoint_workspace_size.restype = C.c_size_t
    L.lbm_adjoint_workspace_size.argtypes = [vp, C.c_int32, C.c_int32]
    L.lbm_adjoint.restype = C.c_int
    L.lbm_adjoint.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, vp, C.c_int32, vp, C.c_size_t, vp, P(C.c_double)]
    L.lbm_anisotropy_buffer_size.restype = C.c_size_t
    L.lbm_anisotropy_buffer_size.argtypes = [vp]
    L.lbm_set_anisotropy.restype = C.c_int
    L.lbm_set_anisotropy.argtypes = [vp, vp, vp, C.c_size_t, C.c_int32, C.c_float]
    L.lbm_porosity_workspace_size.restype = C.c_size_t
    L.lbm_porosity_workspace_size.argtypes = [C.c_int32, C.c_int32, C.c_int32]
    L.lbm_porosity_average.restype = C.c_int
    L.lbm_porosity_average.argtypes = [C.c_int32, C.c_int32, C.c_int32, vp, vp, C.c_int32, C.c_float, vp, vp,
                                       C.c_size_t, vp]
    L.lbm_slab_bounds.restype = C.c_int
    L.lbm_slab_bounds.argtypes = [P(lbm_grid), vp, C.c_int32, P(C.c_int32)]
    L.lbm_plane_slots.restype = C.c_int
    L.lbm_plane_slots.argtypes = [P(lbm_grid), vp, C.c_int32, P(C.c_int64), P(C.c_int64)]
    L.lbm_set_halo.restype = C.c_int
    L.lbm_set_halo.argtypes = [vp, C.c_int32, C.c_int32]
    L.lbm_halo_message_size.restype = C.c_size_t
    L.lbm_halo_message_size.argtypes = [vp, C.c_int32]
    L.lbm_halo_pack.restype = C.c_int
    L.lbm_halo_pack.argtypes = [vp, C.c_int32, vp]
    L.lbm_halo_unpack.restype = C.c_int
    L.lbm_halo_unpack.argtypes = [vp, C.c_int32, vp]
    L.lbm_halo_exchange.restype = C.c_int
    L.lbm_halo_exchange.argtypes = [vp, vp]
    L.lbm_set_l2_window.restype = C.c_int
    L.lbm_set_l2_window.argtypes = [vp, C.c_int64]
    L.lbm_l2_window_bytes.restype = C.c_int64
    L.lbm_l2_window_bytes.argtypes = [vp]
    L.lbm_set_l2_group.restype = C.c_int
    L.lbm_set_l2_group.argtypes = [vp, C.c_int64]
    L.lbm_step_slabs.restype = C.c_int
    L.lbm_step_slabs.argtypes = [C.POINTER(vp), C.c_int32, C.c_int32, vp]
    L.lbm_destroy.restype = None
    L.lbm_destroy.argtypes = [vp]
    _lib = L
    return L


def _check(ctx, status):
    if status != LBM_OK:
        msg = load().lbm_last_error(ctx).decode() if ctx else ""
        raise LBMError(status, msg)


# ----------------------------------------------------------------- structs

def make_grid(dims, q, storage, periodic):
    g = lbm_grid()
    g.nx, g.ny, g.nz = dims
    g.q = q
    g.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    g.periodic = (C.c_int32 * 3)(*[int(p) for p in periodic])
    return g


def make_params(rheology, porous, bc):
    r = lbm_rheology(rheology["mu0"], rheology["mu_inf"], rheology["lam"], rheology["n"], rheology["a"],
                     rheology["rho0"], rheology["dx"], rheology["dt"])
    p = lbm_porous(porous["d_p"], porous["k_const"], porous["nu_darcy"], int(porous["forchheimer"]))
    b = lbm_bc()
    b.body_force = (C.c_double * 3)(*bc["body_force"])
    b.inlet_axis, b.inlet_side = bc["inlet_axis"], bc["inlet_side"]
    b.inlet_center = (C.c_double * 3)(*bc["inlet_center"])
    b.inlet_radius, b.u0, b.amp = bc["inlet_radius"], bc["u0"], bc["amp"]
    b.period, b.ramp_steps = bc["period"], bc["ramp_steps"]
    b.outlet_axis, b.outlet_side, b.rho_out = bc["outlet_axis"], bc["outlet_side"], bc["rho_out"]
    return r, p, b


# ----------------------------------------------------------------- C ABI, same names

def lbm_list_length(grid, flags_host):
    return int(load().lbm_list_length(C.byref(grid), C.c_void_p(flags_host)))


def lbm_workspace_size(grid, n_list=-1):
    return int(load().lbm_workspace_size(C.byref(grid), int(n_list)))


def lbm_init(grid, flags, porosity, inputs_on_device, rheology, porous, bc, workspace, workspace_bytes, stream):
    """Returns a context handle.  flags / porosity / workspace are raw addresses
    (ints) of host or device memory; stream is a cudaStream_t as int."""
    h = C.c_void_p()
    st = load().lbm_init(C.byref(h), C.byref(grid), C.c_void_p(flags), C.c_void_p(porosity),
                         int(inputs_on_device), C.byref(rheology), C.byref(porous), C.byref(bc),
                         C.c_void_p(workspace), C.c_size_t(workspace_bytes), C.c_void_p(stream))
    if st != LBM_OK:
        msg = load().lbm_last_error(h).decode() if h else ""
        if h:
            load().lbm_destroy(h)
        raise LBMError(st, msg)
    return h


def lbm_step(ctx, n):
    _check(ctx, load().lbm_step(ctx, int(n)))


def lbm_moments(ctx, rho, u, shear_rate, omega, dst_on_device):
    _check(ctx, load().lbm_moments(ctx, C.c_void_p(rho), C.c_void_p(u), C.c_void_p(shear_rate),
                                   C.c_void_p(omega), int(dst_on_device)))


def lbm_diag(ctx, region, region_on_device):
    out = (C.c_double * 8)()
    _check(ctx, load().lbm_diag(ctx, C.c_void_p(region), int(region_on_device), out))
    return np.array(out[:], dtype=np.float64)


def lbm_diag_noalloc(ctx, region_device):
    """lbm_diag for callers without scratch memory; region_device is a device
    address or None."""
    out = (C.c_double * 8)()
    _check(ctx, load().lbm_diag_noalloc(ctx, C.c_void_p(region_device), out))
    return np.array(out[:], dtype=np.float64)


def lbm_wall_shear(ctx, wss, dst_on_device):
    _check(ctx, load().lbm_wall_shear(ctx, C.c_void_p(wss), int(dst_on_device)))


def lbm_set_l2_window(ctx, max_bytes=-1):
    """max_bytes < 0: the default window; 0: none; > 0: at most that many bytes."""
    _check(ctx, load().lbm_set_l2_window(ctx, int(max_bytes)))


def lbm_l2_window_bytes(ctx):
    return int(load().lbm_l2_window_bytes(ctx))


def lbm_set_l2_group(ctx, group):
    _check(ctx, load().lbm_set_l2_group(ctx, int(group)))


def lbm_step_slabs(ctxs, steps, join_stream=None):
    """Time steps of adjacent z-slab contexts (bottom to top), each on its
    own stream, faces exchanged as they become ready; ordered against
    join_stream (None or 0: the default stream)."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    _check(ctxs[0], load().lbm_step_slabs(arr, len(ctxs), int(steps), join_stream))


def lbm_set_check(ctx, check_every):
    _check(ctx, load().lbm_set_check(ctx, int(check_every)))


def lbm_state_size(ctx):
    return int(load().lbm_state_size(ctx))


def lbm_save(ctx, dst, nbytes, dst_on_device):
    _check(ctx, load().lbm_save(ctx, C.c_void_p(dst), C.c_size_t(nbytes), int(dst_on_device)))


def lbm_load(ctx, src, nbytes, src_on_device):
    _check(ctx, load().lbm_load(ctx, C.c_void_p(src), C.c_size_t(nbytes), int(src_on_device)))


def lbm_time(ctx):
    return int(load().lbm_time(ctx))


def lbm_fluid_count(ctx):
    return int(load().lbm_fluid_count(ctx))


def lbm_last_error(ctx):
    return load().lbm_last_error(ctx).decode()


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_adjoint_workspace_size(ctx, T, K):
    return int(load().lbm_adjoint_workspace_size(ctx, int(T), int(K)))


OBJECTIVES = {"ke": 0, "wss": 1}


def lbm_adjoint(ctx, T, K, objective, region, region_on_device, workspace, workspace_bytes, grad):
    """Runs the adjoint (objective 0: sac kinetic energy, 1: sac-wall shear
    stress); grad is the device address of an FP64 [N] array.  Returns J."""
    J = C.c_double(0.0)
    _check(ctx, load().lbm_adjoint(ctx, int(T), int(K), int(objective), C.c_void_p(region), int(region_on_device),
                                   C.c_void_p(workspace), C.c_size_t(workspace_bytes), C.c_void_p(grad),
                                   C.byref(J)))
    return float(J.value)


def lbm_anisotropy_buffer_size(ctx):
    return int(load().lbm_anisotropy_buffer_size(ctx))


def lbm_set_anisotropy(ctx, shape, buffer, buffer_bytes, max_iter, tol):
    """shape / buffer: device addresses (shape 0 returns to the isotropic closure)."""
    _check(ctx, load().lbm_set_anisotropy(ctx, C.c_void_p(shape or None), C.c_void_p(buffer or None),
                                          C.c_size_t(buffer_bytes), int(max_iter), C.c_float(tol)))


def lbm_slab_bounds(grid, flags_host, nslabs):
    """z0 of each of nslabs balanced z-slabs plus nz (host only)."""
    out = (C.c_int32 * (int(nslabs) + 1))()
    st = load().lbm_slab_bounds(C.byref(grid), C.c_void_p(flags_host), int(nslabs), out)
    if st != LBM_OK:
        raise LBMError(st, "lbm_slab_bounds")
    return [int(v) for v in out]


def lbm_plane_slots(grid, flags_host, z):
    """(first slot, slot count) of z-plane z in the packed layout (host only)."""
    first, count = C.c_int64(), C.c_int64()
    st = load().lbm_plane_slots(C.byref(grid), C.c_void_p(flags_host), int(z), C.byref(first), C.byref(count))
    if st != LBM_OK:
        raise LBMError(st, "lbm_plane_slots")
    return int(first.value), int(count.value)


def lbm_set_halo(ctx, lo_planes, hi_planes):
    _check(ctx, load().lbm_set_halo(ctx, int(lo_planes), int(hi_planes)))


def lbm_halo_message_size(ctx, side):
    return int(load().lbm_halo_message_size(ctx, int(side)))


def lbm_halo_pack(ctx, side, dst):
    _check(ctx, load().lbm_halo_pack(ctx, int(side), C.c_void_p(dst)))


def lbm_halo_unpack(ctx, side, src):
    _check(ctx, load().lbm_halo_unpack(ctx, int(side), C.c_void_p(src)))


def lbm_halo_exchange(lower, upper):
    _check(lower, load().lbm_halo_exchange(lower, upper))


def lbm_porosity_workspace_size(nx, ny, nz):
    return int(load().lbm_porosity_workspace_size(int(nx), int(ny), int(nz)))


def lbm_porosity_average(nx, ny, nz, wire, flags, window, phi_min, phi, workspace, workspace_bytes, stream):
    """Device addresses (ints; flags may be 0); asynchronous on ``stream``."""
    st = load().lbm_porosity_average(int(nx), int(ny), int(nz), C.c_void_p(wire), C.c_void_p(flags or None),
                                     int(window), C.c_float(phi_min), C.c_void_p(phi), C.c_void_p(workspace),
                                     C.c_size_t(workspace_bytes), C.c_void_p(stream))
    if st != LBM_OK:
        raise LBMError(st, "lbm_porosity_average")


def porosity_average(wire, window, phi_min, flags=None, stream=None):
    """Volume-averaged porosity of a wire mask: ``wire`` (and ``flags``) are
    uint8 CUDA tensors of shape (nz, ny, nx); returns a float32 CUDA tensor."""
    import torch

    if wire.dtype != torch.uint8 or not wire.is_cuda or wire.dim() != 3:
        raise ValueError("wire must be a 3-d uint8 CUDA tensor")
    wire = wire.contiguous()
    nz, ny, nx = wire.shape
    if flags is not None:
        if flags.dtype != torch.uint8 or tuple(flags.shape) != tuple(wire.shape) or flags.device != wire.device:
            raise ValueError("flags must be a uint8 tensor of the wire's shape and device")
        flags = flags.contiguous()
    nbytes = lbm_porosity_workspace_size(nx, ny, nz)
    if nbytes == 0:
        raise LBMError(LBM_EINVAL, "bad porosity box")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=wire.device)
    phi = torch.empty(wire.shape, dtype=torch.float32, device=wire.device)
    s = stream if stream is not None else torch.cuda.current_stream(wire.device)
    lbm_porosity_average(nx, ny, nz, wire.data_ptr(), flags.data_ptr() if flags is not None else 0, window,
                         phi_min, phi.data_ptr(), ws.data_ptr(), nbytes, s.cuda_stream)
    return phi


# ----------------------------------------------------------------- convenience owner

class Simulation:
    """Owns one context plus its torch workspace on a CUDA device.

    ``problem`` is a lbm_inputs.Problem (or anything with dims, q, periodic,
    flags, phi, rheology, porous, bc).  Inputs are passed from host memory
    unless ``inputs_on_device`` is set, in which case they are copied to the
    device first through torch.  ``problem.phi`` may itself be a float32 CUDA
    tensor (e.g. from :func:`porosity_average`): it is then passed as is.
    """

    def __init__(self, problem, storage="f32", device="cuda", stream=None, inputs_on_device=False):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.problem = problem
        self.grid = make_grid(problem.dims, problem.q, storage, problem.periodic)
        self.rheo, self.por, self.bc = make_params(problem.rheology, problem.porous, problem.bc)
        flags = np.ascontiguousarray(problem.flags, dtype=np.uint8)
        phi_dev = problem.phi if isinstance(problem.phi, torch.Tensor) else None
        if phi_dev is not None:
            if phi_dev.dtype != torch.float32 or not phi_dev.is_cuda or phi_dev.numel() != flags.size:
                raise ValueError("a device porosity must be a float32 CUDA tensor, one value per cell")
            inputs_on_device = True
            phi = None
        else:
            phi = np.ascontiguousarray(problem.phi, dtype=np.float32)
        n_list = lbm_list_length(self.grid, flags.ctypes.data)
        nbytes = lbm_workspace_size(self.grid, n_list)
        if nbytes == 0:
            raise LBMError(LBM_EINVAL, "bad grid")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if inputs_on_device:
            dflags = torch.from_numpy(flags).to(self.device)
            dphi = (phi_dev.to(self.device).contiguous() if phi_dev is not None
                    else torch.from_numpy(phi).to(self.device))
            fp, pp = dflags.data_ptr(), dphi.data_ptr()
        else:
            fp, pp = flags.ctypes.data, phi.ctypes.data
        with torch.cuda.device(self.device):
            self.ctx = lbm_init(self.grid, fp, pp, int(inputs_on_device), self.rheo, self.por, self.bc,
                                self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        if inputs_on_device:
            self.stream.synchronize()
        self.N = int(flags.size)
        self.shape = flags.shape

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self):
        return lbm_time(self.ctx)

    @property
    def n_fluid(self):
        return lbm_fluid_count(self.ctx)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self, on_device=False):
        """rho, u (3, ...), gdot, omega of the current time on the dense box."""
        torch = self.torch
        if on_device:
            out = torch.empty((6,) + self.shape, dtype=torch.float32, device=self.device)
            lbm_moments(self.ctx, out[0].data_ptr(), out[1].data_ptr(), out[4].data_ptr(), out[5].data_ptr(), 1)
            return dict(rho=out[0], u=out[1:4], gdot=out[4], omega=out[5])
        rho = np.zeros(self.shape, np.float32)
        u = np.zeros((3,) + self.shape, np.float32)
        g = np.zeros(self.shape, np.float32)
        om = np.zeros(self.shape, np.float32)
        lbm_moments(self.ctx, rho.ctypes.data, u.ctypes.data, g.ctypes.data, om.ctypes.data, 0)
        return dict(rho=rho, u=u, gdot=g, omega=om)

    def set_anisotropy(self, shape, max_iter=16, tol=1e-6):
        """Anisotropic permeability K = k(phi) S^{-1}: ``shape`` is the
        (6, nz, ny, nx) shape tensor S (xx yy zz xy xz yz; numpy or a CUDA
        tensor), or None for the isotropic closure."""
        torch = self.torch
        if shape is None:
            lbm_set_anisotropy(self.ctx, 0, 0, 0, max_iter, tol)
            self._aniso = None
            return
        S = shape if isinstance(shape, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(shape, np.float32))
        S = S.to(device=self.device, dtype=torch.float32).contiguous()
        if tuple(S.shape) != (6,) + tuple(self.shape):
            raise ValueError("shape tensor must be (6, nz, ny, nx)")
        nbytes = lbm_anisotropy_buffer_size(self.ctx)
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        lbm_set_anisotropy(self.ctx, S.data_ptr(), buf.data_ptr(), nbytes, max_iter, tol)
        self._aniso = buf  # the context keeps using it

    def wall_shear(self, on_device=False):
        """Voxel wall-shear-stress proxy |tau| of the current time on the dense box."""
        if on_device:
            out = self.torch.empty(self.shape, dtype=self.torch.float32, device=self.device)
            lbm_wall_shear(self.ctx, out.data_ptr(), 1)
            return out
        out = np.zeros(self.shape, np.float32)
        lbm_wall_shear(self.ctx, out.ctypes.data, 0)
        return out

    def diag(self, region=None):
        if region is None:
            return lbm_diag(self.ctx, None, 0)
        if hasattr(region, "data_ptr"):
            return lbm_diag(self.ctx, region.data_ptr(), 1)
        reg = np.ascontiguousarray(region, dtype=np.uint8)
        return lbm_diag(self.ctx, reg.ctypes.data, 0)

    def save(self):
        n = lbm_state_size(self.ctx)
        buf = np.zeros(n, np.uint8)
        lbm_save(self.ctx, buf.ctypes.data, n, 0)
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        lbm_load(self.ctx, buf.ctypes.data, buf.size, 0)

    def adjoint(self, T, K, region, objective="ke"):
        """(J, dJ/dphi) of the sac objective over steps 1..T with a checkpoint
        every K steps: "ke" the mean kinetic energy, "wss" the mean wall shear
        stress over the region's wall cells; dJ/dphi is an FP64 device tensor
        shaped like the box."""
        kind = OBJECTIVES[objective]
        torch = self.torch
        nbytes = lbm_adjoint_workspace_size(self.ctx, T, K)
        if nbytes == 0:
            raise LBMError(LBM_EINVAL, "T and K must be >= 1")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        if hasattr(region, "data_ptr"):
            reg = region.to(device=self.device, dtype=torch.uint8).contiguous()
            J = lbm_adjoint(self.ctx, T, K, kind, reg.data_ptr(), 1, ws.data_ptr(), nbytes, grad.data_ptr())
        else:
            reg = np.ascontiguousarray(region, dtype=np.uint8)
            J = lbm_adjoint(self.ctx, T, K, kind, reg.ctypes.data, 0, ws.data_ptr(), nbytes, grad.data_ptr())
        return J, grad


def sac_kinetic_energy(problem, phi, T, K, region, storage="f32"):
    """J(phi) = time-and-sac mean of rho |u|^2 / 2 over steps 1..T, as a
    differentiable torch function of the porosity tensor phi (any device; the
    computation runs on the current CUDA device).  Backward returns the
    gradient from the hand-written adjoint (lbm_adjoint)."""
    return _sac_objective(problem, phi, T, K, region, storage, "ke")


def sac_wall_shear(problem, phi, T, K, region, storage="f32"):
    """J(phi) = time mean over steps 1..T of the wall-shear-stress proxy |tau|
    averaged over the region's wall cells, as a differentiable torch function
    of phi (backward: lbm_adjoint with objective 1)."""
    return _sac_objective(problem, phi, T, K, region, storage, "wss")


def _sac_objective(problem, phi, T, K, region, storage, objective):
    import torch

    class _SacKE(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi_t):
            prob = _with_porosity(problem, phi_t.detach().cpu().numpy())
            sim = Simulation(prob, storage=storage)
            try:
                J, grad = sim.adjoint(T, K, region, objective)
            finally:
                sim.close()
            ctx.save_for_backward(grad.to(device=phi_t.device, dtype=phi_t.dtype))
            return torch.tensor(J, dtype=phi_t.dtype, device=phi_t.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad

    return _SacKE.apply(phi)


def _with_porosity(problem, phi):
    import dataclasses

    phi = np.ascontiguousarray(phi, dtype=np.float32)
    if dataclasses.is_dataclass(problem):
        return dataclasses.replace(problem, phi=phi)
    problem.phi = phi
    return problem
