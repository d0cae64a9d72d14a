"""ctypes wrapper of the FP64 C oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline leg of the benchmark.  The library path never imports it.
"""

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("q", C.c_int32),
        ("periodic", C.c_int32 * 3),
        ("mu0", C.c_double), ("mu_inf", C.c_double), ("lam", C.c_double), ("n_cy", C.c_double),
        ("a_cy", C.c_double), ("rho0", C.c_double), ("dx", C.c_double), ("dt", C.c_double),
        ("d_p", C.c_double), ("k_const", C.c_double), ("nu_darcy", C.c_double),
        ("forchheimer", C.c_int32),
        ("g", C.c_double * 3),
        ("in_axis", C.c_int32), ("in_side", C.c_int32),
        ("in_center", C.c_double * 3), ("in_radius", C.c_double), ("u0", C.c_double),
        ("amp", C.c_double), ("period", C.c_double), ("ramp", C.c_double),
        ("out_axis", C.c_int32), ("out_side", C.c_int32), ("rho_out", C.c_double),
    ]


def compile_library(src, out):
    """Compile one C oracle source into the shared library ``out`` (gcc, OpenMP)."""
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_GNU_SOURCE",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force=False):
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_library(_SRC, _LIB)


def load_library(path):
    """ctypes handle of a compiled oracle library with its signatures declared."""
    L = C.CDLL(path)
    P = C.POINTER
    d = P(C.c_double)
    L.oracle_create.restype = C.c_void_p
    L.oracle_create.argtypes = [P(OracleParams), P(C.c_uint8), d, P(C.c_int32)]
    L.oracle_destroy.argtypes = [C.c_void_p]
    L.oracle_step.argtypes = [C.c_void_p, C.c_int64]
    L.oracle_moments.argtypes = [C.c_void_p, d, d, d, d, d, d]
    L.oracle_diag.argtypes = [C.c_void_p, P(C.c_uint8), d]
    L.oracle_wss.restype = None
    L.oracle_wss.argtypes = [C.c_void_p, C.c_void_p]
    L.oracle_run_objective.restype = C.c_double
    L.oracle_run_objective.argtypes = [C.c_void_p, C.c_int64, P(C.c_uint8)]
    L.oracle_nfluid.restype = C.c_int64
    L.oracle_nfluid.argtypes = [C.c_void_p]
    L.oracle_time.restype = C.c_int64
    L.oracle_time.argtypes = [C.c_void_p]
    L.oracle_q.restype = C.c_int32
    L.oracle_q.argtypes = [C.c_void_p]
    L.oracle_lattice.argtypes = [C.c_void_p, P(C.c_int32), d, P(C.c_int32)]
    L.oracle_cells.argtypes = [C.c_void_p, P(C.c_int64)]
    L.oracle_get_state.argtypes = [C.c_void_p, d, d]
    L.oracle_set_state.argtypes = [C.c_void_p, d, d, C.c_int64]
    L.oracle_collide_cell.argtypes = [C.c_void_p, C.c_int64, d, C.c_double, d, d]
    L.oracle_apply_boundaries.argtypes = [C.c_void_p, C.c_int64]
    L.oracle_lattice_params.argtypes = [C.c_void_p, d]
    L.oracle_num_threads.restype = C.c_int32
    L.oracle_set_anisotropy.restype = C.c_int32
    L.oracle_set_anisotropy.argtypes = [C.c_void_p, d, d]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params_from_problem(prob):
    """Packs a lbm_inputs.Problem into the oracle's parameter struct."""
    nx, ny, nz = prob.dims
    r, p, b = prob.rheology, prob.porous, prob.bc
    o = OracleParams()
    o.nx, o.ny, o.nz, o.q = nx, ny, nz, prob.q
    o.periodic = (C.c_int32 * 3)(*prob.periodic)
    o.mu0, o.mu_inf, o.lam, o.n_cy, o.a_cy = r["mu0"], r["mu_inf"], r["lam"], r["n"], r["a"]
    o.rho0, o.dx, o.dt = r["rho0"], r["dx"], r["dt"]
    o.d_p, o.k_const, o.nu_darcy = p["d_p"], p["k_const"], p["nu_darcy"]
    o.forchheimer = int(p["forchheimer"])
    o.g = (C.c_double * 3)(*b["body_force"])
    o.in_axis, o.in_side = b["inlet_axis"], b["inlet_side"]
    o.in_center = (C.c_double * 3)(*b["inlet_center"])
    o.in_radius, o.u0, o.amp = b["inlet_radius"], b["u0"], b["amp"]
    o.period, o.ramp = b["period"], b["ramp_steps"]
    o.out_axis, o.out_side, o.rho_out = b["outlet_axis"], b["outlet_side"], b["rho_out"]
    return o


def shape_tensor_sqrt(S):
    """Per-cell square root of the symmetric positive definite shape tensor:
    S is (6, ...) with components xx yy zz xy xz yz; returns the same layout.
    Through the eigendecomposition S = V diag(l) V^T (numpy.linalg.eigh),
    S^{1/2} = V diag(sqrt(l)) V^T."""
    S = np.asarray(S, dtype=np.float64)
    sh = S.shape[1:]
    s = S.reshape(6, -1)
    M = np.empty((s.shape[1], 3, 3))
    for (a, b), c in (((0, 0), 0), ((1, 1), 1), ((2, 2), 2), ((0, 1), 3), ((0, 2), 4), ((1, 2), 5)):
        M[:, a, b] = s[c]
        M[:, b, a] = s[c]
    lam, V = np.linalg.eigh(M)
    if not np.all(lam > 0):
        raise ValueError("shape tensor not positive definite")
    H = np.einsum("nab,nb,ncb->nac", V, np.sqrt(lam), V)
    out = np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 2, 2], H[:, 0, 1], H[:, 0, 2], H[:, 1, 2]])
    return out.reshape((6,) + sh)


class Oracle:
    """FP64 reference simulation of one Problem.  ``shape_tensor``: optional
    (6, nz, ny, nx) symmetric positive definite tensor S per cell (xx yy zz xy
    xz yz) for the anisotropic permeability K = k(phi) S^{-1} of the velocity
    solve's fixed-point iteration (Sec. 3 remark).  ``library``: a handle from
    :func:`load_library` to run another build of the oracle source (the
    pin tests run copies with a planted mistake through it)."""

    def __init__(self, prob, phi=None, shape_tensor=None, library=None):
        self.L = lib() if library is None else library
        self.prob = prob
        self.params = params_from_problem(prob)
        self.flags = np.ascontiguousarray(prob.flags, dtype=np.uint8)
        ph = prob.phi if phi is None else phi
        self.phi = np.ascontiguousarray(ph, dtype=np.float64)
        st = C.c_int32(0)
        self.h = self.L.oracle_create(C.byref(self.params),
                                      self.flags.ctypes.data_as(C.POINTER(C.c_uint8)),
                                      _dptr(self.phi), C.byref(st))
        if st.value != 0:
            if self.h:
                self.L.oracle_destroy(self.h)
            self.h = None
            raise ValueError(f"oracle_create failed with status {st.value}")
        self.q = self.L.oracle_q(self.h)
        self.nf = self.L.oracle_nfluid(self.h)
        self.shape = self.flags.shape
        if shape_tensor is not None:
            S = np.asarray(shape_tensor, dtype=np.float64)
            if S.shape != (6,) + self.shape:
                raise ValueError("shape_tensor must be (6, nz, ny, nx)")
            s = np.ascontiguousarray(S.reshape(6, -1).T)
            h = np.ascontiguousarray(shape_tensor_sqrt(S).reshape(6, -1).T)
            if self.L.oracle_set_anisotropy(self.h, _dptr(s), _dptr(h)) != 0:
                raise MemoryError("oracle_set_anisotropy")

    def close(self):
        if self.h:
            self.L.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self):
        return self.L.oracle_time(self.h)

    def step(self, n=1):
        self.L.oracle_step(self.h, int(n))

    def moments(self):
        """dict of dense float64 fields at the current time: rho, u (3, ...),
        gdot, omega (0 at solid cells)."""
        n = self.flags.size
        arrs = [np.zeros(n) for _ in range(6)]
        self.L.oracle_moments(self.h, *[_dptr(a) for a in arrs])
        sh = self.shape
        return dict(rho=arrs[0].reshape(sh), u=np.stack([a.reshape(sh) for a in arrs[1:4]]),
                    gdot=arrs[4].reshape(sh), omega=arrs[5].reshape(sh))

    def diag(self, region=None):
        out = np.zeros(8)
        reg = None
        if region is not None:
            reg = np.ascontiguousarray(region, dtype=np.uint8)
        self.L.oracle_diag(self.h, reg.ctypes.data_as(C.POINTER(C.c_uint8)) if reg is not None else None,
                           _dptr(out))
        return out

    def wall_shear(self):
        """Voxel wall-shear-stress proxy |tau| of the current time (dense box)."""
        out = np.zeros(int(np.prod(self.shape)))
        self.L.oracle_wss(self.h, _dptr(out))
        return out.reshape(self.shape)

    def run_objective(self, T, region):
        reg = np.ascontiguousarray(region, dtype=np.uint8)
        return self.L.oracle_run_objective(self.h, int(T), reg.ctypes.data_as(C.POINTER(C.c_uint8)))

    def lattice(self):
        c = np.zeros((self.q, 3), dtype=np.int32)
        w = np.zeros(self.q)
        opp = np.zeros(self.q, dtype=np.int32)
        self.L.oracle_lattice(self.h, c.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(w),
                              opp.ctypes.data_as(C.POINTER(C.c_int32)))
        return c, w, opp

    def cells(self):
        c = np.zeros(self.nf, dtype=np.int64)
        self.L.oracle_cells(self.h, c.ctypes.data_as(C.POINTER(C.c_int64)))
        return c

    def get_state(self):
        f = np.zeros((self.nf, self.q))
        om = np.zeros(self.nf)
        self.L.oracle_get_state(self.h, _dptr(f), _dptr(om))
        return f, om

    def set_state(self, f, omega, t):
        f = np.ascontiguousarray(f, dtype=np.float64)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        self.L.oracle_set_state(self.h, _dptr(f), _dptr(om), int(t))

    def collide_cell(self, k, f, omega_prev):
        f = np.ascontiguousarray(f, dtype=np.float64)
        fpost = np.zeros(self.q)
        out = np.zeros(9)
        self.L.oracle_collide_cell(self.h, int(k), _dptr(f), float(omega_prev), _dptr(fpost), _dptr(out))
        return fpost, dict(rho=out[0], u=out[1:4].copy(), F=out[4:7].copy(), gdot=out[7], omega=out[8])

    def apply_boundaries(self, t):
        self.L.oracle_apply_boundaries(self.h, int(t))

    def lattice_params(self):
        out = np.zeros(6)
        self.L.oracle_lattice_params(self.h, _dptr(out))
        return dict(mu0=out[0], mu_inf=out[1], lam=out[2], nu_d=out[3], d_p=out[4], k_const=out[5])


def num_threads():
    return int(lib().oracle_num_threads())
