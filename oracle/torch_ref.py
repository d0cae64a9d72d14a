"""Pull-form restatement of the VANSE LBM step in PyTorch float64 on the CPU.

TEST INFRASTRUCTURE ONLY.  A second, independently written FP64 statement of
the method of Horvat et al. (arXiv 2402.10809, Sec. 2-4): whole-grid tensor
operations in pull form, where ``oracle/lbm_oracle.c`` loops over cells in push
form.  The tests compare the two on tiny grids, and differentiate this one with
autograd to obtain reference gradients of a sac objective with respect to the
porosity field.  It shares no code with the CUDA path and none with the C
oracle.

Conventions: tensors are [Q, nz, ny, nx]; the state f is the pre-collision
population of time t after streaming and boundary reconstruction; omega is the
rate of the previous collision.
"""

import math

import numpy as np
import torch

SOLID, FLUID, INLET, OUTLET = 0, 1, 2, 3
CS2 = 1.0 / 3.0


def velocity_set(q):
    """D3Q19 / D3Q27 velocities and weights, rest first, then the six faces,
    twelve edges and (D3Q27) eight corners."""
    faces = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    edges = [(a, b, 0) for a in (1, -1) for b in (1, -1)] + \
            [(a, 0, b) for a in (1, -1) for b in (1, -1)] + \
            [(0, a, b) for a in (1, -1) for b in (1, -1)]
    corners = [(a, b, c) for a in (1, -1) for b in (1, -1) for c in (1, -1)]
    if q == 19:
        vel = [(0, 0, 0)] + faces + edges
        wts = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
    elif q == 27:
        vel = [(0, 0, 0)] + faces + edges + corners
        wts = [8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8
    else:
        raise ValueError("q must be 19 or 27")
    c = np.array(vel, dtype=np.int64)
    opp = np.array([vel.index(tuple(-v for v in ci)) for ci in vel])
    return c, np.array(wts, dtype=np.float64), opp


def _safe_norm(s):
    """sqrt(s) with a zero (not NaN) derivative at s = 0."""
    pos = s > 0
    return torch.sqrt(torch.where(pos, s, torch.ones_like(s))) * pos


class TorchLBM:
    """Whole-grid FP64 LBM for one lbm_inputs.Problem.  ``shape_tensor``: the
    optional (6, nz, ny, nx) SPD tensor S (xx yy zz xy xz yz) of an anisotropic
    permeability K = k(phi) S^{-1}, solved by the fixed-point iteration of the
    Sec. 3 remark."""

    def __init__(self, prob, shape_tensor=None):
        self.prob = prob
        nx, ny, nz = prob.dims
        self.n = (nx, ny, nz)
        self.c, w, self.opp = velocity_set(prob.q)
        self.Q = len(w)
        self.w = torch.tensor(w, dtype=torch.float64).view(-1, 1, 1, 1)
        self.cf = torch.tensor(self.c, dtype=torch.float64)  # [Q, 3] (x, y, z)
        r, p, b = prob.rheology, prob.porous, prob.bc
        scale = r["dt"] / (r["dx"] * r["dx"])
        # Lattice units from the Table 1 scales: nu = mu / rho0 * dt / dx^2.
        self.mu0 = r["mu0"] / r["rho0"] * scale
        self.mu_inf = r["mu_inf"] / r["rho0"] * scale
        self.lam = r["lam"] / r["dt"]
        self.n_cy, self.a_cy = r["n"], r["a"]
        self.nu_d = p["nu_darcy"] * scale if p["nu_darcy"] > 0 else self.mu0
        self.d_p = p["d_p"] / r["dx"]
        self.k_const = p["k_const"] / (r["dx"] * r["dx"])
        self.forch = bool(p["forchheimer"])
        self.g = torch.tensor(b["body_force"], dtype=torch.float64).view(3, 1, 1, 1)
        self.bc = b
        flags = torch.tensor(prob.flags.astype(np.int64))
        self.flags = flags
        self.fluid = flags != SOLID
        self.periodic = prob.periodic
        self._build_links()
        self.S = self.Sh = None
        if shape_tensor is not None:
            s = torch.tensor(np.asarray(shape_tensor, dtype=np.float64))
            M = torch.empty(s.shape[1:] + (3, 3), dtype=torch.float64)
            for (a, b), k in (((0, 0), 0), ((1, 1), 1), ((2, 2), 2), ((0, 1), 3), ((0, 2), 4), ((1, 2), 5)):
                M[..., a, b] = s[k]
                M[..., b, a] = s[k]
            lam, V = torch.linalg.eigh(M)
            self.S = M  # [..., 3, 3]
            self.Sh = V @ torch.diag_embed(torch.sqrt(lam)) @ V.transpose(-1, -2)
            # the tensor acts where there is a medium (phi < 1, the reading of
            # the C oracle); cells with phi = 1 keep the isotropic closure,
            # which also fixes the one-sided derivative there
            medium = torch.tensor(np.asarray(prob.phi) < 1)[..., None, None]
            eye = torch.eye(3, dtype=torch.float64)
            self.S = torch.where(medium, self.S, eye)
            self.Sh = torch.where(medium, self.Sh, eye)

    # ------------------------------------------------------------ geometry
    def _shift(self, t, d):
        """out[y] = t[y + d] on the periodic torus (d = (dx, dy, dz))."""
        return torch.roll(t, shifts=(-d[2], -d[1], -d[0]), dims=(-3, -2, -1))

    def _inside(self, d):
        """Boolean grid: y + d lies in the box or wraps on a periodic axis.
        Also returns a grid telling whether y + d crosses the inlet / outlet face."""
        nx, ny, nz = self.n
        z, y, x = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
        pos = (x + d[0], y + d[1], z + d[2])
        size = (nx, ny, nz)
        ok = torch.ones_like(x, dtype=torch.bool)
        cross_in = torch.zeros_like(ok)
        cross_out = torch.zeros_like(ok)
        b = self.bc
        for a in range(3):
            out_lo = pos[a] < 0
            out_hi = pos[a] >= size[a]
            if not self.periodic[a]:
                ok &= ~(out_lo | out_hi)
                if b["inlet_axis"] == a:
                    cross_in |= out_lo if b["inlet_side"] == 0 else out_hi
                if b["outlet_axis"] == a:
                    cross_out |= out_lo if b["outlet_side"] == 0 else out_hi
        return ok, cross_in, cross_out

    def _build_links(self):
        Q = self.Q
        pull, bb, unknown, dest_fluid = [], [], [], []
        for i in range(Q):
            ci = tuple(int(v) for v in self.c[i])
            src = tuple(-v for v in ci)
            ok, cin, cout = self._inside(src)
            src_fluid = ok & self._shift(self.fluid, src)
            unk = self.fluid & (((self.flags == INLET) & cin) | ((self.flags == OUTLET) & cout))
            pull.append(self.fluid & src_fluid)
            bb.append(self.fluid & ~src_fluid & ~unk)
            unknown.append(unk)
            okd, _, _ = self._inside(ci)
            dest_fluid.append(okd & self._shift(self.fluid, ci))
        self.pull = torch.stack(pull)
        self.bb = torch.stack(bb)
        self.unknown = torch.stack(unknown)
        self.dest_fluid = torch.stack(dest_fluid)

    # ------------------------------------------------------------ physics
    def closure(self, phi):
        """(1/k, 1/sqrt(k), C_F) from Kozeny-Carman and Ergun (Sec. 2)."""
        if self.k_const > 0:
            solid = phi < 1
            inv_k = torch.where(solid, torch.full_like(phi, 1 / self.k_const), torch.zeros_like(phi))
            inv_sk = torch.where(solid, torch.full_like(phi, 1 / math.sqrt(self.k_const)), torch.zeros_like(phi))
        else:
            # 1/k = 150 (1 - phi)^2 / (phi^3 d^2); 1/sqrt(k) = sqrt(150) (1 - phi) / (phi^1.5 d)
            # on the porosity domain phi <= 1 (so that autograd yields the
            # one-sided derivative at phi = 1, where |1 - phi| has its kink).
            inv_k = 150.0 * (1 - phi) ** 2 / (phi ** 3 * self.d_p ** 2)
            inv_sk = math.sqrt(150.0) * (1 - phi) / (phi ** 1.5 * self.d_p)
        cf = 1.75 / torch.sqrt(150.0 * phi ** 3) if self.forch else torch.zeros_like(phi)
        return inv_k, inv_sk, cf

    def macroscopic(self, f, phi):
        """rho, u, F = rho (g + f_d(u)) with the explicit velocity of Sec. 3."""
        sig = f.sum(0)
        sig = torch.where(self.fluid, sig, phi)  # keep solid cells finite
        rho = sig / phi
        m = torch.einsum("qa,q...->a...", self.cf, f)
        v = (m + 0.5 * rho * self.g) / (phi * rho)
        vn = _safe_norm((v * v).sum(0))
        inv_k, inv_sk, cf = self.closure(phi)
        if self.S is not None:
            u, fd = self._anisotropic(v, phi, inv_k, inv_sk, cf)
            return rho, u, rho * (self.g + fd)
        c0 = 0.5 + phi * self.nu_d * inv_k / 4
        c1 = phi ** 2 * cf * inv_sk / 2
        u = v / (c0 + torch.sqrt(c0 * c0 + c1 * vn))
        un = _safe_norm((u * u).sum(0))
        fd = -(phi ** 2) * self.nu_d * inv_k * u - phi ** 3 * cf * inv_sk * un * u
        F = rho * (self.g + fd)
        return rho, u, F

    def _anisotropic(self, v, phi, inv_k, inv_sk, cf):
        """Velocity and drag with K^{-1} = S / k, K^{-1/2} = S^{1/2} / sqrt(k):
        (A + |u| B) u = v, A = Id + (phi nu / 2) K^{-1},
        B = (phi^2 C_F / 2) K^{-1/2}, by u_{m+1} = (A + |u_m| B)^{-1} v from
        u_0 = v, batched 3x3 solves over the grid (cells without a medium have
        K^{-1} = 0, hence u = v); f(u) = -phi^2 nu K^{-1} u -
        phi^3 C_F |u| K^{-1/2} u."""
        e = (...,) + (None, None)
        Kinv = self.S * inv_k[e]
        Kinvh = self.Sh * inv_sk[e]
        A = torch.eye(3, dtype=torch.float64) + (phi * self.nu_d / 2)[e] * Kinv
        B = (phi ** 2 * cf / 2)[e] * Kinvh
        vv = v.permute(1, 2, 3, 0).unsqueeze(-1)  # [..., 3, 1]
        u = vv
        scale = vv.abs().max()
        for _ in range(200):
            un = _safe_norm((u * u).sum((-2, -1)))
            u_new = torch.linalg.solve(A + un[e] * B, vv)
            done = bool((u_new - u).abs().max() <= 1e-15 * scale)
            u = u_new
            if done:
                break
        un = _safe_norm((u * u).sum((-2, -1)))
        fd = -(phi ** 2 * self.nu_d)[e] * (Kinv @ u) - (phi ** 3 * cf)[e] * un[e] * (Kinvh @ u)
        return u.squeeze(-1).permute(3, 0, 1, 2), fd.squeeze(-1).permute(3, 0, 1, 2)

    def equilibrium(self, phi, rho, u):
        cu = torch.einsum("qa,a...->q...", self.cf, u)
        uu = (u * u).sum(0)
        return self.w * phi * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))

    def shear_rate(self, f, feq, rho, u, F, omega_prev):
        d = f - feq
        P = torch.einsum("qa,qb,q...->ab...", self.cf, self.cf, d)
        P = P + 0.5 * (F.unsqueeze(1) * u.unsqueeze(0) + u.unsqueeze(1) * F.unsqueeze(0))
        nrm = _safe_norm((P * P).sum((0, 1)))
        return omega_prev * nrm / (CS2 * rho)

    def viscosity(self, gdot):
        x = self.lam * gdot
        return self.mu_inf + (self.mu0 - self.mu_inf) * (1 + x ** self.a_cy) ** ((self.n_cy - 1) / self.a_cy)

    @staticmethod
    def rate(rho, mu):
        return 2 * rho * CS2 / (2 * mu + rho * CS2)

    def collide(self, f, omega_prev, phi):
        rho, u, F = self.macroscopic(f, phi)
        feq = self.equilibrium(phi, rho, u)
        gdot = self.shear_rate(f, feq, rho, u, F, omega_prev)
        om = self.rate(rho, self.viscosity(gdot))
        phi_link = torch.stack([torch.where(self.dest_fluid[i], self._shift(phi, tuple(int(v) for v in self.c[i])), phi)
                                for i in range(self.Q)])
        om_phi = self.w * rho * (phi_link - phi)
        cu = torch.einsum("qa,a...->q...", self.cf, u)
        cF = torch.einsum("qa,a...->q...", self.cf, F)
        uF = (u * F).sum(0)
        om_f = self.w * (1 - om / 2) * ((cF - uF) / CS2 + cu * cF / (CS2 * CS2))
        fpost = f + om_phi + om_f - om * (f - feq)
        return fpost, om, rho, u

    # ------------------------------------------------------------ streaming
    def stream(self, fpost):
        out = []
        for i in range(self.Q):
            ci = tuple(int(v) for v in self.c[i])
            pulled = self._shift(fpost[i], tuple(-v for v in ci))
            out.append(torch.where(self.pull[i], pulled,
                                   torch.where(self.bb[i], fpost[self.opp[i]], torch.zeros_like(pulled))))
        return torch.stack(out)

    # ------------------------------------------------------------ boundaries
    def inlet_velocity(self, t):
        b = self.bc
        nx, ny, nz = self.n
        z, y, x = torch.meshgrid(torch.arange(nz, dtype=torch.float64) + 0.5,
                                 torch.arange(ny, dtype=torch.float64) + 0.5,
                                 torch.arange(nx, dtype=torch.float64) + 0.5, indexing="ij")
        pos = (x, y, z)
        r2 = torch.zeros_like(x)
        for a in range(3):
            if a != b["inlet_axis"]:
                r2 = r2 + (pos[a] - b["inlet_center"][a]) ** 2
        prof = torch.clamp(1 - r2 / b["inlet_radius"] ** 2, min=0)
        v = b["u0"] * (1 + b["amp"] * math.sin(2 * math.pi * t / b["period"]))
        if b["ramp_steps"] > 0 and t < b["ramp_steps"]:
            v *= t / b["ramp_steps"]
        u = torch.zeros((3,) + x.shape, dtype=torch.float64)
        sgn = 1.0 if b["inlet_side"] == 0 else -1.0
        u[b["inlet_axis"]] = sgn * 2 * v * prof
        return u

    def boundaries(self, f, t, phi):
        b = self.bc
        if b["inlet_axis"] >= 0 and bool((self.flags == INLET).any()):
            ax = b["inlet_axis"]
            sgn = 1 if b["inlet_side"] == 0 else -1
            cn = torch.tensor(self.c[:, ax] * sgn)
            ub = self.inlet_velocity(t) - 0.5 * self.g
            s0 = f[cn == 0].sum(0)
            sm = f[cn < 0].sum(0)
            rho = (s0 + 2 * sm) / (phi * (1 - ub[ax] * sgn))
            feq = self.equilibrium(phi, rho, ub)
            unk = cn > 0
            new = f.clone()
            idx_u = torch.nonzero(unk).flatten().tolist()
            for i in idx_u:
                j = int(self.opp[i])
                new[i] = f[j] + feq[i] - feq[j]
            is_in = self.flags == INLET
            f = torch.where(is_in.unsqueeze(0) & unk.view(-1, 1, 1, 1), new, f)
        if b["outlet_axis"] >= 0 and bool((self.flags == OUTLET).any()):
            ax = b["outlet_axis"]
            sgn = -1 if b["outlet_side"] == 1 else 1
            d = [0, 0, 0]
            d[ax] = sgn
            f_nb = self._shift(f, tuple(d))
            phi_nb = self._shift(phi, tuple(d))
            fluid_nb = self._shift(self.fluid, tuple(d))
            is_out = self.flags == OUTLET
            safe_f = torch.where(fluid_nb.unsqueeze(0), f_nb, self.w * phi_nb)
            # the neighbour's macroscopic state (computed as if it sat at the outlet cell)
            rho_nb, u_nb = self._macro_at(safe_f, phi_nb)
            feq_out = self.equilibrium(phi, torch.full_like(phi, b["rho_out"]), u_nb)
            feq_nb = self.equilibrium(phi_nb, rho_nb, u_nb)
            new = feq_out + safe_f - feq_nb
            unk = torch.tensor(self.c[:, ax] * sgn > 0)
            f = torch.where(is_out.unsqueeze(0) & unk.view(-1, 1, 1, 1), new, f)
        return f

    def _macro_at(self, f, phi):
        sig = f.sum(0)
        rho = sig / phi
        m = torch.einsum("qa,q...->a...", self.cf, f)
        v = (m + 0.5 * rho * self.g) / (phi * rho)
        vn = _safe_norm((v * v).sum(0))
        inv_k, inv_sk, cf = self.closure(phi)
        c0 = 0.5 + phi * self.nu_d * inv_k / 4
        c1 = phi ** 2 * cf * inv_sk / 2
        u = v / (c0 + torch.sqrt(c0 * c0 + c1 * vn))
        return rho, u

    # ------------------------------------------------------------ driver
    def initial(self, phi):
        f = torch.where(self.fluid.unsqueeze(0), self.w * phi, torch.zeros((self.Q,) + phi.shape, dtype=torch.float64))
        f = self.boundaries(f, 0, phi)
        om = torch.full_like(phi, self.rate(1.0, self.mu0))
        return f, om

    def step(self, f, omega_prev, phi, t):
        """One step from time t to t+1 (collide, stream, boundaries of t+1)."""
        fpost, om, _, _ = self.collide(f, omega_prev, phi)
        fnew = self.stream(fpost)
        fnew = self.boundaries(fnew, t + 1, phi)
        fnew = torch.where(self.fluid.unsqueeze(0), fnew, torch.zeros_like(fnew))
        om = torch.where(self.fluid, om, torch.zeros_like(om))
        return fnew, om

    def run(self, phi, steps):
        f, om = self.initial(phi)
        for t in range(steps):
            f, om = self.step(f, om, phi, t)
        return f, om

    def fields(self, f, omega_prev, phi):
        rho, u, F = self.macroscopic(f, phi)
        feq = self.equilibrium(phi, rho, u)
        gdot = self.shear_rate(f, feq, rho, u, F, omega_prev)
        om = self.rate(rho, self.viscosity(gdot))
        z = torch.zeros_like(rho)
        fl = self.fluid
        return dict(rho=torch.where(fl, rho, z), u=torch.where(fl, u, torch.zeros_like(u)),
                    gdot=torch.where(fl, gdot, z), omega=torch.where(fl, om, z))

    def wall_normal(self):
        """Voxel wall direction of every plain fluid cell: the normalised sum of
        w_i c_i over its links to solid cells or out of the box (zero where
        there are none); and the mask of cells that have such links."""
        walls = torch.stack([~self.dest_fluid[i] for i in range(self.Q)]).to(torch.float64)
        n = torch.einsum("q...,qa->a...", walls * self.w, self.cf)
        nn = torch.sqrt((n * n).sum(0))
        has = (nn > 1e-12) & (self.flags == FLUID)
        return torch.where(has, n / torch.where(has, nn, torch.ones_like(nn)), torch.zeros_like(n)), has

    def wall_shear(self, f, omega_prev, phi):
        """Voxel wall-shear-stress proxy |tau| of state f: tau = sigma n -
        (n . sigma n) n, sigma = -(1 - omega/2) Pi with the corrected second
        moment Pi of the shear rate and omega of the collision of this time."""
        rho, u, F = self.macroscopic(f, phi)
        feq = self.equilibrium(phi, rho, u)
        d = f - feq
        P = torch.einsum("qa,qb,q...->ab...", self.cf, self.cf, d)
        P = P + 0.5 * (F.unsqueeze(1) * u.unsqueeze(0) + u.unsqueeze(1) * F.unsqueeze(0))
        nrm = _safe_norm((P * P).sum((0, 1)))
        gdot = omega_prev * nrm / (CS2 * rho)
        om = self.rate(rho, self.viscosity(gdot))
        n, has = self.wall_normal()
        sn = -(1 - om / 2) * torch.einsum("ab...,b...->a...", P, n)
        tau = sn - (sn * n).sum(0) * n
        return torch.where(has, _safe_norm((tau * tau).sum(0)), torch.zeros_like(rho))

    def objective(self, phi, T, region, checkpoint=True, kind="ke"):
        """J = (1/T) sum_{t=1..T} of the region mean of rho |u|^2 / 2
        (kind "ke"), or of |tau| over the region's cells with wall links
        (kind "wss")."""
        reg = torch.as_tensor(region.astype(bool)) & self.fluid
        if kind == "wss":
            reg = reg & self.wall_normal()[1]
        cnt = float(reg.sum())
        f, om = self.initial(phi)
        J = torch.zeros((), dtype=torch.float64)

        def one(f, om, t):
            f2, om2 = self.step(f, om, phi, t)
            if kind == "wss":
                val = self.wall_shear(f2, om2, phi)
            else:
                rho, u, _ = self.macroscopic(f2, phi)
                val = 0.5 * rho * (u * u).sum(0)
            ke = torch.where(reg, val, torch.zeros_like(val)).sum() / cnt
            return f2, om2, ke

        for t in range(T):
            if checkpoint:
                from torch.utils.checkpoint import checkpoint as ckpt
                f, om, ke = ckpt(one, f, om, t, use_reentrant=False)
            else:
                f, om, ke = one(f, om, t)
            J = J + ke
        return J / T

    def gradient(self, phi_np, T, region, kind="ke"):
        phi = torch.tensor(np.asarray(phi_np, dtype=np.float64), requires_grad=True)
        J = self.objective(phi, T, region, kind=kind)
        J.backward()
        return float(J.detach()), phi.grad.detach().numpy()
