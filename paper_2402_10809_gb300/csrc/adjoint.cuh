// Discrete adjoint of the fused VANSE LBM time step (reverse mode of the step
// in kernels.cuh), for gradients of a sac objective with respect to the
// porosity field phi (Sec. 2: phi is the coil's volume fraction complement,
// the design variable of a coil distribution).
//
// Notation.  S(t) is the stored post-collision state of time t (deviation
// form), omega(t) the relaxation rate of the collision of time t, f(t) the
// pre-collision populations of time t (S(t-1) pulled, boundary conditions of
// time t applied).  The objective is
//     J = kappa sum_{t=1..T} sum_{y in R} rho(t, y) |u(t, y)|^2 / 2,
// kappa = 1 / (T |R|), with rho and u from f(t) as in the collision of time t,
// or (obj_kind 1) the same time-and-region mean of the wall-shear-stress proxy
// |tau(t, y)| of lbm_wall_shear over the cells of R with wall links.
// The adjoint states are lambda(t) = dJ/dS(t) (FP32, same [Q][n_store] layout) and
// mu(t) = dJ/domega(t) (per slot).
//
// The pull of step t reads every slot of S(t-1) exactly once (normal pull by
// y + c_i, or the cell's own bounce-back), so its transpose is a permutation:
// each cell writes the adjoints of its pulled values straight back to their
// source slots, without atomics.  Two couplings reach other cells:
//  * the porosity link term w_i (rho - 1)(phi(y + c_i) - phi(y)) of the
//    collision at time t-1 gives dJ/dphi(y + c_i); the receiving cell gathers
//    it while it writes lambda(t-1)[y, i], using rho(t-1) - 1 of the source cell;
//  * the extrapolation outlet reads its interior neighbour's pulled values;
//    its contributions go to a small per-outlet buffer that a fix-up kernel
//    adds to the neighbour's source slots after the main kernel.
// dJ/dphi accumulates in FP64 per slot; the host scatters it to the caller's
// dense array at the end.
#pragma once

#include "kernels.cuh"

namespace lbm {

struct AdjParams {
    Params F;               // forward parameters: F.fsrc = S(t-1), F.omega = omega(t-1), F.t = t
    const float* lam_in;    // lambda(t) [Q][n_store] (not read when first)
    float* lam_out;         // lambda(t-1) [Q][n_store] (not written when last)
    float* mu;              // [n_store]: mu(t) in, mu(t-1) out
    const float* drho_prev; // [n_store] rho(t-1) - 1: porosity-link gather (not read when last)
    double* gphi;           // [n_store] dJ/dphi, accumulated
    const uint8_t* region;  // dense objective region R
    float kappa;            // 1 / (T |R|)
    int obj_kind;           // 0: rho |u|^2 / 2 over R; 1: wall-shear-stress proxy |tau| over R's wall cells
    int first;              // t = T: no collision of time t in the objective's history
    int objective;          // t >= 1: the kinetic-energy term of time t belongs to J
    int last;               // t = 0: S(-1) and omega(-1) are constants
    const uint32_t* out_slots;  // [n_out] slots of the outlet cells, ascending
    uint32_t* out_ord;          // [n_store] ordinal of each outlet slot in out_slots (others unused)
    int n_out;
    float* bnd_delta;       // [Q][n_out]: outlet contributions to the neighbour's slots
    double* bnd_dphi;       // [n_out]: outlet contribution to the neighbour's porosity
    double* jpart;          // [blocks][kBlock / 32]: per-warp sums of the objective (accumulated over launches)
};

// out_ord[out_slots[q]] = q, once per adjoint call.
template <int Q>
__global__ void adjoint_outlet_ordinals(const AdjParams A)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < A.n_out) A.out_ord[A.out_slots[q]] = (uint32_t)q;
}

// ------------------------------------------------------------------ pieces

// d alpha / d phi and d C1 / d phi of the coefficients of the explicit
// velocity solve, alpha = K1 / (4 phi), C1 = K2 / (2 phi) (see darcy_coeffs).
__device__ __forceinline__ void darcy_derivs(const Params& P, float phi, float iphi, float& dalpha, float& dc1)
{
    if (P.drag_kc) {
        // alpha = A (1-phi)^2 / (4 phi^2), C1 = B (1-phi) / (2 phi)
        const float s = 1.0f - phi;
        dalpha = -0.5f * P.drag_a * s * iphi * iphi * iphi;
        dc1 = -0.5f * P.drag_b * iphi * iphi;
    } else if (phi < 1.0f) {
        // alpha = A phi / 4, C1 = B sqrt(phi) / 2
        dalpha = 0.25f * P.drag_a;
        dc1 = 0.25f * P.drag_b * rsqrtf(phi);
    } else {
        dalpha = 0.0f;
        dc1 = 0.0f;
    }
}

// Reverse of macroscopic(): given the adjoints of its outputs (rho, rho - 1,
// sigma, sd as used directly, u, F), adds the adjoints of its inputs: sd
// (returned), the first moment m and phi.
struct MacroBar {
    float rho, drho, sigma, sd;
    float ux, uy, uz, Fx, Fy, Fz;
};

__device__ __forceinline__ float macro_adjoint(const Params& P, float phi, float mx, float my, float mz,
                                               const Macro& M, MacroBar b, float& mbx, float& mby, float& mbz,
                                               float& phib)
{
    const float iphi = __frcp_rn(phi);
    const float isig = __fdividef(1.0f, M.sigma);
    const float hg = 0.5f * iphi;
    const float vx = fmaf(P.gx, hg, mx * isig);
    const float vy = fmaf(P.gy, hg, my * isig);
    const float vz = fmaf(P.gz, hg, mz * isig);
    float k1, k2;
    darcy_coeffs(P, phi, iphi, k1, k2);
    const float alpha = 0.25f * k1 * iphi;
    const float c1 = 0.5f * k2 * iphi;
    const float vn = sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
    const float c1v = c1 * vn;
    const float c0 = 0.5f + alpha;
    const float r = sqrtf(fmaf(c0, c0, c1v));
    const float dm1 = alpha + __fdividef(fmaf(alpha, alpha, alpha + c1v), r + 0.5f);
    const float id = __fdividef(1.0f, 1.0f + dm1);
    // F = rho g - 2 sigma (D - 1) u
    b.rho += fmaf(b.Fx, P.gx, fmaf(b.Fy, P.gy, b.Fz * P.gz));
    const float Fu = fmaf(b.Fx, M.ux, fmaf(b.Fy, M.uy, b.Fz * M.uz));
    b.sigma -= 2.0f * dm1 * Fu;
    float dm1b = -2.0f * M.sigma * Fu;
    const float s2 = 2.0f * M.sigma * dm1;
    b.ux -= s2 * b.Fx;
    b.uy -= s2 * b.Fy;
    b.uz -= s2 * b.Fz;
    // u = v / D
    float vbx = b.ux * id, vby = b.uy * id, vbz = b.uz * id;
    dm1b -= fmaf(b.ux, M.ux, fmaf(b.uy, M.uy, b.uz * M.uz)) * id;
    // D - 1 = c0 + sqrt(c0^2 + C1 |v|) - 1, c0 = 1/2 + alpha
    const float ir = __fdividef(1.0f, r);
    const float alphab = dm1b * fmaf(c0, ir, 1.0f);
    const float c1vb = 0.5f * dm1b * ir;
    const float c1b = c1vb * vn;
    if (vn > 0.0f) {
        const float k = c1vb * c1 * __fdividef(1.0f, vn);
        vbx = fmaf(k, vx, vbx);
        vby = fmaf(k, vy, vby);
        vbz = fmaf(k, vz, vbz);
    }
    // v = m / sigma + g / (2 phi)
    mbx = vbx * isig;
    mby = vby * isig;
    mbz = vbz * isig;
    b.sigma -= fmaf(vbx, mx, fmaf(vby, my, vbz * mz)) * isig * isig;
    phib -= 0.5f * fmaf(vbx, P.gx, fmaf(vby, P.gy, vbz * P.gz)) * iphi * iphi;
    float dalpha, dc1;
    darcy_derivs(P, phi, iphi, dalpha, dc1);
    phib = fmaf(alphab, dalpha, fmaf(c1b, dc1, phib));
    // in the independent variables (phi, sd): sigma = phi + sd and
    // rho = 1 + sd / phi, so d rho / d phi = -(rho - 1) / phi (taking it as
    // d(sigma/phi) would cancel two O(1) terms at rho ~ 1)
    const float rd = (b.rho + b.drho) * iphi;
    b.sd += b.sigma + rd;
    phib += b.sigma - rd * M.drho;
    return b.sd;
}

// Reverse of macroscopic_aniso() at a cell with phi < 1, same interface as
// macro_adjoint.  Forward: v = m / sigma + g / (2 phi); u solves
// G(u) = (Id + Ah + |u| B) u - v = 0 with Ah = a(phi) S, B = b(phi) S^{1/2}
// (a = 2 alpha, b = C1 of the isotropic closure); F = rho g - 2 sigma w,
// w = Ah u + |u| B u.  Reverse: wbar = -2 sigma Fbar; ubar gains
// Ah wbar + |u| B wbar + (wbar . B u) u / |u|; the implicit function gives
// vbar = lambda with J^T lambda = ubar, J = dG/du = Id + Ah + |u| B + (B u) u^T / |u|;
// phi enters through a and b: phibar += (a'/a) (wbar - lambda) . Ah u +
// (b'/b) |u| (wbar - lambda) . B u (Ah u / a = S u, B u / b = S^{1/2} u).
__device__ __forceinline__ float macro_adjoint_aniso(const Params& P, int p, float phi, float mx, float my, float mz,
                                                     const Macro& M, MacroBar b, float& mbx, float& mby, float& mbz,
                                                     float& phib)
{
    const float iphi = __frcp_rn(phi);
    const float isig = __fdividef(1.0f, M.sigma);
    const size_t n = (size_t)P.n_store;
    const float* q = P.aniso + p;
    const float axx = __ldg(q), ayy = __ldg(q + n), azz = __ldg(q + 2 * n);
    const float axy = __ldg(q + 3 * n), axz = __ldg(q + 4 * n), ayz = __ldg(q + 5 * n);
    const float bxx = __ldg(q + 6 * n), byy = __ldg(q + 7 * n), bzz = __ldg(q + 8 * n);
    const float bxy = __ldg(q + 9 * n), bxz = __ldg(q + 10 * n), byz = __ldg(q + 11 * n);
    const float ux = M.ux, uy = M.uy, uz = M.uz;
    const float un = sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
    const float iun = un > 0.0f ? __fdividef(1.0f, un) : 0.0f;
    const float hx = ux * iun, hy = uy * iun, hz = uz * iun;
    // A u and B u
    const float Aux = fmaf(axx, ux, fmaf(axy, uy, axz * uz));
    const float Auy = fmaf(axy, ux, fmaf(ayy, uy, ayz * uz));
    const float Auz = fmaf(axz, ux, fmaf(ayz, uy, azz * uz));
    const float Bux = fmaf(bxx, ux, fmaf(bxy, uy, bxz * uz));
    const float Buy = fmaf(bxy, ux, fmaf(byy, uy, byz * uz));
    const float Buz = fmaf(bxz, ux, fmaf(byz, uy, bzz * uz));
    const float wx = fmaf(un, Bux, Aux), wy = fmaf(un, Buy, Auy), wz = fmaf(un, Buz, Auz);
    // F = rho g - 2 sigma w
    b.rho += fmaf(b.Fx, P.gx, fmaf(b.Fy, P.gy, b.Fz * P.gz));
    b.sigma -= 2.0f * fmaf(b.Fx, wx, fmaf(b.Fy, wy, b.Fz * wz));
    const float wbx = -2.0f * M.sigma * b.Fx, wby = -2.0f * M.sigma * b.Fy, wbz = -2.0f * M.sigma * b.Fz;
    // ubar += A wbar + |u| B wbar + (wbar . B u) u / |u|
    const float wBu = fmaf(wbx, Bux, fmaf(wby, Buy, wbz * Buz));
    const float ubx = b.ux + fmaf(axx, wbx, fmaf(axy, wby, axz * wbz)) +
                      fmaf(un, fmaf(bxx, wbx, fmaf(bxy, wby, bxz * wbz)), wBu * hx);
    const float uby = b.uy + fmaf(axy, wbx, fmaf(ayy, wby, ayz * wbz)) +
                      fmaf(un, fmaf(bxy, wbx, fmaf(byy, wby, byz * wbz)), wBu * hy);
    const float ubz = b.uz + fmaf(axz, wbx, fmaf(ayz, wby, azz * wbz)) +
                      fmaf(un, fmaf(bxz, wbx, fmaf(byz, wby, bzz * wbz)), wBu * hz);
    // J^T = Id + A + |u| B + h (B u)^T: element (r, c) = sym(r, c) + h_r (Bu)_c
    const float j00 = 1.0f + fmaf(un, bxx, axx) + hx * Bux, j01 = fmaf(un, bxy, axy) + hx * Buy,
                j02 = fmaf(un, bxz, axz) + hx * Buz;
    const float j10 = fmaf(un, bxy, axy) + hy * Bux, j11 = 1.0f + fmaf(un, byy, ayy) + hy * Buy,
                j12 = fmaf(un, byz, ayz) + hy * Buz;
    const float j20 = fmaf(un, bxz, axz) + hz * Bux, j21 = fmaf(un, byz, ayz) + hz * Buy,
                j22 = 1.0f + fmaf(un, bzz, azz) + hz * Buz;
    // lambda = (J^T)^{-1} ubar by the adjugate
    const float c00 = fmaf(j11, j22, -j12 * j21), c01 = fmaf(j02, j21, -j01 * j22), c02 = fmaf(j01, j12, -j02 * j11);
    const float c10 = fmaf(j12, j20, -j10 * j22), c11 = fmaf(j00, j22, -j02 * j20), c12 = fmaf(j02, j10, -j00 * j12);
    const float c20 = fmaf(j10, j21, -j11 * j20), c21 = fmaf(j01, j20, -j00 * j21), c22 = fmaf(j00, j11, -j01 * j10);
    const float idet = __frcp_rn(fmaf(j00, c00, fmaf(j01, c10, j02 * c20)));
    const float lx = fmaf(c00, ubx, fmaf(c01, uby, c02 * ubz)) * idet;
    const float ly = fmaf(c10, ubx, fmaf(c11, uby, c12 * ubz)) * idet;
    const float lz = fmaf(c20, ubx, fmaf(c21, uby, c22 * ubz)) * idet;
    // phi through a(phi) = 2 alpha and b(phi) = C1
    float k1, k2, dalpha, dc1;
    darcy_coeffs(P, phi, iphi, k1, k2);
    darcy_derivs(P, phi, iphi, dalpha, dc1);
    const float alpha = 0.25f * k1 * iphi, c1 = 0.5f * k2 * iphi;
    const float dx = wbx - lx, dy = wby - ly, dz = wbz - lz;
    if (alpha > 0.0f) phib = fmaf(__fdividef(dalpha, alpha), fmaf(dx, Aux, fmaf(dy, Auy, dz * Auz)), phib);
    if (c1 > 0.0f) phib = fmaf(__fdividef(dc1, c1) * un, fmaf(dx, Bux, fmaf(dy, Buy, dz * Buz)), phib);
    // v = m / sigma + g / (2 phi)
    mbx = lx * isig;
    mby = ly * isig;
    mbz = lz * isig;
    b.sigma -= fmaf(lx, mx, fmaf(ly, my, lz * mz)) * isig * isig;
    phib -= 0.5f * fmaf(lx, P.gx, fmaf(ly, P.gy, lz * P.gz)) * iphi * iphi;
    const float rd = (b.rho + b.drho) * iphi;
    b.sd += b.sigma + rd;
    phib += b.sigma - rd * M.drho;
    return b.sd;
}

// Reverse of zou_he() in place on park (adjoints of the populations after the
// boundary condition in, adjoints of the pulled populations out; the unknown
// slots end at zero).  The condition is affine in the pulled populations and
// in phi of the inlet cell: with P = phi rho = (g0 + 2 gm + phi) / (1 - ub.n),
// unknown g_i = g_opp + 6 w_i P (c_i.ub).
template <int Q>
__device__ __forceinline__ void zou_he_adjoint(const Params& P, float prof, volatile float* park, float& phib)
{
    using L = Lattice<Q>;
    const int ax = P.in_axis;
    const int sgn = P.in_side == 0 ? 1 : -1;
    const float un = (float)((double)prof * inflow_mean(P, P.t));
    const float ubx = -0.5f * P.gx + (ax == 0 ? sgn * un : 0.0f);
    const float uby = -0.5f * P.gy + (ax == 1 ? sgn * un : 0.0f);
    const float ubz = -0.5f * P.gz + (ax == 2 ? sgn * un : 0.0f);
    const float ubn = (ax == 0 ? ubx : ax == 1 ? uby : ubz) * sgn;
    const float inv = 1.0f / (1.0f - ubn);
    float Pb = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (c_axis<Q>(i, ax) * sgn > 0) {
            const float a = park[i * kBlock];
            const float cu = cdot(L::cx(i), L::cy(i), L::cz(i), ubx, uby, ubz);
            park[opp(i) * kBlock] += a;
            Pb += 6.0f * L::w(i) * cu * a;
            park[i * kBlock] = 0.0f;
        }
    }
    const float pw = Pb * inv;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int cn = c_axis<Q>(k, ax) * sgn;
        if (cn == 0) park[k * kBlock] += pw;
        if (cn < 0) park[k * kBlock] += 2.0f * pw;
    }
    phib += pw;
}

// Reverse of outlet(): the unknown populations
//   g_i = w_i phi (rho_out - 1) + w_i (phi rho_out - sigma_nb) pe_i(u_nb) + g_nb,i - w_i sd_nb
// depend on this cell's phi and on the interior neighbour nb (its pulled
// populations and phi).  The neighbour's part is stored for the fix-up kernel;
// the unknown slots of this cell end at zero.
template <int Q, class T>
__device__ __forceinline__ void outlet_adjoint(const AdjParams& A, const Coords& c, float phi, int p,
                                               volatile float* park, float& phib)
{
    using L = Lattice<Q>;
    const Params& P = A.F;
    const int ax = P.out_axis;
    const int sgn = P.out_side == 1 ? -1 : 1;
    const uint32_t nbmask = P.bnd_nbmask[p];
    const int q = (int)A.out_ord[p];
    const Coords nc = make_coords(P, c.x + (ax == 0 ? sgn : 0), c.y + (ax == 1 ? sgn : 0), c.z + (ax == 2 ? sgn : 0));
    const float phin = __ldg(P.phi + nc.slot);
    const T* f = static_cast<const T*>(P.fsrc);
    float sd = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float v = Store<T>::ld(f + pull_offset<Q>(P, nc, nbmask, i));
        sd += v;
        if (L::cx(i)) mx += L::cx(i) > 0 ? v : -v;
        if (L::cy(i)) my += L::cy(i) > 0 ? v : -v;
        if (L::cz(i)) mz += L::cz(i) > 0 ? v : -v;
    }
    const Macro M = macroscopic(P, phin, sd, mx, my, mz);
    const float uu = M.ux * M.ux + M.uy * M.uy + M.uz * M.uz;
    // phi rho_out - sigma_nb without cancelling O(1) terms
    const float sfac = fmaf(phi, P.rho_out - 1.0f, (phi - phin) - M.sd);
    MacroBar b{};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (c_axis<Q>(i, ax) * sgn > 0) {
            const float d = park[i * kBlock];
            const float w = L::w(i);
            const float cu = cdot(L::cx(i), L::cy(i), L::cz(i), M.ux, M.uy, M.uz);
            const float pe = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
            phib += d * w * (P.rho_out - 1.0f + P.rho_out * pe);
            b.sigma -= d * w * pe;
            b.sd -= d * w;
            // d pe / d u = 3 c + 9 (c.u) c - 3 u
            const float k = d * w * sfac;
            const float kc = k * fmaf(9.0f, cu, 3.0f);
            b.ux += (L::cx(i) ? (L::cx(i) > 0 ? kc : -kc) : 0.0f) - 3.0f * k * M.ux;
            b.uy += (L::cy(i) ? (L::cy(i) > 0 ? kc : -kc) : 0.0f) - 3.0f * k * M.uy;
            b.uz += (L::cz(i) ? (L::cz(i) > 0 ? kc : -kc) : 0.0f) - 3.0f * k * M.uz;
        }
    }
    float mbx, mby, mbz, phinb = 0.0f;
    const float sdb = macro_adjoint(P, phin, mx, my, mz, M, b, mbx, mby, mbz, phinb);
    const int nb_count = A.n_out;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        float d = sdb;
        if (L::cx(j)) d += L::cx(j) > 0 ? mbx : -mbx;
        if (L::cy(j)) d += L::cy(j) > 0 ? mby : -mby;
        if (L::cz(j)) d += L::cz(j) > 0 ? mbz : -mbz;
        if (c_axis<Q>(j, ax) * sgn > 0) {
            d += park[j * kBlock];
            park[j * kBlock] = 0.0f;
        }
        A.bnd_delta[(size_t)j * nb_count + q] = d;
    }
    A.bnd_dphi[q] = phinb;
}

// ------------------------------------------------------------------ the cell

// Reverse of one cell of the time step t (see cell_impl): recompute the
// forward quantities from S(t-1), omega(t-1), form the adjoints of the pulled
// populations and write them to lambda(t-1) at the source slots; add the
// cell's dJ/dphi terms; write mu(t-1).  jv accumulates the objective term.
// park / lampark / dpark: this thread's columns of three Q x kBlock shared
// arrays (pulled populations, lambda(t) at the cell's slots, rho(t-1) - 1 at
// its pull sources), all filled by asynchronous copies issued at the start so
// that their latencies overlap; the per-cell scalars are loaded before any
// wait for the same reason.
// Lean cells (fast) get their row id, porosity, omega(t-1) and mu(t) from the
// caller, which loads them together with the mask.
template <int Q, class T, bool fast, bool AN>
__device__ __forceinline__ void adjoint_cell(const AdjParams& A, int p, uint32_t mask, volatile float* park,
                                             volatile float* lampark, volatile float* dpark, double& jv,
                                             uint32_t row_pre = 0, float phi_pre = 0.0f, float om_pre = 0.0f,
                                             float mu_pre = 0.0f)
{
    using L = Lattice<Q>;
    const Params& P = A.F;
    const float phi = fast ? phi_pre : __ldg(P.phi + p);
    const float om_prev = fast ? om_pre : P.omega[p];
    const float bmu = A.first ? 0.0f : (fast ? mu_pre : A.mu[p]);
    const double gphi0 = A.gphi[p];
    const bool porous = (mask & kPorousBit) != 0u;
    const T* __restrict__ fs = static_cast<const T*>(P.fsrc);
    const uint32_t n = (uint32_t)P.n_store;
    int type = kBulk;
    Coords cg;
    RowBases rb;
    int x = 0;
    uint32_t row = 0;
    {
        float g[Q];
        constexpr bool f32 = sizeof(T) == 4;
        if (!A.first) {
#pragma unroll
            for (int i = 0; i < Q; ++i) cp_async4(lampark + i * kBlock, A.lam_in + (size_t)i * n + p);
        }
        if (fast) {
            row = row_pre;
            rb = row_bases(P, row);
            x = p - rb.b[4];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = ((mask >> i) & 1u) != 0u;
                const uint32_t src = lean_slot(rb, x, -L::cx(i), -L::cy(i), -L::cz(i));
                const uint32_t o = bb ? (uint32_t)opp(i) * n + (uint32_t)p : (uint32_t)i * n + src;
                if (f32)
                    cp_async4(park + i * kBlock, reinterpret_cast<const float*>(fs) + o);
                else
                    g[i] = Store<T>::ld(fs + o);
                if (!A.last && !bb && i != 0) cp_async4(dpark + i * kBlock, A.drho_prev + src);
            }
            cp_async_wait_all();
        } else {
            cg = coords_of(P, p);
            if (!A.last) {
#pragma unroll
                for (int i = 1; i < Q; ++i)
                    if (!((mask >> i) & 1u))
                        cp_async4(dpark + i * kBlock,
                                  A.drho_prev + shifted(P, cg, -L::cx(i), -L::cy(i), -L::cz(i)));
            }

            pull_general<Q, T>(P, fs, cg, mask, g);
            cp_async_wait_all();
            type = (mask >> kTypeShift) & 3u;
            if (type == kInlet) {
                zou_he<Q>(P, P.bnd_prof[p], g);
            } else if (type == kOutlet) {
                outlet<Q, T>(P, cg, phi, P.bnd_nbmask[p], g);
            }
        }
        if (!(fast && f32)) {  // the FP32 lean pull already sits in park
#pragma unroll
            for (int i = 0; i < Q; ++i) park[i * kBlock] = g[i];
        }
    }
    // ---- forward recompute (as in cell_impl)
    float smx, smy, smz;
    Macro M;
    float pxx, pyy, pzz, pxy, pxz, pyz;
    {
        float g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = park[i * kBlock];
        const Moments<Q> m = moments<Q>(g);
        smx = m.mx;
        smy = m.my;
        smz = m.mz;
        if constexpr (AN)
            M = macroscopic_aniso(P, p, phi, m.sd, m.mx, m.my, m.mz);
        else
            M = macroscopic(P, phi, m.sd, m.mx, m.my, m.mz);
        const float sd3 = M.sd * (1.0f / 3.0f);
        pxx = fmaf(M.ux, fmaf(-M.sigma, M.ux, M.Fx), m.sxx - sd3);
        pyy = fmaf(M.uy, fmaf(-M.sigma, M.uy, M.Fy), m.syy - sd3);
        pzz = fmaf(M.uz, fmaf(-M.sigma, M.uz, M.Fz), m.szz - sd3);
        pxy = fmaf(M.ux, fmaf(-M.sigma, M.uy, 0.5f * M.Fy), fmaf(0.5f * M.Fx, M.uy, m.sxy));
        pxz = fmaf(M.ux, fmaf(-M.sigma, M.uz, 0.5f * M.Fz), fmaf(0.5f * M.Fx, M.uz, m.sxz));
        pyz = fmaf(M.uy, fmaf(-M.sigma, M.uz, 0.5f * M.Fz), fmaf(0.5f * M.Fy, M.uz, m.syz));
    }
    const float pn = sqrtf(fmaf(pxx, pxx, fmaf(pyy, pyy, fmaf(pzz, pzz, 2.0f * fmaf(pxy, pxy, fmaf(pxz, pxz, pyz * pyz))))));
    const float irho = __fdividef(1.0f, M.rho);
    const float gdot = 3.0f * om_prev * pn * irho;
    // Carreau-Yasuda viscosity and rate with the pieces of their derivatives
    const float lx = P.lam * gdot;
    const float xa = P.cy_a_two ? lx * lx : __powf(lx, P.cy_a);
    const float base = 1.0f + xa;
    const float pw = exp2f(P.cy_e * __log2f(base));
    const float mu = fmaf(P.mu0 - P.mu_inf, pw, P.mu_inf);
    const float E = fmaf(6.0f, mu, M.rho);
    const float iE = __fdividef(1.0f, E);
    const float om = 2.0f * M.rho * iE;

    // wall-shear-stress objective at a wall cell of the region: |tau| =
    // (1 - omega/2) |v|, v = (I - n n^T) Pi n; its seeds for omega and for the
    // symmetric adjoint of Pi, (1 - omega/2) (t n^T + n t^T) / 2 with t = v / |v|
    float w_om = 0.0f, wxx = 0.0f, wyy = 0.0f, wzz = 0.0f, wxy = 0.0f, wxz = 0.0f, wyz = 0.0f;
    if (A.objective && A.obj_kind == 1 && type == kBulk &&
        A.region[fast ? (long long)x + (long long)P.nx * row : cg.idx]) {
        float nx = 0.0f, ny = 0.0f, nz = 0.0f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if ((mask >> opp(i)) & 1u) {
                nx += L::w(i) * L::cx(i);
                ny += L::w(i) * L::cy(i);
                nz += L::w(i) * L::cz(i);
            }
        }
        const float nn = sqrtf(nx * nx + ny * ny + nz * nz);
        if (nn > 0.0f) {
            nx /= nn;
            ny /= nn;
            nz /= nn;
            const float qx = fmaf(pxx, nx, fmaf(pxy, ny, pxz * nz));
            const float qy = fmaf(pxy, nx, fmaf(pyy, ny, pyz * nz));
            const float qz = fmaf(pxz, nx, fmaf(pyz, ny, pzz * nz));
            const float qn = fmaf(qx, nx, fmaf(qy, ny, qz * nz));
            const float vx = qx - qn * nx, vy = qy - qn * ny, vz = qz - qn * nz;
            const float vn = sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
            const float h2 = fmaf(-0.5f, om, 1.0f);
            jv += (double)A.kappa * (double)(h2 * vn);
            w_om = -0.5f * A.kappa * vn;
            if (vn > 0.0f) {
                const float k = A.kappa * h2 / vn;
                wxx = k * vx * nx;
                wyy = k * vy * ny;
                wzz = k * vz * nz;
                wxy = 0.5f * k * fmaf(vx, ny, vy * nx);
                wxz = 0.5f * k * fmaf(vx, nz, vz * nx);
                wyz = 0.5f * k * fmaf(vy, nz, vz * ny);
            }
        }
    }

    // ---- reverse of the collision: out_i = (1 - omega) g_i
    //      + w_i [omega (sd + sigma pe_i) + (1 - omega/2) q_i] + w_i (rho - 1)(phi_i - phi),
    // pe_i = 3 c.u + 4.5 (c.u)^2 - 1.5 u.u, q_i = 3 c.F - 3 u.F + 9 (c.u)(c.F).
    MacroBar b{};
    float omb = 0.0f, phib = 0.0f;
    if (!A.first) {
        float h[Q];
        float Ag = 0.0f, Wd = 0.0f, Aphi = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float a = lampark[i * kBlock];
            Ag = fmaf(a, park[i * kBlock], Ag);
            h[i] = L::w(i) * a;
            // the link term exists where y + c_i (i != 0) is a fluid cell that
            // pulls from y (mask bit of the opposite direction clear)
            if (i != 0 && !((mask >> opp(i)) & 1u)) {
                Wd += h[i];
                if (porous) {
                    const uint32_t ni = fast ? lean_slot(rb, x, L::cx(i), L::cy(i), L::cz(i))
                                             : (uint32_t)shifted(P, cg, L::cx(i), L::cy(i), L::cz(i));
                    Aphi = fmaf(h[i], __ldg(P.phi + ni) - phi, Aphi);
                }
            }
        }
        const Moments<Q> am = moments<Q>(h);  // A0, A1, A2 = sums of w a, w a c, w a c c
        const float A0 = am.sd;
        const float uu = fmaf(M.ux, M.ux, fmaf(M.uy, M.uy, M.uz * M.uz));
        const float uF = fmaf(M.ux, M.Fx, fmaf(M.uy, M.Fy, M.uz * M.Fz));
        // A2 u, A2 F
        const float A2ux = fmaf(am.sxx, M.ux, fmaf(am.sxy, M.uy, am.sxz * M.uz));
        const float A2uy = fmaf(am.sxy, M.ux, fmaf(am.syy, M.uy, am.syz * M.uz));
        const float A2uz = fmaf(am.sxz, M.ux, fmaf(am.syz, M.uy, am.szz * M.uz));
        const float A2Fx = fmaf(am.sxx, M.Fx, fmaf(am.sxy, M.Fy, am.sxz * M.Fz));
        const float A2Fy = fmaf(am.sxy, M.Fx, fmaf(am.syy, M.Fy, am.syz * M.Fz));
        const float A2Fz = fmaf(am.sxz, M.Fx, fmaf(am.syz, M.Fy, am.szz * M.Fz));
        const float A1u = fmaf(am.mx, M.ux, fmaf(am.my, M.uy, am.mz * M.uz));
        const float A1F = fmaf(am.mx, M.Fx, fmaf(am.my, M.Fy, am.mz * M.Fz));
        const float uA2u = fmaf(A2ux, M.ux, fmaf(A2uy, M.uy, A2uz * M.uz));
        const float uA2F = fmaf(A2Fx, M.ux, fmaf(A2Fy, M.uy, A2Fz * M.uz));
        const float Ape = 3.0f * A1u + 4.5f * uA2u - 1.5f * uu * A0;
        const float Aq = 3.0f * A1F - 3.0f * uF * A0 + 9.0f * uA2F;
        const float h2 = fmaf(-0.5f, om, 1.0f);
        omb = bmu - Ag + M.sd * A0 + M.sigma * Ape - 0.5f * Aq;
        b.sd = om * A0;
        b.sigma = om * Ape;
        b.drho = Aphi;
        // Bu = 3 A1 + 9 A2 u - 3 A0 u, BF = 9 A2 F - 3 A0 F
        const float Bux = 3.0f * am.mx + 9.0f * A2ux - 3.0f * A0 * M.ux;
        const float Buy = 3.0f * am.my + 9.0f * A2uy - 3.0f * A0 * M.uy;
        const float Buz = 3.0f * am.mz + 9.0f * A2uz - 3.0f * A0 * M.uz;
        const float os = om * M.sigma;
        b.ux = os * Bux + h2 * (9.0f * A2Fx - 3.0f * A0 * M.Fx);
        b.uy = os * Buy + h2 * (9.0f * A2Fy - 3.0f * A0 * M.Fy);
        b.uz = os * Buz + h2 * (9.0f * A2Fz - 3.0f * A0 * M.Fz);
        b.Fx = h2 * Bux;
        b.Fy = h2 * Buy;
        b.Fz = h2 * Buz;
        phib = -M.drho * Wd;
    }
    omb += w_om;
    // omega = 2 rho / (6 mu + rho)
    b.rho = omb * 12.0f * mu * iE * iE;
    const float mub = -omb * 12.0f * M.rho * iE * iE;
    // mu = mu_inf + (mu0 - mu_inf)(1 + x^a)^((n-1)/a):
    // dmu/dx = (mu0 - mu_inf)(n - 1)(1 + x^a)^((n-1)/a - 1) x^(a-1)
    const float xam1 = P.cy_a_two ? lx : (lx > 0.0f ? __fdividef(xa, lx) : 0.0f);
    const float dmudx = (P.mu0 - P.mu_inf) * (P.cy_e * P.cy_a) * __fdividef(pw, base) * xam1;
    const float gdb = P.lam * mub * dmudx;
    // gdot = 3 omega(t-1) |Pi| / rho
    const float mu_prev = gdb * 3.0f * pn * irho;
    const float pnb = gdb * 3.0f * om_prev * irho;
    b.rho -= gdb * gdot * irho;
    // objective term of time t
    if (A.objective && A.obj_kind == 0 && A.region[fast ? (long long)x + (long long)P.nx * row : cg.idx]) {
        const float uu = fmaf(M.ux, M.ux, fmaf(M.uy, M.uy, M.uz * M.uz));
        jv += (double)A.kappa * 0.5 * (double)M.rho * (double)uu;
        b.rho = fmaf(0.5f * A.kappa, uu, b.rho);
        const float kr = A.kappa * M.rho;
        b.ux = fmaf(kr, M.ux, b.ux);
        b.uy = fmaf(kr, M.uy, b.uy);
        b.uz = fmaf(kr, M.uz, b.uz);
    }
    // Pi = S - (sd/3) I - sigma u u^T + (F u^T + u F^T) / 2, |Pi| its Frobenius norm
    const float s = pn > 0.0f ? __fdividef(pnb, pn) : 0.0f;
    const float bxx = fmaf(s, pxx, wxx), byy = fmaf(s, pyy, wyy), bzz = fmaf(s, pzz, wzz);
    const float bxy = fmaf(s, pxy, wxy), bxz = fmaf(s, pxz, wxz), byz = fmaf(s, pyz, wyz);
    {
        const float Pux = fmaf(bxx, M.ux, fmaf(bxy, M.uy, bxz * M.uz));
        const float Puy = fmaf(bxy, M.ux, fmaf(byy, M.uy, byz * M.uz));
        const float Puz = fmaf(bxz, M.ux, fmaf(byz, M.uy, bzz * M.uz));
        const float PFx = fmaf(bxx, M.Fx, fmaf(bxy, M.Fy, bxz * M.Fz));
        const float PFy = fmaf(bxy, M.Fx, fmaf(byy, M.Fy, byz * M.Fz));
        const float PFz = fmaf(bxz, M.Fx, fmaf(byz, M.Fy, bzz * M.Fz));
        const float ts = -2.0f * M.sigma;
        b.ux += fmaf(ts, Pux, PFx);
        b.uy += fmaf(ts, Puy, PFy);
        b.uz += fmaf(ts, Puz, PFz);
        b.Fx += Pux;
        b.Fy += Puy;
        b.Fz += Puz;
        b.sigma -= fmaf(Pux, M.ux, fmaf(Puy, M.uy, Puz * M.uz));
        b.sd -= (bxx + byy + bzz) * (1.0f / 3.0f);
    }
    float mbx, mby, mbz;
    float sdb;
    if (AN && phi < 1.0f)
        sdb = macro_adjoint_aniso(P, p, phi, smx, smy, smz, M, b, mbx, mby, mbz, phib);
    else
        sdb = macro_adjoint(P, phi, smx, smy, smz, M, b, mbx, mby, mbz, phib);

    // ---- adjoints of the populations after the boundary condition:
    // gbar_i = (1 - omega) a_i + sdbar + mbar.c_i + c_i^T Pibar c_i (a = 0 at t = T)
    const float omo = 1.0f - om;
    auto gbar = [&](int i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        float v = A.first ? sdb : fmaf(omo, lampark[i * kBlock], sdb);
        if (cx) v += cx > 0 ? mbx : -mbx;
        if (cy) v += cy > 0 ? mby : -mby;
        if (cz) v += cz > 0 ? mbz : -mbz;
        if (cx) v += bxx;
        if (cy) v += byy;
        if (cz) v += bzz;
        if (cx && cy) v += cx * cy > 0 ? 2.0f * bxy : -2.0f * bxy;
        if (cx && cz) v += cx * cz > 0 ? 2.0f * bxz : -2.0f * bxz;
        if (cy && cz) v += cy * cz > 0 ? 2.0f * byz : -2.0f * byz;
        return v;
    };
    double gacc = (double)phib;
    float gat = 0.0f;
    if (fast) {
        // ---- transpose of the pull, written as each gbar_i is formed: lambda(t-1)
        // at the source slots, plus the porosity-link gather
        // w_i (rho(t-1, y - c_i) - 1) lambda(t-1)[y - c_i, i]
        if (!A.last) {
            float* __restrict__ lo = A.lam_out;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float v = gbar(i);
                const bool bb = ((mask >> i) & 1u) != 0u;
                const uint32_t src = lean_slot(rb, x, -L::cx(i), -L::cy(i), -L::cz(i));
                lo[bb ? (uint32_t)opp(i) * n + (uint32_t)p : (uint32_t)i * n + src] = v;
                if (!bb && i != 0) gat = fmaf(L::w(i) * dpark[i * kBlock], v, gat);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) park[i * kBlock] = gbar(i);
        if (type == kInlet) {
            zou_he_adjoint<Q>(P, P.bnd_prof[p], park, phib);
        } else if (type == kOutlet) {
            outlet_adjoint<Q, T>(A, cg, phi, p, park, phib);
        }
        gacc = (double)phib;
        if (!A.last) {
            float* __restrict__ lo = A.lam_out;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float v = park[i * kBlock];
                lo[pull_offset<Q>(P, cg, mask, i)] = v;
                if (!((mask >> i) & 1u) && i != 0) gat = fmaf(L::w(i) * dpark[i * kBlock], v, gat);
            }
        }
    }
    if (!A.last) {
        gacc += (double)gat;
        A.mu[p] = mu_prev;
    }
    A.gphi[p] = gphi0 + gacc;
}

template <int Q, class T, bool AN>
__device__ __noinline__ void adjoint_general(const AdjParams& A, int p, uint32_t mask, volatile float* park,
                                             volatile float* lampark, volatile float* dpark, double& jv)
{
    adjoint_cell<Q, T, false, AN>(A, p, mask, park, lampark, dpark, jv);
}

// Dynamic shared memory of adjoint_kernel: three Q x kBlock float arrays.  The
// kernel is compiled for 512 resident threads per SM (128 registers), which
// that shared memory allows (83 KB per 256 threads).
template <int Q>
constexpr size_t adjoint_smem_bytes()
{
    return (size_t)3 * Q * kBlock * sizeof(float);
}

// TPS: resident threads per SM the kernel is compiled for.  512 (128
// registers, some spills) hides more latency on large grids; 384 (168
// registers, no spills) runs each cell faster, which wins when the grid is
// only one or two waves (measured: 47.9 against 52.1 us per reverse step at
// 128^3, 140 against 128 us at 256^3).  AN: the reverse of the anisotropic
// velocity solve at cells with phi < 1.
template <int Q, class T, int TPS, bool AN>
__global__ void __launch_bounds__(kBlock, TPS / kBlock) adjoint_kernel(const AdjParams A)
{
    const Params& P = A.F;
    const int nbg = general_blocks(P);
    extern __shared__ float adj_smem[];
    volatile float* park = adj_smem + threadIdx.x;
    volatile float* lampark = park + Q * kBlock;
    volatile float* dpark = park + 2 * Q * kBlock;
    double jv = 0.0;
    // programmatic launch (see lbm_kernel): static words before the wait,
    // everything a previous kernel writes after it
    grid_dependents_launch();
    if ((int)blockIdx.x < nbg) {
        grid_dependency_wait();
        const int k = (int)blockIdx.x * P.gen_block + (int)threadIdx.x;
        if ((int)threadIdx.x < P.gen_block && k < P.n_general) {
            const int p = (int)P.general[k];
            adjoint_general<Q, T, AN>(A, p, P.mask[p], park, lampark, dpark, jv);
        }
    } else {
        const int p = ((int)blockIdx.x - nbg) * kBlock + (int)threadIdx.x;
        if (p >= P.n_store) grid_dependency_wait();
        if (p < P.n_store) {
            // every per-slot word of the cell at once (one memory latency
            // before the row record instead of one per word)
            const uint32_t mask = ld_early_u32(P.mask + p);
            const uint32_t row = ld_early_u32(P.rows + p);
            const float phi = ld_early_nc(P.phi + p);
            grid_dependency_wait();
            const float om = ld_early_nc(P.omega + p);
            const float mu = A.first ? 0.0f : ld_early(A.mu + p);
            // ghost slots hold no state; general cells belong to the general blocks
            if (!(mask & (kGhostBit | kGeneralBits)) && !P.wide)
                adjoint_cell<Q, T, true, AN>(A, p, mask, park, lampark, dpark, jv, row, phi, om, mu);
        }
    }
    if (A.objective) {
        // warp sum of the objective terms, added to this warp's running partial
        // (one writer per slot: deterministic, no block barrier)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) jv += __shfl_xor_sync(0xffffffffu, jv, off);
        if ((threadIdx.x & 31) == 0) A.jpart[(size_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5)] += jv;
    }
}

// Fix-up after adjoint_kernel: adds each outlet's contributions to its interior
// neighbour's source slots of lambda(t-1) (with the porosity-link gather those
// slots carry) and to the neighbour's porosity.  One thread per outlet cell.
template <int Q>
__global__ void adjoint_outlet_fixup(const AdjParams A)
{
    using L = Lattice<Q>;
    const Params& P = A.F;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.n_out) return;
    const int p = (int)A.out_slots[q];
    const Coords c = coords_of(P, p);
    const int ax = P.out_axis;
    const int sgn = P.out_side == 1 ? -1 : 1;
    const Coords nc = make_coords(P, c.x + (ax == 0 ? sgn : 0), c.y + (ax == 1 ? sgn : 0), c.z + (ax == 2 ? sgn : 0));
    const uint32_t nbmask = P.bnd_nbmask[p];
    double acc = A.bnd_dphi[q];
    if (!A.last) {
        float gat = 0.0f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float d = A.bnd_delta[(size_t)j * A.n_out + q];
            A.lam_out[pull_offset<Q>(P, nc, nbmask, j)] += d;
            if (j != 0 && !((nbmask >> j) & 1u))
                gat = fmaf(L::w(j) * A.drho_prev[shifted(P, nc, -L::cx(j), -L::cy(j), -L::cz(j))], d, gat);
        }
        acc += (double)gat;
    }
    A.gphi[nc.slot] += acc;
}

}  // namespace lbm
