// Fused pull-scheme collide-and-stream kernel for the VANSE lattice Boltzmann
// method with Carreau-Yasuda rheology (Horvat et al., arXiv 2402.10809,
// Sec. 2-4), plus the moments and diagnostics epilogues that reuse its pull.
//
// One thread owns one non-solid cell, taken from a compact cell list (bulk
// cells sorted by dense index, then inlet cells, then outlet cells), so no
// thread idles on solid voxels of the sparse aneurysm box.  The distributions
// live in two dense SoA buffers f[i][N]; a warp of consecutive list entries
// reads and writes consecutive addresses of each direction plane.
//
// Stored values are deviations g_i = f_i - w_i phi_hat_i, where phi_hat_i is
// the porosity of the cell the value streams to (own porosity across solid or
// open links).  The reading cell therefore always decodes with its own
// porosity, the rest state is g = 0 everywhere, and every balance below is
// evaluated on small numbers in FP32 registers whatever the storage type.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lattice.cuh"

namespace lbm {

// Per-cell mask word: bit i (i < Q) set when direction i cannot be pulled from
// its source y - c_i (solid, box wall, or an open face); bits 27-28 cell type;
// bit 29 set when some fluid neighbour has a different porosity.
constexpr uint32_t kTypeShift = 27;
constexpr uint32_t kPorousBit = 1u << 29;
enum { kBulk = 0, kInlet = 1, kOutlet = 2 };
enum { kModeStep = 0, kModeMoments = 1, kModeDiag = 2 };
constexpr int kBlock = 256;
constexpr int kDiagSlots = 9;

struct Params {
    // geometry
    int nx, ny, nz;
    long long N;
    int n_cells, n_bulk;
    const uint32_t* cells;    // packed x | y << 10 | z << 20, list order
    const uint32_t* mask;     // list order
    const float* phi;         // dense porosity
    const float* bnd_prof;    // [n_cells - n_bulk]: inlet profile 2 max(0, 1 - r^2/R^2)
    const uint32_t* bnd_nbmask;  // [n_cells - n_bulk]: mask of the outlet's interior neighbour
    // physics, lattice units
    float gx, gy, gz;         // body force per unit mass
    int drag_kc;              // 1 Kozeny-Carman, 0 constant permeability
    float drag_a, drag_b;     // see darcy_coeffs
    float mu0, mu_inf, lam, cy_a, cy_e;  // Carreau-Yasuda, cy_e = (n - 1) / a
    int cy_a_two;             // a == 2: (lambda gdot)^a as a square
    // open boundaries
    int in_axis, in_side, out_axis, out_side;
    double u0, amp, period, ramp;
    float rho_out;
    // state
    const void* fsrc;
    void* fdst;
    float* omega;             // list order; omega(t-1) in, omega(t) out
    long long t;
    // moments outputs (dense or list order, any may be null)
    float *o_rho, *o_ux, *o_uy, *o_uz, *o_gdot, *o_omega;
    int o_compact;
    // diagnostics
    const uint8_t* region;    // dense, may be null
    double* partials;         // [gridDim.x][kDiagSlots]
};

// ------------------------------------------------------------------ storage

template <class T>
struct Store;

template <>
struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { __stcs(p, v); }
};

template <>
struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
};

template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { __stcs(p, __float2bfloat16_rn(v)); }
};

// ------------------------------------------------------------------ physics

// Darcy and Forchheimer coefficients K1 = phi^2 nu / k, K2 = phi^3 C_F / sqrt(k)
// of f(u) = -(K1 + K2 |u|) u (Sec. 2).  Kozeny-Carman k = phi^3 d^2 / (150 (1-phi)^2)
// with Ergun C_F = 1.75 / sqrt(150 phi^3) reduce to K1 = (150 nu / d^2)(1-phi)^2 / phi
// and K2 = (1.75 / d)(1 - phi): drag_a = 150 nu / d^2, drag_b = 1.75 / d.  For a
// constant permeability kc: K1 = (nu / kc) phi^2, K2 = (1.75 / sqrt(150 kc)) phi^1.5,
// only where phi < 1.
__device__ __forceinline__ void darcy_coeffs(const Params& P, float phi, float& k1, float& k2)
{
    if (P.drag_kc) {
        float s = 1.0f - phi;
        k1 = P.drag_a * s * s / phi;
        k2 = P.drag_b * s;
    } else if (phi < 1.0f) {
        k1 = P.drag_a * phi * phi;
        k2 = P.drag_b * phi * sqrtf(phi);
    } else {
        k1 = 0.0f;
        k2 = 0.0f;
    }
}

struct Macro {
    float sd;      // sum_i g_i = phi rho - phi
    float sigma;   // phi rho
    float rho;
    float drho;    // rho - 1
    float ux, uy, uz;
    float Fx, Fy, Fz;  // rho (g + f_d(u))
};

// Macroscopic quantities of Sec. 3 from the deviations: rho = phi^{-1} sum f,
// u from phi rho u = sum f c + rho f(u) / 2 solved explicitly,
// u = v / (C0 + sqrt(C0^2 + C1 |v|)), v = (sum f c + rho g / 2) / (phi rho),
// C0 = 1/2 + K1 / (4 phi), C1 = K2 / (2 phi).  D - 1 is formed without
// cancellation, so f_d = -2 phi (D - 1) u keeps full precision for weak drag.
__device__ __forceinline__ Macro macroscopic(const Params& P, float phi, float sd, float mx, float my, float mz)
{
    Macro M;
    M.sd = sd;
    M.sigma = phi + sd;
    float iphi = 1.0f / phi;
    M.rho = M.sigma * iphi;
    M.drho = sd * iphi;
    float isig = 1.0f / M.sigma;
    float hg = 0.5f * iphi;
    float vx = mx * isig + P.gx * hg;
    float vy = my * isig + P.gy * hg;
    float vz = mz * isig + P.gz * hg;
    float k1, k2;
    darcy_coeffs(P, phi, k1, k2);
    float alpha = 0.25f * k1 * iphi;
    float c1 = 0.5f * k2 * iphi;
    float c1v = c1 * sqrtf(vx * vx + vy * vy + vz * vz);
    float c0 = 0.5f + alpha;
    float r = sqrtf(c0 * c0 + c1v);
    float dm1 = alpha + (alpha + alpha * alpha + c1v) / (r + 0.5f);
    float id = 1.0f / (1.0f + dm1);
    M.ux = vx * id;
    M.uy = vy * id;
    M.uz = vz * id;
    float s2 = 2.0f * M.sigma * dm1;
    M.Fx = M.rho * P.gx - s2 * M.ux;
    M.Fy = M.rho * P.gy - s2 * M.uy;
    M.Fz = M.rho * P.gz - s2 * M.uz;
    return M;
}

// Carreau-Yasuda law, Eq. (3), and omega = 2 rho c_s^2 / (2 mu + rho c_s^2).
__device__ __forceinline__ float relaxation_rate(const Params& P, float rho, float gdot)
{
    float x = P.lam * gdot;
    float xa = P.cy_a_two ? x * x : powf(x, P.cy_a);
    float mu = P.mu_inf + (P.mu0 - P.mu_inf) * exp2f(P.cy_e * log2f(1.0f + xa));
    return 2.0f * rho / (6.0f * mu + rho);
}

// ------------------------------------------------------------------ helpers

struct Coords {
    int x, y, z;
    long long idx;
    int X[3];        // x - 1, x, x + 1 (wrapped)
    long long Y[3];  // (y - 1, y, y + 1) * nx (wrapped)
    long long Z[3];  // (z - 1, z, z + 1) * nx * ny (wrapped)
};

__device__ __forceinline__ Coords make_coords(const Params& P, int x, int y, int z)
{
    Coords c;
    c.x = x; c.y = y; c.z = z;
    long long sy = P.nx, sz = (long long)P.nx * P.ny;
    c.idx = x + sy * y + sz * z;
    c.X[0] = x == 0 ? P.nx - 1 : x - 1;
    c.X[1] = x;
    c.X[2] = x == P.nx - 1 ? 0 : x + 1;
    c.Y[0] = sy * (y == 0 ? P.ny - 1 : y - 1);
    c.Y[1] = sy * y;
    c.Y[2] = sy * (y == P.ny - 1 ? 0 : y + 1);
    c.Z[0] = sz * (z == 0 ? P.nz - 1 : z - 1);
    c.Z[1] = sz * z;
    c.Z[2] = sz * (z == P.nz - 1 ? 0 : z + 1);
    return c;
}

// Dense index of y + (dx, dy, dz) with periodic wrap (dx etc. in {-1, 0, 1}).
__device__ __forceinline__ long long shifted(const Coords& c, int dx, int dy, int dz)
{
    return c.X[dx + 1] + c.Y[dy + 1] + c.Z[dz + 1];
}

// Pull of all Q deviations of a cell: g_i = f*_i(y - c_i), or the cell's own
// f*_opp(i) (half-way bounce-back, Sec. 4) where the source is not available.
template <int Q, class T>
__device__ __forceinline__ void pull(const T* __restrict__ f, long long N, const Coords& c, uint32_t mask, float* g)
{
    using L = Lattice<Q>;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        long long src = ((mask >> i) & 1u) ? (long long)opp(i) * N + c.idx
                                           : (long long)i * N + shifted(c, -L::cx(i), -L::cy(i), -L::cz(i));
        g[i] = Store<T>::ld(f + src);
    }
}

// Mean inflow v(t) = u0 (1 + amp sin(2 pi t / period)), linear ramp over the
// first ramp steps (the pre-run of Sec. 4).
__device__ __forceinline__ double inflow_mean(const Params& P, long long t)
{
    double v = P.u0 * (1.0 + P.amp * sin(6.283185307179586 * (double)t / P.period));
    if (P.ramp > 0.0 && (double)t < P.ramp) v *= (double)t / P.ramp;
    return v;
}

// Zou-He velocity inlet (Sec. 4) in non-equilibrium bounce-back form, in
// deviation variables (phi = 1 on inlet cells).  With ub = u_in - g/2 and the
// inward normal n: rho = (sum_{c.n=0} f + 2 sum_{c.n<0} f) / (1 - ub.n);
// unknown f_i (c_i.n > 0) = f_opp + f_i^eq - f_opp^eq; then the tangential
// residual N_t = sum_{c.n=0} (f - f^eq) c_t is removed so sum f c = rho ub.
template <int Q>
__device__ __forceinline__ void zou_he(const Params& P, float prof, float* g)
{
    using L = Lattice<Q>;
    const int ax = P.in_axis;
    const int sgn = P.in_side == 0 ? 1 : -1;
    float un = (float)((double)prof * inflow_mean(P, P.t));
    float ub[3] = {-0.5f * P.gx, -0.5f * P.gy, -0.5f * P.gz};
    ub[ax] += sgn * un;
    float ubn = ub[ax] * sgn;
    float g0 = 0.0f, gm = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int cn = c_axis<Q>(i, ax) * sgn;
        if (cn == 0) g0 += g[i];
        if (cn < 0) gm += g[i];
    }
    float drho = (g0 + 2.0f * gm + ubn) / (1.0f - ubn);
    float rho = 1.0f + drho;
    float uu = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (c_axis<Q>(i, ax) * sgn > 0) {
            float cu = L::cx(i) * ub[0] + L::cy(i) * ub[1] + L::cz(i) * ub[2];
            g[i] = g[opp(i)] + 6.0f * L::w(i) * rho * cu;
        }
    }
#pragma unroll
    for (int tg = 0; tg < 3; ++tg) {
        if (tg == ax) continue;
        float nres = 0.0f, ncnt = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int cn = c_axis<Q>(i, ax) * sgn;
            int ct = c_axis<Q>(i, tg);
            if (cn == 0 && ct != 0) {
                float cu = L::cx(i) * ub[0] + L::cy(i) * ub[1] + L::cz(i) * ub[2];
                float geq = L::w(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
                nres += (g[i] - geq) * ct;
            }
            if (cn > 0) ncnt += ct * ct;
        }
        float corr = nres / ncnt;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (c_axis<Q>(i, ax) * sgn > 0) g[i] -= c_axis<Q>(i, tg) * corr;
    }
}

// Extrapolation outlet (Sec. 4) with prescribed density: unknown populations
// f_i = f_i^eq(rho_out, u_nb) + f_i(nb) - f_i^eq(rho_nb, u_nb), nb = y + n the
// first interior neighbour along the inward normal n, pulled afresh.
template <int Q, class T>
__device__ __forceinline__ void outlet(const Params& P, const Coords& c, float phi, uint32_t nbmask, float* g)
{
    using L = Lattice<Q>;
    const int ax = P.out_axis;
    const int sgn = P.out_side == 1 ? -1 : 1;
    int nx = c.x + (ax == 0 ? sgn : 0);
    int ny = c.y + (ax == 1 ? sgn : 0);
    int nz = c.z + (ax == 2 ? sgn : 0);
    Coords nc = make_coords(P, nx, ny, nz);
    float phin = P.phi[nc.idx];
    float gn[Q];
    pull<Q, T>(static_cast<const T*>(P.fsrc), P.N, nc, nbmask, gn);
    float sd = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        sd += gn[i];
        mx += L::cx(i) * gn[i];
        my += L::cy(i) * gn[i];
        mz += L::cz(i) * gn[i];
    }
    Macro M = macroscopic(P, phin, sd, mx, my, mz);
    float uu = M.ux * M.ux + M.uy * M.uy + M.uz * M.uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (c_axis<Q>(i, ax) * sgn > 0) {
            float cu = L::cx(i) * M.ux + L::cy(i) * M.uy + L::cz(i) * M.uz;
            float pe = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
            // (f^eq(rho_out) - w phi) + (g_nb + w phi_nb) - f^eq(rho_nb)
            float w = L::w(i);
            g[i] = w * phi * (P.rho_out - 1.0f + P.rho_out * pe) + gn[i] - w * phin * (M.drho + M.rho * pe);
        }
    }
}

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ void block_reduce_diag(double* v, double* partials)
{
    __shared__ double sm[kBlock / 32][kDiagSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
        v[5] = fmax(v[5], __shfl_xor_sync(0xffffffffu, v[5], off));
        v[6] = fmin(v[6], __shfl_xor_sync(0xffffffffu, v[6], off));
        v[7] = fmax(v[7], __shfl_xor_sync(0xffffffffu, v[7], off));
        v[8] += __shfl_xor_sync(0xffffffffu, v[8], off);
    }
    if (lane == 0)
        for (int k = 0; k < kDiagSlots; ++k) sm[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[kDiagSlots];
        for (int k = 0; k < kDiagSlots; ++k) r[k] = sm[0][k];
        for (int w = 1; w < kBlock / 32; ++w) {
            for (int k = 0; k < 5; ++k) r[k] += sm[w][k];
            r[5] = fmax(r[5], sm[w][5]);
            r[6] = fmin(r[6], sm[w][6]);
            r[7] = fmax(r[7], sm[w][7]);
            r[8] += sm[w][8];
        }
        for (int k = 0; k < kDiagSlots; ++k) partials[(size_t)blockIdx.x * kDiagSlots + k] = r[k];
    }
}

// ------------------------------------------------------------------ the kernel

// MODE kModeStep: full time step (pull, boundaries, moments, relaxation rate,
// collision, store).  kModeMoments: pull + boundaries + moments and fields of
// the current time.  kModeDiag: the same fields reduced to diagnostics.
template <int Q, class T, int MODE>
__global__ void __launch_bounds__(kBlock) lbm_kernel(const Params P)
{
    using L = Lattice<Q>;
    const int p = blockIdx.x * kBlock + threadIdx.x;
    double dv[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1e300, 0.0, 0.0};
    // dv: 0 sum phi, 1 sum (phi rho - phi), 2 kinetic energy, 3 region sum |u|,
    //     4 region count, 5 max |u|, 6 min omega, 7 max omega, 8 non-finite count
    if (MODE == kModeDiag) dv[7] = -1e300;
    if (p < P.n_cells) {
        const uint32_t pc = P.cells[p];
        const uint32_t mask = P.mask[p];
        const Coords c = make_coords(P, pc & 1023u, (pc >> 10) & 1023u, pc >> 20);
        const float phi = P.phi[c.idx];
        float g[Q];
        pull<Q, T>(static_cast<const T*>(P.fsrc), P.N, c, mask, g);
        const int type = (mask >> kTypeShift) & 3u;
        if (type == kInlet) {
            zou_he<Q>(P, P.bnd_prof[p - P.n_bulk], g);
        } else if (type == kOutlet) {
            outlet<Q, T>(P, c, phi, P.bnd_nbmask[p - P.n_bulk], g);
        }
        // moments: sum g, sum g c, sum g c c
        float sd = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
        float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const float v = g[i];
            sd += v;
            if (cx) mx += cx * v;
            if (cy) my += cy * v;
            if (cz) mz += cz * v;
            if (cx) sxx += v;
            if (cy) syy += v;
            if (cz) szz += v;
            if (cx * cy) sxy += (cx * cy) * v;
            if (cx * cz) sxz += (cx * cz) * v;
            if (cy * cz) syz += (cy * cz) * v;
        }
        const Macro M = macroscopic(P, phi, sd, mx, my, mz);
        // corrected second moment Pi (Sec. 3), via sum f^eq c c = phi rho (c_s^2 I + u u)
        const float cs2 = 1.0f / 3.0f;
        const float pxx = sxx - M.sd * cs2 - M.sigma * M.ux * M.ux + M.Fx * M.ux;
        const float pyy = syy - M.sd * cs2 - M.sigma * M.uy * M.uy + M.Fy * M.uy;
        const float pzz = szz - M.sd * cs2 - M.sigma * M.uz * M.uz + M.Fz * M.uz;
        const float pxy = sxy - M.sigma * M.ux * M.uy + 0.5f * (M.Fx * M.uy + M.ux * M.Fy);
        const float pxz = sxz - M.sigma * M.ux * M.uz + 0.5f * (M.Fx * M.uz + M.ux * M.Fz);
        const float pyz = syz - M.sigma * M.uy * M.uz + 0.5f * (M.Fy * M.uz + M.uy * M.Fz);
        const float pn = sqrtf(pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz));
        // semi-explicit shear rate gdot(t) = omega(t-1) ||Pi||_F / (c_s^2 rho)
        const float om_prev = P.omega[p];
        const float gdot = 3.0f * om_prev * pn / M.rho;
        const float om = relaxation_rate(P, M.rho, gdot);

        if (MODE == kModeStep) {
            T* __restrict__ fd = static_cast<T*>(P.fdst);
            const bool porous = (mask & kPorousBit) != 0u;
            const float uu = M.ux * M.ux + M.uy * M.uy + M.uz * M.uz;
            const float uF = M.ux * M.Fx + M.uy * M.Fy + M.uz * M.Fz;
            const float h = 1.0f - 0.5f * om;
            const float one_m_om = 1.0f - om;
            // rest direction
            {
                const float w = L::w(0);
                const float geq = w * (M.sd - 1.5f * M.sigma * uu);
                const float gf = w * h * (-3.0f * uF);
                Store<T>::st(fd + c.idx, one_m_om * g[0] + om * geq + gf);
            }
#pragma unroll
            for (int i = 1; i < Q; i += 2) {
                const int j = i + 1;
                const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
                const float w = L::w(i);
                const float cu = cx * M.ux + cy * M.uy + cz * M.uz;
                const float cF = cx * M.Fx + cy * M.Fy + cz * M.Fz;
                // f^eq - w phi split into even and odd parts in c
                const float ev = w * (M.sd + M.sigma * (4.5f * cu * cu - 1.5f * uu));
                const float od = 3.0f * w * M.sigma * cu;
                // Guo forcing w (1 - omega/2)((c - u)/c_s^2 + (c.u) c / c_s^4) . F
                const float fe = w * h * (9.0f * cu * cF - 3.0f * uF);
                const float fo = 3.0f * w * h * cF;
                float pi = 0.0f, pj = 0.0f;
                if (porous) {
                    // Omega^phi_i = w rho (phi(y + c_i) - phi(y)) in deviation form
                    // (the stored reference moves to phi(y + c_i)): w (rho - 1) dphi.
                    if (!((mask >> j) & 1u)) pi = w * M.drho * (P.phi[shifted(c, cx, cy, cz)] - phi);
                    if (!((mask >> i) & 1u)) pj = w * M.drho * (P.phi[shifted(c, -cx, -cy, -cz)] - phi);
                }
                Store<T>::st(fd + (long long)i * P.N + c.idx, one_m_om * g[i] + om * (ev + od) + fe + fo + pi);
                Store<T>::st(fd + (long long)j * P.N + c.idx, one_m_om * g[j] + om * (ev - od) + fe - fo + pj);
            }
            P.omega[p] = om;
        } else if (MODE == kModeMoments) {
            const long long o = P.o_compact ? (long long)p : c.idx;
            if (P.o_rho) P.o_rho[o] = M.rho;
            if (P.o_ux) P.o_ux[o] = M.ux;
            if (P.o_uy) P.o_uy[o] = M.uy;
            if (P.o_uz) P.o_uz[o] = M.uz;
            if (P.o_gdot) P.o_gdot[o] = gdot;
            if (P.o_omega) P.o_omega[o] = om;
        } else {
            const float un = sqrtf(M.ux * M.ux + M.uy * M.uy + M.uz * M.uz);
            if (!isfinite(M.rho) || !isfinite(un) || !isfinite(om)) {
                dv[8] = 1.0;
            } else {
                dv[0] = phi;
                dv[1] = M.sd;
                dv[2] = 0.5 * (double)M.rho * (double)un * (double)un;
                if (P.region && P.region[c.idx]) {
                    dv[3] = un;
                    dv[4] = 1.0;
                }
                dv[5] = un;
                dv[6] = om;
                dv[7] = om;
            }
        }
    }
    if (MODE == kModeDiag) block_reduce_diag(dv, P.partials);
}

// Final deterministic reduction of the per-block diagnostics (one block).
__global__ void diag_finish(const double* __restrict__ partials, int nblk, double* __restrict__ out);

}  // namespace lbm
