// Fused pull-scheme collide-and-stream kernel for the VANSE lattice Boltzmann
// method with Carreau-Yasuda rheology (Horvat et al., arXiv 2402.10809,
// Sec. 2-4), plus the moments and diagnostics epilogues that reuse its pull.
//
// Row-packed layout.  Each x-row (y, z) of the box stores only the span
// [xmin, xmax] of its non-solid cells, and the spans of all rows are packed
// back to back: the slot of (x, y, z) is rowbase[y + ny z] + x.  One thread
// owns one slot, so no thread idles on the solid voxels of a sparse aneurysm
// box, and the few solid cells inside a span (gaps between vessel and sac) are
// ghost slots.  A warp of consecutive slots reads and writes consecutive
// addresses of each direction plane, also across the ends of rows, because
// the source of every pull lies in a packed span too.  The distributions live
// in two SoA buffers f[i][n_store].  Cells off periodic faces and off the
// open boundaries take the lean path (source slots from one per-row record of
// the nine neighbour-row bases); the others call the general path.
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

// Per-slot mask word: bit i (i < Q) set when direction i cannot be pulled from
// its source y - c_i (solid, box wall, or an open face); bits 27-28 cell type;
// bit 29 set when some fluid neighbour has a different porosity; bit 30 set
// when the cell lies on a periodic face; bit 31 marks a ghost slot (a solid
// cell inside a packed span, or any slot of a halo plane of a z-slab, whose
// state the neighbouring slab provides), whose bit 0 asks for zero stores (it
// shares an aligned 8-slot group with a fluid slot).
constexpr uint32_t kTypeShift = 27;
constexpr uint32_t kPorousBit = 1u << 29;
constexpr uint32_t kWrapBit = 1u << 30;
constexpr uint32_t kGhostBit = 1u << 31;
constexpr uint32_t kGeneralBits = (3u << kTypeShift) | kWrapBit;
enum { kBulk = 0, kInlet = 1, kOutlet = 2 };
enum { kModeStep = 0, kModeMoments = 1, kModeDiag = 2 };
// Threads per block of the slot-parallel kernels, and the resident blocks per
// SM the step kernel is compiled for (which sets its register cap: 80 for six
// blocks of 128, 24 warps per SM).  Measured at 384^3 against three blocks of
// 256 at the same register cap: 2.4 % faster with FP32 storage, 4.4 % with
// FP16 (finer retirement of blocks: a block slot frees when its 4 warps end).
#ifndef LBM_BLOCK
#define LBM_BLOCK 128
#endif
#ifndef LBM_MIN_BLOCKS
#define LBM_MIN_BLOCKS 6
#endif
constexpr int kBlock = LBM_BLOCK;
constexpr int kDiagSlots = 9;

struct Params {
    // geometry
    int nx, ny, nz;
    long long N;              // box cells (dense outputs)
    int n_store;              // slots of the packed layout
    int wide;                 // Q n_store >= 2^32: every cell takes the general path (64-bit offsets)
    int n_general;            // cells of the general path (periodic faces, inlet, outlet; all when wide)
    int gen_block;            // general cells per block (32 or kBlock)
    const uint32_t* general;  // [n_general] their slots, ascending
    const uint32_t* rows;     // [n_store] row y + ny z of each slot
    const int4* rownb;        // [ny nz][3] per row: bases of the neighbour rows (y + sy, z + sz)
                              // (wrapped on periodic axes) at index (sy + 1) + 3 (sz + 1),
                              // then y, z, 0, 0
    const int* rowbase;       // [ny nz] slot of (x, row) = rowbase[row] + x
    const uint32_t* mask;     // [n_store]
    const float* phi;         // [n_store] porosity
    const float* bnd_prof;    // [n_store] inlet cells: profile 2 max(0, 1 - r^2/R^2)
    const uint32_t* bnd_nbmask;  // [n_store] outlet cells: mask of the interior neighbour
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
    float* omega;             // [n_store] omega(t-1) in, omega(t) out
    long long t;
    // moments outputs (dense or slot order, any may be null)
    float *o_rho, *o_ux, *o_uy, *o_uz, *o_gdot, *o_omega;
    int o_compact;
    float* o_drho;            // time step: rho - 1 of time t per slot (may be null)
    // anisotropic permeability (kernels instantiated with AN = true): per slot
    // [12][n_store] Ah xx yy zz xy xz yz, then B in the same order
    const float* aniso;
    int aniso_iters;
    float aniso_tol;
    // L2 residency of the step: [l2_base, l2_base + l2_bytes) (the row records
    // and the per-slot words) is kept in the persisting part of L2 with hit
    // ratio l2_hit; l2_bytes = 0 launches without a window
    const void* l2_base;
    size_t l2_bytes;
    float l2_hit;
    // diagnostics
    const uint8_t* region;    // dense, may be null
    double* partials;         // [gridDim.x][kDiagSlots]
};

// Blocks of a launch: first the general-path cells, gen_block per block, then
// one thread per slot for the lean path, which skips ghost and general slots.
// Leading the grid lets the slower general blocks overlap the bulk.  Their
// cells lie in different rows, so their loads do not coalesce: on small grids
// the host asks for one warp's worth per block (gen_block = 32) to spread them
// over many SMs; on large grids full blocks keep the block slots for the bulk.
__host__ __device__ inline int general_blocks(const Params& P)
{
    return (P.n_general + P.gen_block - 1) / P.gen_block;
}
__host__ __device__ inline int total_blocks(const Params& P)
{
    return general_blocks(P) + (P.n_store + kBlock - 1) / kBlock;
}

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

// 4-byte global -> shared copy that stays in flight without occupying a
// register (LDGSTS, sm_80 and later); cp_async_wait_all commits the thread's
// copies and waits for them.
__device__ __forceinline__ void cp_async4(volatile float* dst, const float* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared((const void*)dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Programmatic dependent launch of the time steps: a step's blocks may start
// while the previous step's last blocks finish.  Before grid_dependency_wait()
// a step reads only data no step writes (mask, row id, porosity, row
// records); the wait returns once the previous step has completed and its
// writes are visible.  Outside a programmatic launch both are no-ops.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Loads issued in program order (inline PTX, so that the compiler neither
// sinks them to their first use nor places them behind a branch): a lean
// cell requests all its per-slot words before its first dependent load, so
// it waits for one memory latency before the row record instead of one per
// word.
__device__ __forceinline__ uint32_t ld_early_u32(const uint32_t* a)
{
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(a));
    return v;
}
__device__ __forceinline__ float ld_early_nc(const float* a)
{
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(a));
    return v;
}
__device__ __forceinline__ float ld_early(const float* a)
{
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(a));
    return v;
}

// c . v for a lattice vector c with components in {-1, 0, 1}: only the needed
// additions and sign flips (after unrolling every branch is decided at compile
// time; IEEE arithmetic would not let the compiler drop 0 * v or v + 0).
__device__ __forceinline__ float cdot(int cx, int cy, int cz, float x, float y, float z)
{
    float r = 0.0f;
    bool has = false;
    if (cx != 0) { r = cx > 0 ? x : -x; has = true; }
    if (cy != 0) { r = has ? (cy > 0 ? r + y : r - y) : (cy > 0 ? y : -y); has = true; }
    if (cz != 0) { r = has ? (cz > 0 ? r + z : r - z) : (cz > 0 ? z : -z); has = true; }
    return r;
}

// ------------------------------------------------------------------ physics

// Darcy and Forchheimer coefficients K1 = phi^2 nu / k, K2 = phi^3 C_F / sqrt(k)
// of f(u) = -(K1 + K2 |u|) u (Sec. 2).  Kozeny-Carman k = phi^3 d^2 / (150 (1-phi)^2)
// with Ergun C_F = 1.75 / sqrt(150 phi^3) reduce to K1 = (150 nu / d^2)(1-phi)^2 / phi
// and K2 = (1.75 / d)(1 - phi): drag_a = 150 nu / d^2, drag_b = 1.75 / d.  For a
// constant permeability kc: K1 = (nu / kc) phi^2, K2 = (1.75 / sqrt(150 kc)) phi^1.5,
// only where phi < 1.
__device__ __forceinline__ void darcy_coeffs(const Params& P, float phi, float iphi, float& k1, float& k2)
{
    if (P.drag_kc) {
        float s = 1.0f - phi;
        k1 = P.drag_a * s * s * iphi;
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
    const float iphi = __frcp_rn(phi);
    M.rho = M.sigma * iphi;
    M.drho = sd * iphi;
    const float isig = __fdividef(1.0f, M.sigma);
    const float hg = 0.5f * iphi;
    const float vx = fmaf(P.gx, hg, mx * isig);
    const float vy = fmaf(P.gy, hg, my * isig);
    const float vz = fmaf(P.gz, hg, mz * isig);
    float k1, k2;
    darcy_coeffs(P, phi, iphi, k1, k2);
    const float alpha = 0.25f * k1 * iphi;
    const float c1 = 0.5f * k2 * iphi;
    const float c1v = c1 * sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
    const float c0 = 0.5f + alpha;
    const float r = sqrtf(fmaf(c0, c0, c1v));
    const float dm1 = alpha + __fdividef(fmaf(alpha, alpha, alpha + c1v), r + 0.5f);
    const float id = __fdividef(1.0f, 1.0f + dm1);
    M.ux = vx * id;
    M.uy = vy * id;
    M.uz = vz * id;
    const float s2 = 2.0f * M.sigma * dm1;
    M.Fx = fmaf(M.rho, P.gx, -s2 * M.ux);
    M.Fy = fmaf(M.rho, P.gy, -s2 * M.uy);
    M.Fz = fmaf(M.rho, P.gz, -s2 * M.uz);
    return M;
}

// Anisotropic permeability (Sec. 3 remark).  With K = k(phi) S^{-1} (the
// isotropic closure k(phi) and a per-cell shape tensor S) the drag
// f(u) = -phi^2 nu K^{-1} u - phi^3 C_F |u| K^{-1/2} u turns the velocity
// equation into (Id + Ah + |u| B) u = v, Ah = (phi nu / 2) K^{-1},
// B = (phi^2 C_F / 2) K^{-1/2}, both precomputed per slot.  Fixed-point
// iteration u_{m+1} = (Id + Ah + |u_m| B)^{-1} v from u_0 = v, each step one
// 3x3 solve by the adjugate, until |u_{m+1} - u_m| <= tol |v| or aniso_iters
// steps; then F = rho g - 2 phi rho (Ah u + |u| B u).  Cells with phi = 1 have
// no medium and take the explicit solution.
__device__ __forceinline__ Macro macroscopic_aniso(const Params& P, int p, float phi, float sd, float mx, float my,
                                                   float mz)
{
    if (!(phi < 1.0f)) return macroscopic(P, phi, sd, mx, my, mz);
    Macro M;
    M.sd = sd;
    M.sigma = phi + sd;
    const float iphi = __frcp_rn(phi);
    M.rho = M.sigma * iphi;
    M.drho = sd * iphi;
    const float isig = __fdividef(1.0f, M.sigma);
    const float hg = 0.5f * iphi;
    const float vx = fmaf(P.gx, hg, mx * isig);
    const float vy = fmaf(P.gy, hg, my * isig);
    const float vz = fmaf(P.gz, hg, mz * isig);
    const size_t n = (size_t)P.n_store;
    const float* a = P.aniso + p;
    const float axx = __ldg(a), ayy = __ldg(a + n), azz = __ldg(a + 2 * n);
    const float axy = __ldg(a + 3 * n), axz = __ldg(a + 4 * n), ayz = __ldg(a + 5 * n);
    const float bxx = __ldg(a + 6 * n), byy = __ldg(a + 7 * n), bzz = __ldg(a + 8 * n);
    const float bxy = __ldg(a + 9 * n), bxz = __ldg(a + 10 * n), byz = __ldg(a + 11 * n);
    const float tol = P.aniso_tol * sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
    float ux = vx, uy = vy, uz = vz, un = sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
    for (int m = 0; m < P.aniso_iters; ++m) {
        const float xx = 1.0f + fmaf(un, bxx, axx), yy = 1.0f + fmaf(un, byy, ayy), zz = 1.0f + fmaf(un, bzz, azz);
        const float xy = fmaf(un, bxy, axy), xz = fmaf(un, bxz, axz), yz = fmaf(un, byz, ayz);
        const float c00 = fmaf(yy, zz, -yz * yz), c01 = fmaf(xz, yz, -xy * zz), c02 = fmaf(xy, yz, -yy * xz);
        const float c11 = fmaf(xx, zz, -xz * xz), c12 = fmaf(xy, xz, -xx * yz), c22 = fmaf(xx, yy, -xy * xy);
        const float idet = __frcp_rn(fmaf(xx, c00, fmaf(xy, c01, xz * c02)));
        const float nx = fmaf(c00, vx, fmaf(c01, vy, c02 * vz)) * idet;
        const float ny = fmaf(c01, vx, fmaf(c11, vy, c12 * vz)) * idet;
        const float nz = fmaf(c02, vx, fmaf(c12, vy, c22 * vz)) * idet;
        const float dx = nx - ux, dy = ny - uy, dz = nz - uz;
        ux = nx;
        uy = ny;
        uz = nz;
        un = sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
        if (sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) <= tol) break;
    }
    M.ux = ux;
    M.uy = uy;
    M.uz = uz;
    // drag per unit phi rho, halved: Ah u + |u| B u
    const float dxv = fmaf(axx, ux, fmaf(axy, uy, axz * uz)) + un * fmaf(bxx, ux, fmaf(bxy, uy, bxz * uz));
    const float dyv = fmaf(axy, ux, fmaf(ayy, uy, ayz * uz)) + un * fmaf(bxy, ux, fmaf(byy, uy, byz * uz));
    const float dzv = fmaf(axz, ux, fmaf(ayz, uy, azz * uz)) + un * fmaf(bxz, ux, fmaf(byz, uy, bzz * uz));
    const float s2 = 2.0f * M.sigma;
    M.Fx = fmaf(M.rho, P.gx, -s2 * dxv);
    M.Fy = fmaf(M.rho, P.gy, -s2 * dyv);
    M.Fz = fmaf(M.rho, P.gz, -s2 * dzv);
    return M;
}

// Carreau-Yasuda law, Eq. (3), and omega = 2 rho c_s^2 / (2 mu + rho c_s^2).
__device__ __forceinline__ float relaxation_rate(const Params& P, float rho, float gdot)
{
    const float x = P.lam * gdot;
    const float xa = P.cy_a_two ? x * x : __powf(x, P.cy_a);
    const float mu = fmaf(P.mu0 - P.mu_inf, exp2f(P.cy_e * __log2f(1.0f + xa)), P.mu_inf);
    return __fdividef(2.0f * rho, fmaf(6.0f, mu, rho));
}

// ------------------------------------------------------------------ moments

// sum g, sum g c and sum g c c of the Q deviations, factorised by the rows of
// constant (c_y, c_z) so that every addition is used once.
template <int Q>
struct Moments {
    float sd, mx, my, mz, sxx, syy, szz, sxy, sxz, syz;
};

// g_i is read from g[i * S] (S = 1: a register array; S = block size: the
// shared-memory column of one thread).
template <int Q, int S = 1>
__device__ __forceinline__ Moments<Q> moments(const float* g)
{
    float rs[9], rx[9], rxx[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int cy = r % 3 - 1, cz = r / 3 - 1;
        const int ip = find_dir<Q>(1, cy, cz), im = find_dir<Q>(-1, cy, cz), i0 = find_dir<Q>(0, cy, cz);
        if (ip >= 0) {
            rxx[r] = g[ip * S] + g[im * S];
            rx[r] = g[ip * S] - g[im * S];
            rs[r] = rxx[r] + g[i0 * S];
        } else {
            rxx[r] = 0.0f;
            rx[r] = 0.0f;
            rs[r] = g[i0 * S];
        }
    }
    Moments<Q> m;
    // rows: r = (cy + 1) + 3 (cz + 1)
    const float ym = rs[0] + rs[3] + rs[6];  // c_y = -1
    const float yp = rs[2] + rs[5] + rs[8];  // c_y = +1
    const float zm = rs[0] + rs[1] + rs[2];  // c_z = -1
    const float zp = rs[6] + rs[7] + rs[8];  // c_z = +1
    m.sd = (ym + yp) + (rs[1] + rs[4] + rs[7]);
    m.my = yp - ym;
    m.syy = yp + ym;
    m.mz = zp - zm;
    m.szz = zp + zm;
    m.mx = ((rx[0] + rx[1]) + (rx[2] + rx[3])) + ((rx[4] + rx[5]) + (rx[6] + rx[7]) + rx[8]);
    m.sxx = ((rxx[0] + rxx[1]) + (rxx[2] + rxx[3])) + ((rxx[4] + rxx[5]) + (rxx[6] + rxx[7]) + rxx[8]);
    m.sxy = (rx[2] + rx[5] + rx[8]) - (rx[0] + rx[3] + rx[6]);
    m.sxz = (rx[6] + rx[7] + rx[8]) - (rx[0] + rx[1] + rx[2]);
    m.syz = (rs[0] + rs[8]) - (rs[2] + rs[6]);
    return m;
}

// ------------------------------------------------------------------ helpers

// Bases of the nine neighbour rows of a cell, index (sy + 1) + 3 (sz + 1) for the
// row (y + sy, z + sz), wrapped on periodic axes.
struct RowBases {
    int b[9];
};

__device__ __forceinline__ RowBases row_bases(const Params& P, uint32_t r)
{
    const int4* rn = P.rownb + 3 * (size_t)r;
    const int4 a = __ldg(rn), c = __ldg(rn + 1), d = __ldg(rn + 2);
    RowBases R;
    R.b[0] = a.x; R.b[1] = a.y; R.b[2] = a.z; R.b[3] = a.w;
    R.b[4] = c.x; R.b[5] = c.y; R.b[6] = c.z; R.b[7] = c.w;
    R.b[8] = d.x;
    return R;
}

// A cell of the general path: its coordinates, slot and dense index, the
// wrapped neighbour x and the bases of its neighbour rows.
struct Coords {
    int x, y, z;
    long long slot;  // packed slot
    long long idx;   // dense index x + nx (y + ny z)
    int X[3];        // x - 1, x, x + 1 (wrapped)
    RowBases rb;
};

__device__ __forceinline__ Coords make_coords(const Params& P, int x, int y, int z)
{
    Coords c;
    c.x = x; c.y = y; c.z = z;
    c.idx = x + (long long)P.nx * (y + (long long)P.ny * z);
    c.rb = row_bases(P, (uint32_t)(y + P.ny * z));
    c.slot = (long long)c.rb.b[4] + x;
    c.X[0] = x == 0 ? P.nx - 1 : x - 1;
    c.X[1] = x;
    c.X[2] = x == P.nx - 1 ? 0 : x + 1;
    return c;
}

// Coordinates of slot p (row from the slot's row id, x from the row base).
__device__ __forceinline__ Coords coords_of(const Params& P, int p)
{
    const uint32_t r = P.rows[p];
    Coords c;
    c.rb = row_bases(P, r);
    const int4 yz = __ldg(P.rownb + 3 * (size_t)r + 2);
    c.y = yz.y;
    c.z = yz.z;
    c.x = p - c.rb.b[4];
    c.slot = p;
    c.idx = c.x + (long long)P.nx * r;
    c.X[0] = c.x == 0 ? P.nx - 1 : c.x - 1;
    c.X[1] = c.x;
    c.X[2] = c.x == P.nx - 1 ? 0 : c.x + 1;
    return c;
}

// Slot of y + (dx, dy, dz) with periodic wrap (dx etc. in {-1, 0, 1}); only
// meaningful where that cell is non-solid.
__device__ __forceinline__ long long shifted(const Params& P, const Coords& c, int dx, int dy, int dz)
{
    return (long long)c.rb.b[(dy + 1) + 3 * (dz + 1)] + c.X[dx + 1];
}

// Source (plane, slot) of direction i: g_i = f*_i(y - c_i), or the cell's own
// f*_opp(i) (half-way bounce-back, Sec. 4) where the source is not available.
template <int Q>
__device__ __forceinline__ long long pull_offset(const Params& P, const Coords& c, uint32_t mask, int i)
{
    using L = Lattice<Q>;
    const long long n = P.n_store;
    return ((mask >> i) & 1u) ? (long long)opp(i) * n + c.slot
                              : (long long)i * n + shifted(P, c, -L::cx(i), -L::cy(i), -L::cz(i));
}

template <int Q, class T>
__device__ __forceinline__ void pull_general(const Params& P, const T* __restrict__ f, const Coords& c,
                                             uint32_t mask, float* g)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Store<T>::ld(f + pull_offset<Q>(P, c, mask, i));
}

// Lean-path slot of (x + dx, y + dy, z + dz) in 32-bit arithmetic.
__device__ __forceinline__ uint32_t lean_slot(const RowBases& R, int x, int dx, int dy, int dz)
{
    return (uint32_t)(R.b[(dy + 1) + 3 * (dz + 1)] + x + dx);
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
// unknown f_i (c_i.n > 0) = f_opp + f_i^eq - f_opp^eq, so that sum f = rho and
// sum f c.n = rho ub.n.  No tangential correction: in D3Q27 it makes the
// inlet unstable at the low relaxation times of the Carreau-Yasuda law.
template <int Q>
__device__ __forceinline__ void zou_he(const Params& P, float prof, float* g)
{
    using L = Lattice<Q>;
    const int ax = P.in_axis;
    const int sgn = P.in_side == 0 ? 1 : -1;
    const float un = (float)((double)prof * inflow_mean(P, P.t));
    const float ubx = -0.5f * P.gx + (ax == 0 ? sgn * un : 0.0f);
    const float uby = -0.5f * P.gy + (ax == 1 ? sgn * un : 0.0f);
    const float ubz = -0.5f * P.gz + (ax == 2 ? sgn * un : 0.0f);
    const float ubn = (ax == 0 ? ubx : ax == 1 ? uby : ubz) * sgn;
    float g0 = 0.0f, gm = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cn = c_axis<Q>(i, ax) * sgn;
        if (cn == 0) g0 += g[i];
        if (cn < 0) gm += g[i];
    }
    const float drho = (g0 + 2.0f * gm + ubn) / (1.0f - ubn);
    const float rho = 1.0f + drho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (c_axis<Q>(i, ax) * sgn > 0) {
            const float cu = cdot(L::cx(i), L::cy(i), L::cz(i), ubx, uby, ubz);
            g[i] = g[opp(i)] + 6.0f * L::w(i) * rho * cu;
        }
    }
}

// Extrapolation outlet (Sec. 4) with prescribed density: unknown populations
// f_i = f_i^eq(rho_out, u_nb) + f_i(nb) - f_i^eq(rho_nb, u_nb), nb = y + n the
// first interior neighbour along the inward normal n, pulled afresh.  Two
// passes over the neighbour's populations keep the register footprint small.
template <int Q, class T>
__device__ __forceinline__ void outlet(const Params& P, const Coords& c, float phi, uint32_t nbmask, float* g)
{
    using L = Lattice<Q>;
    const int ax = P.out_axis;
    const int sgn = P.out_side == 1 ? -1 : 1;
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
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (c_axis<Q>(i, ax) * sgn > 0) {
            const float gn = Store<T>::ld(f + pull_offset<Q>(P, nc, nbmask, i));
            const float cu = cdot(L::cx(i), L::cy(i), L::cz(i), M.ux, M.uy, M.uz);
            const float pe = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
            // (f^eq(rho_out) - w phi) + (g_nb + w phi_nb) - f^eq(rho_nb)
            const float w = L::w(i);
            g[i] = w * phi * (P.rho_out - 1.0f + P.rho_out * pe) + gn - w * phin * (M.drho + M.rho * pe);
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

// One cell of the fused step / moments / diagnostics: slot p with its link
// mask, lean or general path; diagnostics accumulate into dv.
// MODE kModeStep: full time step (pull, boundaries, moments, relaxation rate,
// collision, store).  kModeMoments: pull + boundaries + moments and fields of
// the current time.  kModeDiag: the same fields reduced to diagnostics.
// park: this thread's column of a Q x kBlock shared array (time step only).
// Lean cells (fast) get their row id, porosity and omega(t-1) from the caller,
// which loads them together with the mask; general cells load their own.
template <int Q, class T, int MODE, bool fast, bool AN>
__device__ __forceinline__ void cell_impl(const Params& P, int p, uint32_t mask, double* dv, volatile float* park,
                                          uint32_t row_pre = 0, float phi_pre = 0.0f, float om_pre = 0.0f)
{
    using L = Lattice<Q>;
    const float phi = fast ? phi_pre : __ldg(P.phi + p);
    const T* __restrict__ fs = static_cast<const T*>(P.fsrc);
    const uint32_t n = (uint32_t)P.n_store;
    float g[Q];
    Coords cg;     // general path: wrapped neighbour coordinates of this cell
    RowBases rb;   // lean path: bases of the nine neighbour rows
    int x = 0;
    uint32_t row = 0;
    if (fast) {
        // y - c_i never wraps here and every offset fits 32 bits (the host
        // sends larger layouts down the general path).
        row = row_pre;
        rb = row_bases(P, row);
        x = p - rb.b[4];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t o = ((mask >> i) & 1u) ? (uint32_t)opp(i) * n + (uint32_t)p
                                                  : (uint32_t)i * n + lean_slot(rb, x, -L::cx(i), -L::cy(i), -L::cz(i));
            g[i] = Store<T>::ld(fs + o);
        }
    } else {
        cg = coords_of(P, p);
        pull_general<Q, T>(P, fs, cg, mask, g);
        const int type = (mask >> kTypeShift) & 3u;
        if (type == kInlet) {
            zou_he<Q>(P, P.bnd_prof[p], g);
        } else if (type == kOutlet) {
            outlet<Q, T>(P, cg, phi, P.bnd_nbmask[p], g);
        }
    }
    // The time step parks the pulled populations in this thread's column of
    // shared memory: the moments below consume the register copies, and the
    // collision re-reads them from shared memory, so the Q values need not stay
    // in registers through the macroscopic, shear-rate and viscosity phase.
    if (MODE == kModeStep) {
#pragma unroll
        for (int i = 0; i < Q; ++i) park[i * kBlock] = g[i];
    }
    const Moments<Q> m = moments<Q>(g);
    Macro M;
    if constexpr (AN)
        M = macroscopic_aniso(P, p, phi, m.sd, m.mx, m.my, m.mz);
    else
        M = macroscopic(P, phi, m.sd, m.mx, m.my, m.mz);
    // corrected second moment Pi (Sec. 3), via sum f^eq c c = phi rho (c_s^2 I + u u)
    const float sd3 = M.sd * (1.0f / 3.0f);
    const float pxx = fmaf(M.ux, fmaf(-M.sigma, M.ux, M.Fx), m.sxx - sd3);
    const float pyy = fmaf(M.uy, fmaf(-M.sigma, M.uy, M.Fy), m.syy - sd3);
    const float pzz = fmaf(M.uz, fmaf(-M.sigma, M.uz, M.Fz), m.szz - sd3);
    const float pxy = fmaf(M.ux, fmaf(-M.sigma, M.uy, 0.5f * M.Fy), fmaf(0.5f * M.Fx, M.uy, m.sxy));
    const float pxz = fmaf(M.ux, fmaf(-M.sigma, M.uz, 0.5f * M.Fz), fmaf(0.5f * M.Fx, M.uz, m.sxz));
    const float pyz = fmaf(M.uy, fmaf(-M.sigma, M.uz, 0.5f * M.Fz), fmaf(0.5f * M.Fy, M.uz, m.syz));
    const float pn2 = fmaf(pxx, pxx, fmaf(pyy, pyy, fmaf(pzz, pzz, 2.0f * fmaf(pxy, pxy, fmaf(pxz, pxz, pyz * pyz)))));
    // semi-explicit shear rate gdot(t) = omega(t-1) ||Pi||_F / (c_s^2 rho)
    const float om_prev = fast ? om_pre : P.omega[p];
    const float gdot = __fdividef(3.0f * om_prev * sqrtf(pn2), M.rho);
    const float om = relaxation_rate(P, M.rho, gdot);

    if (MODE == kModeStep) {
        T* __restrict__ fd = static_cast<T*>(P.fdst);
        const bool porous = (mask & kPorousBit) != 0u;
        const float uu = fmaf(M.ux, M.ux, fmaf(M.uy, M.uy, M.uz * M.uz));
        const float uF = fmaf(M.ux, M.Fx, fmaf(M.uy, M.Fy, M.uz * M.Fz));
        const float h = fmaf(-0.5f, om, 1.0f);
        const float omo = 1.0f - om;
        // Per unit weight: even part omega (f^eq - w phi) + Guo even part,
        // coefficients of (c.u)^2 and (c.u)(c.F), odd coefficients of c.u and c.F.
        const float e0 = fmaf(om, fmaf(-1.5f * M.sigma, uu, M.sd), -3.0f * h * uF);
        const float ek = 4.5f * om * M.sigma;
        const float gk = 9.0f * h;
        const float os = 3.0f * om * M.sigma;
        const float of = 3.0f * h;
        T* __restrict__ dp = fd + p;  // this cell in plane 0; plane i at + i n_store
        {
            const float w = L::w(0);
            Store<T>::st(dp, fmaf(omo, park[0], w * e0));
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const int j = i + 1;
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const float w = L::w(i);
            const float cu = cdot(cx, cy, cz, M.ux, M.uy, M.uz);
            const float cF = cdot(cx, cy, cz, M.Fx, M.Fy, M.Fz);
            // f^eq - w phi = w (sd + sigma (3 cu + 4.5 cu^2 - 1.5 uu)); Guo:
            // w (1 - omega/2)(3 cF - 3 uF + 9 cu cF)
            const float ev = w * fmaf(cu * cu, ek, fmaf(cu * cF, gk, e0));
            const float od = w * fmaf(cu, os, cF * of);
            float vi = fmaf(omo, park[i * kBlock], ev + od);
            float vj = fmaf(omo, park[j * kBlock], ev - od);
            if (porous) {
                // Omega^phi_i = w rho (phi(y + c_i) - phi(y)) in deviation form
                // (the stored reference moves to phi(y + c_i)): w (rho - 1) dphi.
                // A set mask bit means that neighbour is solid or outside: the
                // cell reads its own porosity there, so dphi = 0 without a branch.
                const float wd = w * M.drho;
                uint32_t ni, nj;
                if (fast) {
                    ni = ((mask >> j) & 1u) ? (uint32_t)p : lean_slot(rb, x, cx, cy, cz);
                    nj = ((mask >> i) & 1u) ? (uint32_t)p : lean_slot(rb, x, -cx, -cy, -cz);
                } else {
                    ni = ((mask >> j) & 1u) ? (uint32_t)p : (uint32_t)shifted(P, cg, cx, cy, cz);
                    nj = ((mask >> i) & 1u) ? (uint32_t)p : (uint32_t)shifted(P, cg, -cx, -cy, -cz);
                }
                vi = fmaf(wd, __ldg(P.phi + ni) - phi, vi);
                vj = fmaf(wd, __ldg(P.phi + nj) - phi, vj);
            }
            Store<T>::st(dp + (size_t)i * n, vi);
            Store<T>::st(dp + (size_t)j * n, vj);
        }
        P.omega[p] = om;
        if (P.o_drho) P.o_drho[p] = M.drho;  // density deviation of time t (adjoint replay)
    } else if (MODE == kModeMoments) {
        const long long idx = fast ? (long long)x + (long long)P.nx * row : cg.idx;
        const long long o = P.o_compact ? (long long)p : idx;
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
            const long long idx = fast ? (long long)x + (long long)P.nx * row : cg.idx;
            if (P.region && P.region[idx]) {
                dv[3] = un;
                dv[4] = 1.0;
            }
            dv[5] = un;
            dv[6] = om;
            dv[7] = om;
        }
    }
}

// Cells of the general path (periodic wrap, inlet, outlet) in a function of
// their own, so that their register needs do not bound the lean path.
template <int Q, class T, int MODE, bool AN>
__device__ __noinline__ void cell_general(const Params& P, int p, uint32_t mask, double* dv, volatile float* park)
{
    cell_impl<Q, T, MODE, false, AN>(P, p, mask, dv, park);
}

// A ghost slot: complete its sectors with zeros where it shares an aligned
// 8-slot group with fluid slots (nothing ever reads it).
template <int Q, class T, int MODE>
__device__ __forceinline__ void ghost_slot(const Params& P, int p, uint32_t mask)
{
    if (MODE == kModeStep && (mask & 1u)) {
        T* __restrict__ gd = static_cast<T*>(P.fdst) + p;
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<T>::st(gd + (size_t)i * P.n_store, 0.0f);
    }
}

// Lean-path thread of slot p: ghost slots store zeros where needed, general
// cells are left to the general blocks.
template <int Q, class T, int MODE, bool AN>
__device__ __forceinline__ void lean_body(const Params& P, int p, uint32_t mask, double* dv, volatile float* park,
                                          uint32_t row, float phi, float om)
{
    if (mask & kGhostBit)
        ghost_slot<Q, T, MODE>(P, p, mask);
    else if (!(mask & kGeneralBits) && !P.wide)
        cell_impl<Q, T, MODE, true, AN>(P, p, mask, dv, park, row, phi, om);
}

// Shared column for parking the pulled populations during a time step.
template <int Q, int MODE>
__device__ __forceinline__ volatile float* park_column()
{
    if (MODE != kModeStep) return nullptr;
    __shared__ float sg[Q * kBlock];
    return sg + threadIdx.x;
}

// MODE kModeStep: full time step (pull, boundaries, moments, relaxation rate,
// collision, store).  kModeMoments: pull + boundaries + moments and fields of
// the current time.  kModeDiag: the same fields reduced to diagnostics.  AN:
// the anisotropic velocity solve (macroscopic_aniso) at porous cells.
template <int Q, class T, int MODE, bool AN = false>
__global__ void __launch_bounds__(kBlock, LBM_MIN_BLOCKS) lbm_kernel(const Params P)
{
    const int nbg = general_blocks(P);
    double dv[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
    // dv: 0 sum phi, 1 sum (phi rho - phi), 2 kinetic energy, 3 region sum |u|,
    //     4 region count, 5 max |u|, 6 min omega, 7 max omega, 8 non-finite count
    volatile float* park = park_column<Q, MODE>();
    // the next step may be scheduled once every block of this one has started
    if (MODE == kModeStep) grid_dependents_launch();
    if ((int)blockIdx.x < nbg) {
        if (MODE == kModeStep) grid_dependency_wait();
        const int k = (int)blockIdx.x * P.gen_block + (int)threadIdx.x;
        if ((int)threadIdx.x < P.gen_block && k < P.n_general) {
            const int p = (int)P.general[k];
            cell_general<Q, T, MODE, AN>(P, p, P.mask[p], dv, park);
        }
    } else {
        const int p = ((int)blockIdx.x - nbg) * kBlock + (int)threadIdx.x;
        if (p < P.n_store) {
            // all per-slot words of the cell at once (ghost and general
            // slots load them too, harmlessly: every slot has all four)
            const uint32_t mask = ld_early_u32(P.mask + p);
            const uint32_t row = ld_early_u32(P.rows + p);
            const float phi = ld_early_nc(P.phi + p);
            // omega and the populations are the previous step's outputs, and
            // this step's stores go to the buffer the previous step read
            if (MODE == kModeStep) grid_dependency_wait();
            const float om = ld_early(P.omega + p);
            lean_body<Q, T, MODE, AN>(P, p, mask, dv, park, row, phi, om);
        }
    }
    if (MODE == kModeDiag) block_reduce_diag(dv, P.partials);
}

}  // namespace lbm
