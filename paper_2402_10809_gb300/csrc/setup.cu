// Set-up kernels: the compact cell list, the per-cell link masks and boundary
// data, the initial state, checkpoints and the final diagnostics reduction.
//
// The cell list is built by a deterministic three-pass compaction (count per
// chunk, single-block scan, emit), ordered as bulk fluid cells by dense index,
// then inlet cells, then outlet cells, so that boundary cells fill their own
// warps at the end of the step launch.
#include <stdint.h>

#include "kernels.cuh"
#include "setup.cuh"

namespace lbm {

__device__ __forceinline__ bool on_periodic_face(long long idx, const CellGrid& G)
{
    const long long plane = (long long)G.nx * G.ny;
    const int z = (int)(idx / plane);
    const long long r = idx - (long long)z * plane;
    const int y = (int)(r / G.nx);
    const int x = (int)(r - (long long)y * G.nx);
    return (G.periodic[0] && (x == 0 || x == G.nx - 1)) || (G.periodic[1] && (y == 0 || y == G.ny - 1)) ||
           (G.periodic[2] && (z == 0 || z == G.nz - 1));
}

// List group of a cell: 0 bulk off periodic faces (and ghosts, see setup.cuh),
// 1 bulk on a periodic face, 2 inlet, 3 outlet, -1 not listed.
__device__ __forceinline__ int category(uint8_t f, long long idx, const CellGrid& G, bool group_has_bulk)
{
    if (f == 2) return 2;
    if (f == 3) return 3;
    if (f == 0) return group_has_bulk ? 0 : -1;
    if (f != 1) return -1;
    return on_periodic_face(idx, G) ? 1 : 0;
}

// Whether the ghost group of this thread's cells holds a bulk cell of group 0.
__device__ __forceinline__ bool group_has_bulk(const uint8_t* flags, long long base, long long N, const CellGrid& G)
{
    for (int k = 0; k < kSetupCellsPerThread; ++k) {
        const long long idx = base + k;
        if (idx < N && flags[idx] == 1 && !on_periodic_face(idx, G)) return true;
    }
    return false;
}

// Inclusive scan over a 256-thread block; returns the exclusive prefix and the
// block total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t warp_tot[kSetupThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    uint32_t base = 0, tot = 0;
    for (int w = 0; w < kSetupThreads / 32; ++w) {
        if (w < wid) base += warp_tot[w];
        tot += warp_tot[w];
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

__global__ void setup_count(const uint8_t* __restrict__ flags, long long N, CellGrid G, int nblk,
                            uint32_t* __restrict__ counts)
{
    const long long base = (long long)blockIdx.x * kSetupChunk + (long long)threadIdx.x * kSetupCellsPerThread;
    const bool gb = group_has_bulk(flags, base, N, G);
    uint32_t c[kCounters] = {0, 0, 0, 0, 0};
    for (int k = 0; k < kSetupCellsPerThread; ++k) {
        const long long idx = base + k;
        if (idx < N) {
            const int cat = category(flags[idx], idx, G, gb);
            if (cat >= 0) c[cat] += 1;
            if (cat == 0 && flags[idx] == 0) c[kCategories] += 1;
        }
    }
    for (int cat = 0; cat < kCounters; ++cat) {
        uint32_t tot;
        block_exclusive_scan(c[cat], &tot);
        if (threadIdx.x == 0) counts[cat * nblk + blockIdx.x] = tot;
    }
}

// One block: exclusive scan of counts[kCategories * nblk] (category-major) into
// offsets, and the category totals.
__global__ void setup_scan(const uint32_t* __restrict__ counts, int nblk, uint32_t* __restrict__ offsets,
                           uint32_t* __restrict__ totals)
{
    __shared__ uint32_t part[1024];
    const int n = kCategories * nblk;
    const int per = (n + 1023) / 1024;
    const int lo = threadIdx.x * per;
    const int hi = min(n, lo + per);
    uint32_t s = 0;
    for (int k = lo; k < hi; ++k) s += counts[k];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int k = 0; k < 1024; ++k) {
            uint32_t v = part[k];
            part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int k = lo; k < hi; ++k) {
        offsets[k] = run;
        run += counts[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int cat = 0; cat < kCounters; ++cat) {
            uint32_t t = 0;
            for (int b = 0; b < nblk; ++b) t += counts[cat * nblk + b];
            totals[cat] = t;
        }
    }
}

__global__ void setup_emit(const uint8_t* __restrict__ flags, long long N, CellGrid G, int nblk,
                           const uint32_t* __restrict__ offsets, uint32_t* __restrict__ cells)
{
    const long long base = (long long)blockIdx.x * kSetupChunk + (long long)threadIdx.x * kSetupCellsPerThread;
    const bool gb = group_has_bulk(flags, base, N, G);
    uint32_t c[kCategories] = {0, 0, 0, 0};
    for (int k = 0; k < kSetupCellsPerThread; ++k) {
        const long long idx = base + k;
        if (idx < N) {
            const int cat = category(flags[idx], idx, G, gb);
            if (cat >= 0) c[cat] += 1;
        }
    }
    uint32_t pos[kCategories];
    for (int cat = 0; cat < kCategories; ++cat) {
        uint32_t tot;
        pos[cat] = offsets[cat * nblk + blockIdx.x] + block_exclusive_scan(c[cat], &tot);
    }
    for (int k = 0; k < kSetupCellsPerThread; ++k) {
        const long long idx = base + k;
        if (idx < N) {
            const int cat = category(flags[idx], idx, G, gb);
            if (cat >= 0) cells[pos[cat]++] = (uint32_t)idx | (flags[idx] == 0 ? kGhostFlag : 0u);
        }
    }
}

// Position of (x, y, z) + d; returns false when it leaves the box across a
// non-periodic face (axis / side of that face in *ax / *sd).
__device__ __forceinline__ bool step_to(const SetupParams& S, int x, int y, int z, int dx, int dy, int dz,
                                        long long* out, int* ax, int* sd)
{
    int v[3] = {x + dx, y + dy, z + dz};
    const int n[3] = {S.nx, S.ny, S.nz};
    *ax = -1;
    *sd = 0;
    for (int a = 0; a < 3; ++a) {
        if (v[a] < 0 || v[a] >= n[a]) {
            if (S.periodic[a]) {
                v[a] = v[a] < 0 ? v[a] + n[a] : v[a] - n[a];
            } else {
                *ax = a;
                *sd = v[a] < 0 ? 0 : 1;
                return false;
            }
        }
    }
    *out = v[0] + (long long)n[0] * (v[1] + (long long)n[1] * v[2]);
    return true;
}

// Link mask of a non-solid cell (see kernels.cuh for the bit layout).
template <int Q>
__device__ uint32_t link_mask(const SetupParams& S, int x, int y, int z, int type)
{
    using L = Lattice<Q>;
    const long long idx = x + (long long)S.nx * (y + (long long)S.ny * z);
    const float phi = S.phi[idx];
    uint32_t m = (uint32_t)type << kTypeShift;
    if ((S.periodic[0] && (x == 0 || x == S.nx - 1)) || (S.periodic[1] && (y == 0 || y == S.ny - 1)) ||
        (S.periodic[2] && (z == 0 || z == S.nz - 1)))
        m |= kWrapBit;
    for (int i = 0; i < Q; ++i) {
        long long s;
        int ax, sd;
        if (!step_to(S, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i), &s, &ax, &sd) || S.flags[s] == 0) m |= 1u << i;
    }
    for (int i = 1; i < Q; ++i) {
        long long d;
        int ax, sd;
        if (step_to(S, x, y, z, L::cx(i), L::cy(i), L::cz(i), &d, &ax, &sd) && S.flags[d] != 0 && S.phi[d] != phi)
            m |= kPorousBit;
    }
    return m;
}

template <int Q>
__global__ void setup_mask(const SetupParams S)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n_cells) return;
    const uint32_t pc = S.cells[p];
    if (pc & kGhostFlag) {
        S.mask[p] = kGhostFlag;
        return;
    }
    const long long idx = pc;
    const long long plane = (long long)S.nx * S.ny;
    const int z = (int)(idx / plane);
    const int y = (int)((idx - (long long)z * plane) / S.nx);
    const int x = (int)(idx - (long long)z * plane - (long long)y * S.nx);
    const uint8_t fl = S.flags[idx];
    const float phi = S.phi[idx];
    uint32_t err = 0;
    if (!(phi > 0.0f) || !(phi <= 1.0f)) err |= kErrPorosity;
    const int type = fl == 2 ? kInlet : fl == 3 ? kOutlet : kBulk;
    S.mask[p] = link_mask<Q>(S, x, y, z, type);
    if (type == kInlet) {
        const int a = S.in_axis;
        const int coord = a == 0 ? x : a == 1 ? y : z;
        const int extent = a == 0 ? S.nx : a == 1 ? S.ny : S.nz;
        const int per = a == 0 ? S.periodic[0] : a == 1 ? S.periodic[1] : S.periodic[2];
        const int face = S.in_side == 0 ? 0 : extent - 1;
        uint32_t why = 0;
        if (a < 0 || a > 2) why |= 1u;
        if (per) why |= 2u;
        if (coord != face) why |= 4u;
        if (phi != 1.0f) why |= 8u;
        if (why) {
            err |= kErrInlet | (why << 8);
        } else {
            const double px = x + 0.5, py = y + 0.5, pz = z + 0.5;
            const double dx = a == 0 ? 0.0 : px - S.in_center[0];
            const double dy = a == 1 ? 0.0 : py - S.in_center[1];
            const double dz = a == 2 ? 0.0 : pz - S.in_center[2];
            const double prof = 1.0 - (dx * dx + dy * dy + dz * dz) / (S.in_radius * S.in_radius);
            S.bnd_prof[p - S.n_bulk] = (float)(2.0 * (prof > 0.0 ? prof : 0.0));
            S.bnd_nbmask[p - S.n_bulk] = 0u;
        }
    } else if (type == kOutlet) {
        const int a = S.out_axis;
        const int coord = a == 0 ? x : a == 1 ? y : z;
        const int extent = a == 0 ? S.nx : a == 1 ? S.ny : S.nz;
        const int per = a == 0 ? S.periodic[0] : a == 1 ? S.periodic[1] : S.periodic[2];
        const int face = S.out_side == 0 ? 0 : extent - 1;
        bool ok = a >= 0 && a <= 2 && !per && coord == face && phi == 1.0f;
        if (ok) {
            const int sg = S.out_side == 1 ? -1 : 1;
            const int bx = x + (a == 0 ? sg : 0), by = y + (a == 1 ? sg : 0), bz = z + (a == 2 ? sg : 0);
            const int bc = coord + sg;
            ok = bc >= 0 && bc < extent;
            if (ok) {
                const long long nb = bx + (long long)S.nx * (by + (long long)S.ny * bz);
                ok = S.flags[nb] == 1 && S.phi[nb] == 1.0f;
                if (ok) S.bnd_nbmask[p - S.n_bulk] = link_mask<Q>(S, bx, by, bz, kBulk);
            }
            S.bnd_prof[p - S.n_bulk] = 0.0f;
        }
        if (!ok) err |= kErrOutlet;
    }
    if (err) {
        // keep the first offending cell for the error message: err[1] = 1 + list
        // position, err[2] = packed coordinates, err[3] = porosity bits,
        // err[4] = inlet reason bits
        if (atomicCAS(S.err + 1, 0u, (uint32_t)p + 1u) == 0u) {
            S.err[2] = pc;
            S.err[3] = __float_as_uint(phi);
            S.err[4] = err >> 8;
        }
        atomicOr(S.err, err & 0xffu);
    }
}


// Rest state: all deviations zero (f_i = w_i phi, rho = 1, u = 0) and the
// relaxation rate of mu0 at rho = 1.
template <class T>
__global__ void init_state(const uint32_t* __restrict__ cells, int n_cells, int nx, int ny, long long N, int Q,
                           T* __restrict__ f, float* __restrict__ omega, float omega0)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_cells) return;
    const long long idx = cells[p] & ~kGhostFlag;
    for (int i = 0; i < Q; ++i) f[(long long)i * N + idx] = T(0.0f);
    omega[p] = omega0;
}

// Checkpoints in list order: state[i][p] = f[i][idx(p)] (raw storage type).
template <class T>
__global__ void pack_state(const uint32_t* __restrict__ cells, int n_cells, int nx, int ny, long long N, int Q,
                           const T* __restrict__ f, T* __restrict__ state, int unpack, T* __restrict__ fout,
                           const T* __restrict__ state_in)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_cells) return;
    const long long idx = cells[p] & ~kGhostFlag;
    if (unpack) {
        for (int i = 0; i < Q; ++i) fout[(long long)i * N + idx] = state_in[(long long)i * n_cells + p];
    } else {
        for (int i = 0; i < Q; ++i) state[(long long)i * n_cells + p] = f[(long long)i * N + idx];
    }
}

__global__ void diag_finish(const double* __restrict__ partials, int nblk, double* __restrict__ out)
{
    __shared__ double sm[kBlock][kDiagSlots];
    double r[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1e300, -1e300, 0.0};
    for (int b = threadIdx.x; b < nblk; b += kBlock) {
        const double* v = partials + (size_t)b * kDiagSlots;
        for (int k = 0; k < 5; ++k) r[k] += v[k];
        r[5] = fmax(r[5], v[5]);
        r[6] = fmin(r[6], v[6]);
        r[7] = fmax(r[7], v[7]);
        r[8] += v[8];
    }
    for (int k = 0; k < kDiagSlots; ++k) sm[threadIdx.x][k] = r[k];
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 5; ++k) sm[threadIdx.x][k] += sm[threadIdx.x + s][k];
            sm[threadIdx.x][5] = fmax(sm[threadIdx.x][5], sm[threadIdx.x + s][5]);
            sm[threadIdx.x][6] = fmin(sm[threadIdx.x][6], sm[threadIdx.x + s][6]);
            sm[threadIdx.x][7] = fmax(sm[threadIdx.x][7], sm[threadIdx.x + s][7]);
            sm[threadIdx.x][8] += sm[threadIdx.x + s][8];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double* v = sm[0];
        out[0] = v[0] + v[1];  // mass: sum phi + sum (phi rho - phi)
        out[1] = v[2];
        out[2] = v[3];
        out[3] = v[4];
        out[4] = v[5];
        out[5] = v[6];
        out[6] = v[7];
        out[7] = v[8];
    }
}

// v into p[0..n).
__global__ void fill_f32(float* p, long long n, float v)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Number of listed non-ghost cells whose region byte is set.
__global__ void region_count(const uint32_t* cells, int n_cells, const uint8_t* region, unsigned long long* out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int hit = 0;
    if (p < n_cells) {
        const uint32_t e = cells[p];
        hit = !(e & kGhostFlag) && region[e] ? 1 : 0;
    }
    const unsigned int warp_hits = __popc(__ballot_sync(0xffffffffu, hit));
    if ((threadIdx.x & 31) == 0 && warp_hits) atomicAdd(out, (unsigned long long)warp_hits);
}

// Host launchers (kernel templates cannot be launched across translation units).
cudaError_t launch_fill_f32(float* p, long long n, float v, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    fill_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_region_count(const uint32_t* cells, int n_cells, const uint8_t* region, unsigned long long* out,
                                cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n_cells == 0) return e;
    region_count<<<(n_cells + 255) / 256, 256, 0, s>>>(cells, n_cells, region, out);
    return cudaGetLastError();
}

cudaError_t launch_setup_mask(int q, const SetupParams& S, cudaStream_t s)
{
    if (S.n_cells == 0) return cudaSuccess;
    const int g = (S.n_cells + 255) / 256;
    if (q == 19)
        setup_mask<19><<<g, 256, 0, s>>>(S);
    else
        setup_mask<27><<<g, 256, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int storage, const uint32_t* cells, int n_cells, int nx, int ny, long long N, int Q,
                              void* f, float* omega, float omega0, cudaStream_t s)
{
    if (n_cells == 0) return cudaSuccess;
    const int g = (n_cells + 255) / 256;
    if (storage == 0)
        init_state<float><<<g, 256, 0, s>>>(cells, n_cells, nx, ny, N, Q, static_cast<float*>(f), omega, omega0);
    else if (storage == 1)
        init_state<__half><<<g, 256, 0, s>>>(cells, n_cells, nx, ny, N, Q, static_cast<__half*>(f), omega, omega0);
    else
        init_state<__nv_bfloat16><<<g, 256, 0, s>>>(cells, n_cells, nx, ny, N, Q, static_cast<__nv_bfloat16*>(f),
                                                     omega, omega0);
    return cudaGetLastError();
}

cudaError_t launch_pack_state(int storage, const uint32_t* cells, int n_cells, int nx, int ny, long long N, int Q,
                              void* f, void* state, int unpack, cudaStream_t s)
{
    if (n_cells == 0) return cudaSuccess;
    const int g = (n_cells + 255) / 256;
    if (storage == 0)
        pack_state<float><<<g, 256, 0, s>>>(cells, n_cells, nx, ny, N, Q, static_cast<const float*>(f),
                                             static_cast<float*>(state), unpack, static_cast<float*>(f),
                                             static_cast<const float*>(state));
    else if (storage == 1)
        pack_state<__half><<<g, 256, 0, s>>>(cells, n_cells, nx, ny, N, Q, static_cast<const __half*>(f),
                                              static_cast<__half*>(state), unpack, static_cast<__half*>(f),
                                              static_cast<const __half*>(state));
    else
        pack_state<__nv_bfloat16><<<g, 256, 0, s>>>(cells, n_cells, nx, ny, N, Q,
                                                     static_cast<const __nv_bfloat16*>(f),
                                                     static_cast<__nv_bfloat16*>(state), unpack,
                                                     static_cast<__nv_bfloat16*>(f),
                                                     static_cast<const __nv_bfloat16*>(state));
    return cudaGetLastError();
}

cudaError_t launch_setup_cells(const uint8_t* flags, long long N, const CellGrid& G, uint32_t* counts,
                               uint32_t* offsets, uint32_t* totals, cudaStream_t s, int phase, uint32_t* cells)
{
    const int nblk = (int)((N + kSetupChunk - 1) / kSetupChunk);
    if (phase == 0) {
        setup_count<<<nblk, kSetupThreads, 0, s>>>(flags, N, G, nblk, counts);
        setup_scan<<<1, 1024, 0, s>>>(counts, nblk, offsets, totals);
    } else {
        setup_emit<<<nblk, kSetupThreads, 0, s>>>(flags, N, G, nblk, offsets, cells);
    }
    return cudaGetLastError();
}

cudaError_t launch_diag_finish(const double* partials, int nblk, double* out, cudaStream_t s)
{
    if (nblk == 0) return cudaSuccess;
    diag_finish<<<1, kBlock, 0, s>>>(partials, nblk, out);
    return cudaGetLastError();
}

}  // namespace lbm
