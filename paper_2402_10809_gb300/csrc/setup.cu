// Set-up kernels: the row spans of the packed layout, the per-slot row ids,
// porosity, link masks and boundary data, small utility kernels and the final
// diagnostics reduction.  The spans are scanned on the host (their count is
// the number of rows), so the layout is deterministic.
#include <stdint.h>

#include "kernels.cuh"
#include "setup.cuh"

namespace lbm {

__device__ __forceinline__ bool fluid_flag(uint8_t f) { return f >= 1 && f <= 3; }

// One warp per row (y, z): the span [xmin, xmax] of its non-solid cells
// (ext = 0 for a row without any); flags outside 0..3 raise kErrFlag.
__global__ void setup_rows(const uint8_t* __restrict__ flags, int nx, int nrows, int* __restrict__ xmin,
                           int* __restrict__ ext, uint32_t* __restrict__ err)
{
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const uint8_t* row = flags + (size_t)r * nx;
    int lo = nx, hi = -1;
    bool bad = false;
    for (int x0 = 0; x0 < nx; x0 += 32) {
        const int x = x0 + lane;
        const uint8_t f = x < nx ? row[x] : 0;
        bad |= f > 3;
        const uint32_t b = __ballot_sync(0xffffffffu, fluid_flag(f));
        if (b) {
            lo = min(lo, x0 + __ffs(b) - 1);
            hi = max(hi, x0 + 31 - __clz(b));
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, kErrFlag);
    if (lane == 0) {
        xmin[r] = hi >= 0 ? lo : 0;
        ext[r] = hi >= 0 ? hi - lo + 1 : 0;
    }
}

// One warp per row: the row id of each slot of its span and the packed porosity.
__global__ void setup_slots(const float* __restrict__ phi, int nx, int nrows, const int* __restrict__ rowbase,
                            const int* __restrict__ xmin, const int* __restrict__ ext, uint32_t* __restrict__ rows,
                            float* __restrict__ phi_s)
{
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const int e = ext[r];
    const int x0 = xmin[r];
    const long long s0 = (long long)rowbase[r] + x0;
    for (int k = lane; k < e; k += 32) {
        rows[s0 + k] = (uint32_t)r;
        phi_s[s0 + k] = phi[(size_t)r * nx + x0 + k];
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
    // one visit per neighbour (x, y, z) + c_i: it is the pull source of
    // direction opp(i) (bit opp(i) set when it is not fluid or outside the
    // box) and, when fluid with another porosity, makes the cell porous
    for (int i = 1; i < Q; ++i) {
        long long d;
        int ax, sd;
        if (step_to(S, x, y, z, L::cx(i), L::cy(i), L::cz(i), &d, &ax, &sd) && fluid_flag(S.flags[d])) {
            if (S.phi[d] != phi) m |= kPorousBit;
        } else {
            m |= 1u << opp(i);
        }
    }
    return m;
}

// One thread per row (y, z): the bases of its nine neighbour rows
// (y + sy, z + sz) at index (sy + 1) + 3 (sz + 1), wrapped on periodic axes,
// 0 outside the box (those links are never pulled), then y, z, 0.
__global__ void setup_rownb(const int* __restrict__ rowbase, int ny, int nz, int py, int pz, int* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ny * nz) return;
    const int y = r % ny, z = r / ny;
    int* e = out + (size_t)r * 12;
#pragma unroll
    for (int sz = -1; sz <= 1; ++sz)
#pragma unroll
        for (int sy = -1; sy <= 1; ++sy) {
            int yy = y + sy, zz = z + sz;
            if (py) yy = (yy + ny) % ny;
            if (pz) zz = (zz + nz) % nz;
            e[(sy + 1) + 3 * (sz + 1)] = (yy >= 0 && yy < ny && zz >= 0 && zz < nz) ? rowbase[yy + ny * zz] : 0;
        }
    e[9] = y;
    e[10] = z;
    e[11] = 0;
}

// Dense index of slot q.
__device__ __forceinline__ long long slot_dense(const SetupParams& S, int q)
{
    const uint32_t r = S.rows[q];
    return (long long)(q - S.rowbase[r]) + (long long)S.nx * r;
}

template <int Q>
__global__ void setup_mask(const SetupParams S)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n_store) return;
    const uint32_t r = S.rows[p];
    const int x = p - S.rowbase[r];
    const int y = (int)(r % (uint32_t)S.ny);
    const int z = (int)(r / (uint32_t)S.ny);
    const long long idx = x + (long long)S.nx * r;
    const uint8_t fl = S.flags[idx];
    if (!fluid_flag(fl)) {
        // ghost slot: zero stores only where an aligned 8-slot group holds fluid
        const int g0 = p & ~7;
        bool store = false;
        for (int q = g0; q < g0 + 8 && q < S.n_store; ++q) store |= fluid_flag(S.flags[slot_dense(S, q)]);
        S.mask[p] = kGhostBit | (store ? 1u : 0u);
        S.bnd_prof[p] = 0.0f;
        S.bnd_nbmask[p] = 0u;
        return;
    }
    const float phi = S.phi[idx];
    uint32_t err = 0;
    if (!(phi > 0.0f) || !(phi <= 1.0f)) err |= kErrPorosity;
    const int type = fl == 2 ? kInlet : fl == 3 ? kOutlet : kBulk;
    S.mask[p] = link_mask<Q>(S, x, y, z, type);
    S.bnd_prof[p] = 0.0f;
    S.bnd_nbmask[p] = 0u;
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
            S.bnd_prof[p] = (float)(2.0 * (prof > 0.0 ? prof : 0.0));
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
                if (ok) S.bnd_nbmask[p] = link_mask<Q>(S, bx, by, bz, kBulk);
            }
        }
        if (!ok) err |= kErrOutlet;
    }
    if (err) {
        // keep the first offending cell for the error message: err[1] = 1 + slot,
        // err[2] = packed coordinates x | y << 10 | z << 20, err[3] = porosity
        // bits, err[4] = inlet reason bits
        if (atomicCAS(S.err + 1, 0u, (uint32_t)p + 1u) == 0u) {
            S.err[2] = (uint32_t)x | ((uint32_t)y << 10) | ((uint32_t)z << 20);
            S.err[3] = __float_as_uint(phi);
            S.err[4] = err >> 8;
        }
        atomicOr(S.err, err & 0xffu);
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

// v into p[0..n).
__global__ void fill_u32(uint32_t* p, long long n, uint32_t v)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Slot classes of the host tables, in chunks of kClassChunk slots (each of
// the kClassBlock threads takes kClassPer consecutive slots): general-path
// cells (inlet, outlet, periodic wrap; every cell when wide), outlet cells,
// ghost slots, inlet cells.
constexpr int kClassBlock = 256, kClassPer = 4, kClassChunk = kClassBlock * kClassPer;

__device__ __forceinline__ void slot_classes(const uint32_t* __restrict__ mask, int n, int wide, int first, int& gen,
                                             int& out, int& ghost, int& inl)
{
    gen = out = ghost = inl = 0;
    for (int k = 0; k < kClassPer; ++k) {
        const int p = first + k;
        if (p >= n) break;
        const uint32_t m = mask[p];
        if (m & kGhostBit) {
            ++ghost;
            continue;
        }
        const uint32_t type = (m >> kTypeShift) & 3u;
        gen += (wide || (m & kGeneralBits)) ? 1 : 0;
        out += type == kOutlet;
        inl += type == kInlet;
    }
}

// Exclusive scan over the block of v (ordered by thread), and the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total)
{
    __shared__ int warp_sum[kClassBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < kClassBlock / 32; ++w) {
        before += w < wid ? warp_sum[w] : 0;
        all += warp_sum[w];
    }
    *total = all;
    return before + x - v;
}

// Per chunk: counts of general, outlet, ghost and inlet slots.
__global__ void __launch_bounds__(kClassBlock) classify_count(const uint32_t* __restrict__ mask, int n, int wide,
                                                              int4* __restrict__ counts)
{
    int g, o, h, i;
    slot_classes(mask, n, wide, blockIdx.x * kClassChunk + threadIdx.x * kClassPer, g, o, h, i);
    int tg, to, th, ti;
    block_exclusive_scan(g, &tg);
    __syncthreads();
    block_exclusive_scan(o, &to);
    __syncthreads();
    block_exclusive_scan(h, &th);
    __syncthreads();
    block_exclusive_scan(i, &ti);
    if (threadIdx.x == 0) counts[blockIdx.x] = make_int4(tg, to, th, ti);
}

// The general and outlet slots in ascending order, chunk c starting at
// offsets[c] (x: general list, y: outlet list).
__global__ void __launch_bounds__(kClassBlock) classify_write(const uint32_t* __restrict__ mask, int n, int wide,
                                                              const int2* __restrict__ offsets,
                                                              uint32_t* __restrict__ general,
                                                              uint32_t* __restrict__ outlets)
{
    const int first = blockIdx.x * kClassChunk + threadIdx.x * kClassPer;
    int g, o, h, i, tot;
    slot_classes(mask, n, wide, first, g, o, h, i);
    int pg = offsets[blockIdx.x].x + block_exclusive_scan(g, &tot);
    __syncthreads();
    int po = offsets[blockIdx.x].y + block_exclusive_scan(o, &tot);
    for (int k = 0; k < kClassPer; ++k) {
        const int p = first + k;
        if (p >= n) break;
        const uint32_t m = mask[p];
        if (m & kGhostBit) continue;
        if (wide || (m & kGeneralBits)) general[pg++] = (uint32_t)p;
        if (((m >> kTypeShift) & 3u) == kOutlet) outlets[po++] = (uint32_t)p;
    }
}

// Number of non-ghost slots whose region byte (dense) is set; with wall_bits
// nonzero only plain fluid cells with a wall link (mask & wall_bits) count.
__global__ void region_count(const uint32_t* __restrict__ rows, const int* __restrict__ rowbase,
                             const uint32_t* __restrict__ mask, int n_store, int nx, const uint8_t* __restrict__ region,
                             uint32_t wall_bits, unsigned long long* out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    int hit = 0;
    if (p < n_store && !(mask[p] & kGhostBit)) {
        const uint32_t m = mask[p];
        const bool ok = !wall_bits || ((m & wall_bits) && ((m >> kTypeShift) & 3u) == kBulk);
        const uint32_t r = rows[p];
        hit = ok && region[(long long)(p - rowbase[r]) + (long long)nx * r] ? 1 : 0;
    }
    const unsigned int warp_hits = __popc(__ballot_sync(0xffffffffu, hit));
    if ((threadIdx.x & 31) == 0 && warp_hits) atomicAdd(out, (unsigned long long)warp_hits);
}

// dst[dense index of p] = src[p] for every non-ghost slot p.
__global__ void scatter_f64(const uint32_t* __restrict__ rows, const int* __restrict__ rowbase,
                            const uint32_t* __restrict__ mask, int n_store, int nx, const double* __restrict__ src,
                            double* __restrict__ dst)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_store || (mask[p] & kGhostBit)) return;
    const uint32_t r = rows[p];
    dst[(long long)(p - rowbase[r]) + (long long)nx * r] = src[p];
}

// Task blockIdx.y of a halo copy, grid-strided over its elements.
__global__ void halo_copy(const HaloCopy H)
{
    const int k = blockIdx.y;
    if (k >= H.ntask) return;
    const long long n = H.count[k];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        if (H.elem == 4)
            static_cast<uint32_t*>(H.dst[k])[e] = static_cast<const uint32_t*>(H.src[k])[e];
        else
            static_cast<uint16_t*>(H.dst[k])[e] = static_cast<const uint16_t*>(H.src[k])[e];
    }
}

// Host launchers (kernel templates cannot be launched across translation units).
cudaError_t launch_setup_rows(const uint8_t* flags, int nx, int nrows, int* xmin, int* ext, uint32_t* err,
                              cudaStream_t s)
{
    if (nrows == 0) return cudaSuccess;
    const int per_block = kSetupThreads / 32;
    setup_rows<<<(nrows + per_block - 1) / per_block, kSetupThreads, 0, s>>>(flags, nx, nrows, xmin, ext, err);
    return cudaGetLastError();
}

cudaError_t launch_setup_slots(const float* phi, int nx, int nrows, const int* rowbase, const int* xmin,
                               const int* ext, uint32_t* rows, float* phi_s, cudaStream_t s)
{
    if (nrows == 0) return cudaSuccess;
    const int per_block = kSetupThreads / 32;
    setup_slots<<<(nrows + per_block - 1) / per_block, kSetupThreads, 0, s>>>(phi, nx, nrows, rowbase, xmin, ext,
                                                                              rows, phi_s);
    return cudaGetLastError();
}

cudaError_t launch_setup_rownb(const int* rowbase, int ny, int nz, int py, int pz, int* out, cudaStream_t s)
{
    const int nrows = ny * nz;
    if (nrows == 0) return cudaSuccess;
    setup_rownb<<<(nrows + 255) / 256, 256, 0, s>>>(rowbase, ny, nz, py, pz, out);
    return cudaGetLastError();
}

cudaError_t launch_setup_mask(int q, const SetupParams& S, cudaStream_t s)
{
    if (S.n_store == 0) return cudaSuccess;
    const int g = (S.n_store + 255) / 256;
    if (q == 19)
        setup_mask<19><<<g, 256, 0, s>>>(S);
    else
        setup_mask<27><<<g, 256, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(float* p, long long n, float v, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    fill_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, long long n, uint32_t v, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    fill_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

int classify_chunks(int n) { return (n + kClassChunk - 1) / kClassChunk; }

cudaError_t launch_classify_count(const uint32_t* mask, int n, int wide, int4* counts, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    classify_count<<<classify_chunks(n), kClassBlock, 0, s>>>(mask, n, wide, counts);
    return cudaGetLastError();
}

cudaError_t launch_classify_write(const uint32_t* mask, int n, int wide, const int2* offsets, uint32_t* general,
                                  uint32_t* outlets, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    classify_write<<<classify_chunks(n), kClassBlock, 0, s>>>(mask, n, wide, offsets, general, outlets);
    return cudaGetLastError();
}

cudaError_t launch_region_count(const uint32_t* rows, const int* rowbase, const uint32_t* mask, int n_store, int nx,
                                const uint8_t* region, uint32_t wall_bits, unsigned long long* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n_store == 0) return e;
    region_count<<<(n_store + 255) / 256, 256, 0, s>>>(rows, rowbase, mask, n_store, nx, region, wall_bits, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_f64(const uint32_t* rows, const int* rowbase, const uint32_t* mask, int n_store, int nx,
                               const double* src, double* dst, cudaStream_t s)
{
    if (n_store == 0) return cudaSuccess;
    scatter_f64<<<(n_store + 255) / 256, 256, 0, s>>>(rows, rowbase, mask, n_store, nx, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_halo_copy(const HaloCopy& H, cudaStream_t s)
{
    long long most = 0;
    for (int k = 0; k < H.ntask; ++k) most = H.count[k] > most ? H.count[k] : most;
    if (H.ntask == 0 || most == 0) return cudaSuccess;
    const long long bx = (most + 255) / 256;
    dim3 grid((unsigned)(bx < 1024 ? bx : 1024), (unsigned)H.ntask);
    halo_copy<<<grid, 256, 0, s>>>(H);
    return cudaGetLastError();
}

cudaError_t launch_diag_finish(const double* partials, int nblk, double* out, cudaStream_t s)
{
    if (nblk == 0) return cudaSuccess;
    diag_finish<<<1, kBlock, 0, s>>>(partials, nblk, out);
    return cudaGetLastError();
}

}  // namespace lbm
