// Volume-averaged porosity of a voxelised coil (Sec. 4: windowed convolution
// of the voxelised coil with a uniform averaging kernel; Table 1: averaging
// window).  phi(x) = max(phi_min, (W^3 - count(x)) / W^3), count(x) the number
// of wire voxels in the box [x - lo, x + hi] on every axis (lo = W / 2,
// hi = W - 1 - lo, nothing outside the box), phi = 1 on solid cells.
//
// The box count is separable and exact in integers, so it runs as three
// sliding-window passes, each an HBM stream:
//   x: wire bytes -> per-row counts (uint8, <= W), rows staged in shared memory
//      R at a time (R rows are one contiguous byte range, loaded coalesced);
//   y: uint8 -> uint16 (<= W^2) running sums down y, one thread per V
//      consecutive x and a segment of rows;
//   z: uint16 -> FP32 porosity, the same along z, with the solid override and
//      the correctly rounded quotient (both operands are integers below 2^24).
// The y and z running sums keep their last W inputs in a shared-memory ring
// (the value leaving the window is the one that entered W cells earlier), so
// each input is read once; for windows whose ring would exceed 48 KB they
// read the leaving value again from global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "setup.cuh"

namespace lbm {
namespace {

constexpr int kPorBlock = 256;
constexpr int kSeg = 64;      // cells of the y / z axis per thread
constexpr int kChunk = 32;    // outputs per sliding task of the x pass

// Shared-memory row stride of the x pass: whole words, an odd number of them,
// so that lanes on consecutive rows hit distinct banks.
__host__ __device__ inline int x_stride(int nx)
{
    int words = (nx + 3) / 4;
    if (!(words & 1)) ++words;
    return 4 * words;
}

__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t w)
{
    // bit 0 of each byte becomes the OR of that byte's bits (no carries across
    // bytes reach bit 0), then keep bit 0 only
    w |= w >> 4;
    w |= w >> 2;
    w |= w >> 1;
    return w & 0x01010101u;
}

// x pass: block b handles rows [b R, b R + R) of the nrows = ny nz rows.
template <bool kVec>
__global__ void __launch_bounds__(kPorBlock) box_x(const uint8_t* __restrict__ wire, uint8_t* __restrict__ out,
                                                   int nx, long long nrows, int R, int lo, int hi)
{
    extern __shared__ uint32_t sm_words[];
    uint8_t* sin = reinterpret_cast<uint8_t*>(sm_words);
    const int stride = x_stride(nx);
    uint8_t* sout = sin + (size_t)R * stride;
    const long long r0 = (long long)blockIdx.x * R;
    const int nr = (int)min((long long)R, nrows - r0);
    const uint8_t* src = wire + r0 * nx;
    uint8_t* dst = out + r0 * nx;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarp = kPorBlock / 32;
    // stage: one warp per row, 0/1 bytes
    for (int r = warp; r < nr; r += nwarp) {
        if (kVec) {
            const uint32_t* s = reinterpret_cast<const uint32_t*>(src + (size_t)r * nx);
            uint32_t* d = reinterpret_cast<uint32_t*>(sin + (size_t)r * stride);
            for (int c = lane; c < nx / 4; c += 32) d[c] = nonzero_bytes(__ldcs(s + c));
        } else {
            for (int c = lane; c < nx; c += 32) sin[(size_t)r * stride + c] = src[(size_t)r * nx + c] != 0;
        }
    }
    __syncthreads();
    // sliding sums: task k covers row k % nr, outputs [kChunk (k / nr), + kChunk)
    const int nchunk = (nx + kChunk - 1) / kChunk;
    for (int k = threadIdx.x; k < nr * nchunk; k += kPorBlock) {
        const int r = k % nr;
        const int x0 = (k / nr) * kChunk;
        const int x1 = min(x0 + kChunk, nx);
        const uint8_t* row = sin + (size_t)r * stride;
        uint8_t* orow = sout + (size_t)r * stride;
        int s = 0;
        for (int j = max(0, x0 - lo); j <= min(nx - 1, x0 + hi); ++j) s += row[j];
        orow[x0] = (uint8_t)s;
        for (int x = x0 + 1; x < x1; ++x) {
            if (x + hi < nx) s += row[x + hi];
            if (x - lo - 1 >= 0) s -= row[x - lo - 1];
            orow[x] = (uint8_t)s;
        }
    }
    __syncthreads();
    for (int r = warp; r < nr; r += nwarp) {
        if (kVec) {
            const uint32_t* s = reinterpret_cast<const uint32_t*>(sout + (size_t)r * stride);
            uint32_t* d = reinterpret_cast<uint32_t*>(dst + (size_t)r * nx);
            for (int c = lane; c < nx / 4; c += 32) d[c] = s[c];
        } else {
            for (int c = lane; c < nx; c += 32) dst[(size_t)r * nx + c] = sout[(size_t)r * stride + c];
        }
    }
}

template <int V, class T>
struct Vec;
template <>
struct Vec<1, uint8_t> {
    static __device__ __forceinline__ void ld(const uint8_t* p, int* v) { v[0] = p[0]; }
    static __device__ __forceinline__ void st(uint8_t* p, const int* v) { p[0] = (uint8_t)v[0]; }
};
template <>
struct Vec<4, uint8_t> {
    static __device__ __forceinline__ void ld(const uint8_t* p, int* v)
    {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
        v[0] = w & 0xff;
        v[1] = (w >> 8) & 0xff;
        v[2] = (w >> 16) & 0xff;
        v[3] = w >> 24;
    }
    static __device__ __forceinline__ void st(uint8_t* p, const int* v)
    {
        *reinterpret_cast<uint32_t*>(p) =
            (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) | ((uint32_t)v[3] << 24);
    }
};
template <>
struct Vec<1, uint16_t> {
    static __device__ __forceinline__ void ld(const uint16_t* p, int* v) { v[0] = p[0]; }
    static __device__ __forceinline__ void st(uint16_t* p, const int* v) { p[0] = (uint16_t)v[0]; }
};
template <>
struct Vec<4, uint16_t> {
    static __device__ __forceinline__ void ld(const uint16_t* p, int* v)
    {
        const uint2 w = *reinterpret_cast<const uint2*>(p);
        v[0] = w.x & 0xffff;
        v[1] = w.x >> 16;
        v[2] = w.y & 0xffff;
        v[3] = w.y >> 16;
    }
    static __device__ __forceinline__ void st(uint16_t* p, const int* v)
    {
        uint2 w;
        w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
        w.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
        *reinterpret_cast<uint2*>(p) = w;
    }
};

// Running sum along an axis of n cells with element stride `step` (in
// elements): thread (xv, seg, plane) covers V consecutive x of one line and the
// axis segment [seg kSeg, + kSeg).  `line` is the offset of the line's first
// element.  Emit(k, v) receives the window counts of axis cell k.
template <int V, class Tin, class Emit>
__device__ __forceinline__ void slide(const Tin* __restrict__ in, long long line, long long step, int n, int seg,
                                      int lo, int hi, Emit emit)
{
    const int k0 = seg * kSeg, k1 = min(k0 + kSeg, n);
    int s[V], a[V];
#pragma unroll
    for (int v = 0; v < V; ++v) s[v] = 0;
    for (int j = max(0, k0 - lo); j <= min(n - 1, k0 + hi); ++j) {
        Vec<V, Tin>::ld(in + line + j * step, a);
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] += a[v];
    }
    emit(k0, s);
    for (int k = k0 + 1; k < k1; ++k) {
        if (k + hi < n) {
            Vec<V, Tin>::ld(in + line + (k + hi) * step, a);
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] += a[v];
        }
        if (k - lo - 1 >= 0) {
            Vec<V, Tin>::ld(in + line + (k - lo - 1) * step, a);
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] -= a[v];
        }
        emit(k, s);
    }
}

// The same running sum with the trailing edge from a ring in shared memory:
// the thread keeps the last W = lo + hi + 1 inputs of its V cells (slot j mod W
// holds axis cell j; slots of cells never loaded stay zero, as cells outside
// the box count zero), so every input of the segment and its warm-up is read
// from global memory once.  ring: this thread's first element; slot stride
// `rs` elements.  Segments of seglen cells.
template <int V, class Tin, class Emit>
__device__ __forceinline__ void slide_ring(const Tin* __restrict__ in, long long line, long long step, int n, int seg,
                                           int seglen, int lo, int hi, Tin* ring, int rs, Emit emit)
{
    const int W = lo + hi + 1;
    const int k0 = seg * seglen, k1 = min(k0 + seglen, n);
    int s[V], a[V], z[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        s[v] = 0;
        z[v] = 0;
    }
    for (int j = 0; j < W; ++j) Vec<V, Tin>::st(ring + j * rs, z);
    for (int j = max(0, k0 - lo); j <= min(n - 1, k0 + hi - 1); ++j) {
        Vec<V, Tin>::ld(in + line + j * step, a);
        Vec<V, Tin>::st(ring + (j % W) * rs, a);
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] += a[v];
    }
    int slot = (k0 + hi) % W;
    // cells k + hi enter the window four at a time (their loads in flight
    // together), cell k - lo - 1 (same slot) leaves it
    for (int k = k0; k < k1; k += 4) {
        int a4[4][V];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k + u < k1 && k + u + hi < n)
                Vec<V, Tin>::ld(in + line + (long long)(k + u + hi) * step, a4[u]);
            else
#pragma unroll
                for (int v = 0; v < V; ++v) a4[u][v] = 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k + u >= k1) break;
            int o[V];
            Vec<V, Tin>::ld(ring + slot * rs, o);
            Vec<V, Tin>::st(ring + slot * rs, a4[u]);
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] += a4[u][v] - o[v];
            slot = slot + 1 == W ? 0 : slot + 1;
            emit(k + u, s);
        }
    }
}

// y pass: uint8 row counts -> uint16 counts of the x-y window.
template <int V>
__global__ void __launch_bounds__(kPorBlock) box_y(const uint8_t* __restrict__ in, uint16_t* __restrict__ out, int nx,
                                                   int ny, int nz, int lo, int hi)
{
    const int nxv = nx / V, nseg = (ny + kSeg - 1) / kSeg;
    const long long t = (long long)blockIdx.x * kPorBlock + threadIdx.x;
    if (t >= (long long)nxv * nseg * nz) return;
    const int xv = (int)(t % nxv);
    const long long rest = t / nxv;
    const int seg = (int)(rest % nseg), z = (int)(rest / nseg);
    const long long line = (long long)z * ny * nx + (long long)xv * V;
    slide<V, uint8_t>(in, line, nx, ny, seg, lo, hi,
                      [&](int y, const int* s) { Vec<V, uint16_t>::st(out + line + (long long)y * nx, s); });
}

// z pass: uint16 x-y counts -> porosity.
template <int V>
__global__ void __launch_bounds__(kPorBlock) box_z(const uint16_t* __restrict__ in, const uint8_t* __restrict__ flags,
                                                   float* __restrict__ phi, int nx, int ny, int nz, int lo, int hi,
                                                   float w3, float phi_min)
{
    const int nxv = nx / V, nseg = (nz + kSeg - 1) / kSeg;
    const long long t = (long long)blockIdx.x * kPorBlock + threadIdx.x;
    const long long plane = (long long)nx * ny;
    if (t >= (long long)nxv * ny * nseg) return;
    const int xv = (int)(t % nxv);
    const long long rest = t / nxv;
    const int y = (int)(rest % ny), seg = (int)(rest / ny);
    const long long line = (long long)y * nx + (long long)xv * V;
    slide<V, uint16_t>(in, line, plane, nz, seg, lo, hi, [&](int z, const int* s) {
        const long long o = line + (long long)z * plane;
        float r[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // (W^3 - count) and W^3 are exact in FP32: one correctly rounded division
            r[v] = fmaxf(__fdiv_rn((float)((int)w3 - s[v]), w3), phi_min);
            if (flags && flags[o + v] == 0) r[v] = 1.0f;
        }
        if constexpr (V == 4)
            __stcs(reinterpret_cast<float4*>(phi + o), make_float4(r[0], r[1], r[2], r[3]));
        else
            __stcs(phi + o, r[0]);
    });
}

// Ring-buffered y and z passes: blocks of kRingBlock threads, segments of
// kRingSeg cells (longer than kSeg: the warm-up is read once per segment, and
// the trailing edge comes from the ring), ring of W slots per thread.
constexpr int kRingBlock = 128;
constexpr int kRingSeg = 128;

template <int V>
__global__ void __launch_bounds__(kRingBlock) box_y_ring(const uint8_t* __restrict__ in, uint16_t* __restrict__ out,
                                                         int nx, int ny, int nz, int lo, int hi)
{
    extern __shared__ uint32_t sm_ring[];
    uint8_t* ring = reinterpret_cast<uint8_t*>(sm_ring) + threadIdx.x * V;
    const int nxv = nx / V, nseg = (ny + kRingSeg - 1) / kRingSeg;
    const long long t = (long long)blockIdx.x * kRingBlock + threadIdx.x;
    if (t >= (long long)nxv * nseg * nz) return;
    const int xv = (int)(t % nxv);
    const long long rest = t / nxv;
    const int seg = (int)(rest % nseg), z = (int)(rest / nseg);
    const long long line = (long long)z * ny * nx + (long long)xv * V;
    slide_ring<V, uint8_t>(in, line, nx, ny, seg, kRingSeg, lo, hi, ring, kRingBlock * V,
                           [&](int y, const int* s) { Vec<V, uint16_t>::st(out + line + (long long)y * nx, s); });
}

template <int V>
__global__ void __launch_bounds__(kRingBlock) box_z_ring(const uint16_t* __restrict__ in,
                                                         const uint8_t* __restrict__ flags, float* __restrict__ phi,
                                                         int nx, int ny, int nz, int lo, int hi, float w3,
                                                         float phi_min)
{
    extern __shared__ uint32_t sm_ring[];
    uint16_t* ring = reinterpret_cast<uint16_t*>(sm_ring) + threadIdx.x * V;
    const int nxv = nx / V, nseg = (nz + kRingSeg - 1) / kRingSeg;
    const long long t = (long long)blockIdx.x * kRingBlock + threadIdx.x;
    const long long plane = (long long)nx * ny;
    if (t >= (long long)nxv * ny * nseg) return;
    const int xv = (int)(t % nxv);
    const long long rest = t / nxv;
    const int y = (int)(rest % ny), seg = (int)(rest / ny);
    const long long line = (long long)y * nx + (long long)xv * V;
    slide_ring<V, uint16_t>(in, line, plane, nz, seg, kRingSeg, lo, hi, ring, kRingBlock * V,
                            [&](int z, const int* s) {
                                const long long o = line + (long long)z * plane;
                                float r[V];
#pragma unroll
                                for (int v = 0; v < V; ++v) {
                                    // (W^3 - count) and W^3 are exact in FP32: one correctly rounded division
                                    r[v] = fmaxf(__fdiv_rn((float)((int)w3 - s[v]), w3), phi_min);
                                    if (flags && flags[o + v] == 0) r[v] = 1.0f;
                                }
                                if constexpr (V == 4)
                                    __stcs(reinterpret_cast<float4*>(phi + o), make_float4(r[0], r[1], r[2], r[3]));
                                else
                                    __stcs(phi + o, r[0]);
                            });
}

// Shared memory of a ring pass (W slots of V elements per thread); the ring
// passes run while it stays within the default 48 KB per block.
size_t ring_bytes(int window, int V, size_t elem) { return (size_t)window * kRingBlock * V * elem; }
constexpr size_t kRingMaxBytes = 48 * 1024;

unsigned grid_of(long long threads) { return (unsigned)((threads + kPorBlock - 1) / kPorBlock); }
unsigned ring_grid(long long threads) { return (unsigned)((threads + kRingBlock - 1) / kRingBlock); }

}  // namespace

size_t porosity_rows_per_block(int nx)
{
    const int r = kPorosityRowBytes / x_stride(nx);
    return (size_t)(r > 0 ? r : 1);
}

size_t porosity_smem_bytes(int nx) { return 2 * porosity_rows_per_block(nx) * (size_t)x_stride(nx); }

cudaError_t launch_porosity_average(const uint8_t* wire, const uint8_t* flags, int nx, int ny, int nz, int window,
                                    float phi_min, float* phi, uint8_t* ws_x, uint16_t* ws_y, cudaStream_t s)
{
    const int lo = window / 2, hi = window - 1 - lo;
    const long long nrows = (long long)ny * nz;
    const int R = (int)porosity_rows_per_block(nx);
    const size_t smem = porosity_smem_bytes(nx);
    // vector paths need whole 4-cell groups and aligned rows / pointers
    const bool vec = (nx % 4) == 0 && ((uintptr_t)wire % 4) == 0 && ((uintptr_t)phi % 16) == 0 &&
                     ((uintptr_t)flags % 4) == 0 && ((uintptr_t)ws_x % 4) == 0 && ((uintptr_t)ws_y % 8) == 0;
    const unsigned gx = (unsigned)((nrows + R - 1) / R);
    if (vec)
        box_x<true><<<gx, kPorBlock, smem, s>>>(wire, ws_x, nx, nrows, R, lo, hi);
    else
        box_x<false><<<gx, kPorBlock, smem, s>>>(wire, ws_x, nx, nrows, R, lo, hi);
    const float w3 = (float)window * (float)window * (float)window;
    const int V = vec ? 4 : 1;
    const size_t ry = ring_bytes(window, V, 1), rz = ring_bytes(window, V, 2);
    // y pass
    if (ry <= kRingMaxBytes) {
        const long long th = (long long)(nx / V) * ((ny + kRingSeg - 1) / kRingSeg) * nz;
        if (vec)
            box_y_ring<4><<<ring_grid(th), kRingBlock, ry, s>>>(ws_x, ws_y, nx, ny, nz, lo, hi);
        else
            box_y_ring<1><<<ring_grid(th), kRingBlock, ry, s>>>(ws_x, ws_y, nx, ny, nz, lo, hi);
    } else if (vec) {
        box_y<4><<<grid_of((long long)(nx / 4) * ((ny + kSeg - 1) / kSeg) * nz), kPorBlock, 0, s>>>(ws_x, ws_y, nx,
                                                                                                   ny, nz, lo, hi);
    } else {
        box_y<1><<<grid_of((long long)nx * ((ny + kSeg - 1) / kSeg) * nz), kPorBlock, 0, s>>>(ws_x, ws_y, nx, ny, nz,
                                                                                             lo, hi);
    }
    // z pass
    if (rz <= kRingMaxBytes) {
        const long long th = (long long)(nx / V) * ny * ((nz + kRingSeg - 1) / kRingSeg);
        if (vec)
            box_z_ring<4><<<ring_grid(th), kRingBlock, rz, s>>>(ws_y, flags, phi, nx, ny, nz, lo, hi, w3, phi_min);
        else
            box_z_ring<1><<<ring_grid(th), kRingBlock, rz, s>>>(ws_y, flags, phi, nx, ny, nz, lo, hi, w3, phi_min);
    } else if (vec) {
        box_z<4><<<grid_of((long long)(nx / 4) * ny * ((nz + kSeg - 1) / kSeg)), kPorBlock, 0, s>>>(
            ws_y, flags, phi, nx, ny, nz, lo, hi, w3, phi_min);
    } else {
        box_z<1><<<grid_of((long long)nx * ny * ((nz + kSeg - 1) / kSeg)), kPorBlock, 0, s>>>(ws_y, flags, phi, nx,
                                                                                             ny, nz, lo, hi, w3,
                                                                                             phi_min);
    }
    return cudaGetLastError();
}

}  // namespace lbm
