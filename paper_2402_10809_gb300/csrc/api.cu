// Host side of the C ABI declared in include/lbm.h: workspace layout, input
// validation, unit conversion (Table 1 scales), set-up and the launches of the
// fused step, moments and diagnostics kernels.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "lbm.h"
#include "setup.cuh"

namespace lbm {
cudaError_t launch_step_19_f32(int, const Params&, cudaStream_t);
cudaError_t launch_step_19_f16(int, const Params&, cudaStream_t);
cudaError_t launch_step_19_bf16(int, const Params&, cudaStream_t);
cudaError_t launch_step_27_f32(int, const Params&, cudaStream_t);
cudaError_t launch_step_27_f16(int, const Params&, cudaStream_t);
cudaError_t launch_step_27_bf16(int, const Params&, cudaStream_t);
cudaError_t launch_wall_shear(int q, int storage, const Params& P, float* out, int compact, cudaStream_t s);
cudaError_t launch_setup_aniso(const Params& P, const float* S, long long N, float* out, uint32_t* err, cudaStream_t s);
cudaError_t launch_adjoint_19_f32(int, const AdjParams&, cudaStream_t);
cudaError_t launch_adjoint_19_f16(int, const AdjParams&, cudaStream_t);
cudaError_t launch_adjoint_19_bf16(int, const AdjParams&, cudaStream_t);
cudaError_t launch_adjoint_27_f32(int, const AdjParams&, cudaStream_t);
cudaError_t launch_adjoint_27_f16(int, const AdjParams&, cudaStream_t);
cudaError_t launch_adjoint_27_bf16(int, const AdjParams&, cudaStream_t);
}  // namespace lbm

using namespace lbm;

namespace {

constexpr uint64_t kStateMagic = 0x324d425356414e45ull;  // checkpoint header tag (packed layout)
constexpr size_t kHeader = 256;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t elem_size(int storage) { return storage == LBM_F32 ? 4 : 2; }

// Workspace layout.  The fixed part depends on the box only; the slot part on
// the number of slots of the packed layout (lbm_list_length).
struct Layout {
    size_t flags, phi_dense, region, xmin, ext, rowbase, rownb, err, diag_out, fixed_end;
    size_t rows, mask, omega, phi, bnd_prof, bnd_nbmask, general, partials, staging, f[2], end;
};

bool grid_ok(const lbm_grid* g)
{
    if (!g) return false;
    if (g->q != 19 && g->q != 27) return false;
    if (g->storage < LBM_F32 || g->storage > LBM_BF16DEV) return false;
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a)
        if (n[a] < 2 || n[a] > 1024) return false;
    return true;
}

Layout layout(const lbm_grid* g, long long n_store)
{
    Layout L{};
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    const size_t nrows = (size_t)g->ny * g->nz;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.flags = take(N);
    L.phi_dense = take(N * 4);
    L.region = take(N);
    L.xmin = take(nrows * 4);
    L.ext = take(nrows * 4);
    L.rowbase = take(nrows * 4);
    L.rownb = take(nrows * 48);
    L.err = take(32);
    L.diag_out = take(8 * 8);
    L.fixed_end = o;
    const size_t n = (size_t)(n_store > 0 ? n_store : 1);
    L.rows = take(n * 4);
    L.mask = take(n * 4);
    L.omega = take(n * 4);
    L.phi = take(n * 4);
    L.bnd_prof = take(n * 4);
    L.bnd_nbmask = take(n * 4);
    L.general = take(n * 4);
    L.partials = take(((n + 31) / 32 + (n + kBlock - 1) / kBlock + 1) * kDiagSlots * 8);  // general + lean blocks
    L.staging = take(n * 6 * 4);
    const size_t fb = (size_t)g->q * n * elem_size(g->storage);
    L.f[0] = take(fb);
    L.f[1] = take(fb);
    L.end = o;
    return L;
}

cudaError_t launch(const lbm_grid& g, int mode, const Params& P, cudaStream_t s)
{
    if (g.q == 19) {
        if (g.storage == LBM_F32) return launch_step_19_f32(mode, P, s);
        if (g.storage == LBM_F16DEV) return launch_step_19_f16(mode, P, s);
        return launch_step_19_bf16(mode, P, s);
    }
    if (g.storage == LBM_F32) return launch_step_27_f32(mode, P, s);
    if (g.storage == LBM_F16DEV) return launch_step_27_f16(mode, P, s);
    return launch_step_27_bf16(mode, P, s);
}

// Spans of the non-solid cells of every row (host form of setup_rows).
long long host_spans(const lbm_grid* g, const uint8_t* flags, std::vector<int>* xmin, std::vector<int>* ext)
{
    const long long nx = g->nx, nrows = (long long)g->ny * g->nz;
    long long total = 0;
    if (xmin) xmin->assign(nrows, 0);
    if (ext) ext->assign(nrows, 0);
    for (long long r = 0; r < nrows; ++r) {
        const uint8_t* row = flags + r * nx;
        long long lo = -1, hi = -1;
        for (long long x = 0; x < nx; ++x) {
            if (row[x] >= 1 && row[x] <= 3) {
                if (lo < 0) lo = x;
                hi = x;
            }
        }
        if (lo >= 0) {
            total += hi - lo + 1;
            if (xmin) (*xmin)[r] = (int)lo;
            if (ext) (*ext)[r] = (int)(hi - lo + 1);
        }
    }
    return total;
}

}  // namespace

struct lbm_ctx {
    lbm_grid grid{};
    lbm_rheology rheo{};
    lbm_porous por{};
    lbm_bc bc{};
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    Layout L{};
    long long N = 0;
    int n_store = 0;                  // slots of the packed layout
    int n_ghost = 0;                  // ghost slots among them
    int n_in = 0, n_out = 0;
    int cur = 0;
    long long t = 0;
    int check_every = 0;
    bool ready = false;  // set once lbm_init has fully succeeded
    long long since_check = 0;
    float omega0 = 1.0f;
    Params base{};
    std::vector<long long> host_idx;  // dense index of each slot, -1 for ghost slots
    std::vector<uint32_t> out_slots;  // slots of the outlet cells
    std::vector<uint32_t> general;    // slots of the general-path cells
    std::vector<long long> plane_first;  // [nz + 1] first slot of each z-plane (contiguous per plane)
    int halo_lo = 0, halo_hi = 0;     // halo planes of a z-slab (lbm_set_halo)
    std::vector<uint32_t> halo_masks;    // the masks the halo planes had before they became halos
    std::vector<uint32_t> all_general;   // the general list without halo planes removed
    long long l2_group = 0;           // contexts of one nonzero group share the persisting L2 without resets
    // CUDA graphs of kGraphSteps time steps (problems without a velocity
    // inlet, whose steps do not depend on the time), one per starting buffer,
    // valid while params_gen is the generation they were captured at
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    unsigned long long graph_gen[2] = {0, 0};
    unsigned long long params_gen = 1;
    cudaStream_t capture_stream = nullptr;
    bool graphs_ok = true;
    std::string err;

    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
    void* f(int k) const { return ws + L.f[k]; }
};

static lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

static lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where)
{
    return fail(c, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(call, where)                    \
    do {                                         \
        cudaError_t e_ = (call);                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

// The L2 residency window of the step launches: the per-slot words (row id,
// mask, omega, porosity), which every step reads and which lie back to back
// in the workspace.  At most `cap` bytes of them (a quarter of the L2 by
// default: more would take the L2 from the streaming populations); the
// process's persisting-L2 limit (a per-process CUDA limit) is raised to hold
// the window, never lowered; the hit ratio covers what the limit allows.
// Devices without persisting L2 get no window.
static cudaError_t l2_window(lbm_ctx* c, long long cap)
{
    ++c->params_gen;
    Params& P = c->base;
    P.l2_base = nullptr;
    P.l2_bytes = 0;
    P.l2_hit = 0.0f;
    if (cap == 0 || c->n_store == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int max_persist = 0, max_window = 0, l2 = 0;
    e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    if (e != cudaSuccess) return e;
    if (max_persist <= 0 || max_window <= 0) return cudaSuccess;
    if (cap < 0) cap = l2 / 4;
    size_t win = c->L.bnd_prof - c->L.rows;
    if (win > (size_t)cap) win = (size_t)cap;
    if (win > (size_t)max_window) win = (size_t)max_window;
    size_t cur = 0;
    e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    if (e != cudaSuccess) return e;
    const size_t lim = win < (size_t)max_persist ? win : (size_t)max_persist;
    if (cur < lim) {
        e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, lim);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
        if (e != cudaSuccess) return e;
    }
    P.l2_base = c->ws + c->L.rows;
    P.l2_bytes = win;
    P.l2_hit = (float)((double)(cur < win ? cur : win) / (double)win);
    return cudaSuccess;
}

// The context whose window last claimed the persisting part of L2, per
// device.  When another context starts stepping, the persisting lines of the
// previous one are returned to normal (cudaCtxResetPersistingL2Cache), so that
// a context's window never competes with stale lines of another.
static constexpr int kL2Devices = 64;
static const lbm_ctx* g_l2_owner[kL2Devices] = {};

static cudaError_t l2_claim(const lbm_ctx* c)
{
    if (c->base.l2_bytes == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kL2Devices) return e;
    if (g_l2_owner[dev] == c) return cudaSuccess;
    const lbm_ctx* o = g_l2_owner[dev];
    if (o && c->l2_group != 0 && o->l2_group == c->l2_group) {
        // the slabs of one problem: their windows together stay within the
        // persisting limit, so the lines of the others may stay
        g_l2_owner[dev] = c;
        return cudaSuccess;
    }
    e = cudaCtxResetPersistingL2Cache();
    if (e == cudaSuccess) g_l2_owner[dev] = c;
    return e;
}

static void l2_release(const lbm_ctx* c)
{
    for (int d = 0; d < kL2Devices; ++d) {
        if (g_l2_owner[d] == c) {
            int cur = -1;
            if (cudaGetDevice(&cur) == cudaSuccess && cur == d) cudaCtxResetPersistingL2Cache();
            g_l2_owner[d] = nullptr;
        }
    }
}

extern "C" size_t lbm_workspace_size(const lbm_grid* grid, int64_t n_list)
{
    if (!grid_ok(grid)) return 0;
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    return layout(grid, n_list < 0 ? N : (n_list > N ? N : n_list)).end;
}

// Host mirror of the set-up's layout: the total length of the row spans.
extern "C" int64_t lbm_list_length(const lbm_grid* grid, const uint8_t* flags)
{
    if (!grid_ok(grid) || !flags) return -1;
    return host_spans(grid, flags, nullptr, nullptr);
}

// Dense index of every slot (-1 for ghost slots), for the calls that scatter
// per-slot results to a host array; built from the device's row ids and masks
// on first use.
static lbm_status ensure_host_idx(lbm_ctx* c)
{
    if ((int)c->host_idx.size() == c->n_store) return LBM_OK;
    const size_t n = (size_t)c->n_store;
    std::vector<uint32_t> hm(n), hr(n);
    std::vector<int> rb((size_t)c->grid.ny * c->grid.nz);
    if (n > 0) {
        LBM_CUDA(cudaMemcpyAsync(hm.data(), c->at<uint32_t>(c->L.mask), n * 4, cudaMemcpyDeviceToHost, c->stream),
                 "copy masks");
        LBM_CUDA(cudaMemcpyAsync(hr.data(), c->at<uint32_t>(c->L.rows), n * 4, cudaMemcpyDeviceToHost, c->stream),
                 "copy row ids");
        LBM_CUDA(cudaMemcpyAsync(rb.data(), c->at<int>(c->L.rowbase), rb.size() * 4, cudaMemcpyDeviceToHost,
                                 c->stream), "copy row bases");
        LBM_CUDA(cudaStreamSynchronize(c->stream), "copy sync");
    }
    std::vector<long long> idx(n, -1);
    for (size_t p = 0; p < n; ++p) {
        if (hm[p] & kGhostBit) continue;
        const uint32_t r = hr[p];
        idx[p] = (long long)((long long)p - rb[r]) + (long long)c->grid.nx * r;
    }
    c->host_idx.swap(idx);
    return LBM_OK;
}

static lbm_status run_diag(lbm_ctx* c, const uint8_t* region_dev, double out[8])
{
    Params P = c->base;
    P.fsrc = c->f(c->cur);
    P.fdst = nullptr;
    P.t = c->t;
    P.region = region_dev;
    P.partials = c->at<double>(c->L.partials);
    LBM_CUDA(launch(c->grid, kModeDiag, P, c->stream), "diag kernel");
    const int nblk = total_blocks(P);
    double* dout = c->at<double>(c->L.diag_out);
    if (nblk > 0) {
        LBM_CUDA(launch_diag_finish(P.partials, nblk, dout, c->stream), "diag reduction");
        LBM_CUDA(cudaMemcpyAsync(out, dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "diag copy");
        LBM_CUDA(cudaStreamSynchronize(c->stream), "diag sync");
    } else {
        for (int k = 0; k < 8; ++k) out[k] = 0.0;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_init(lbm_ctx** out, const lbm_grid* grid, const uint8_t* flags, const float* porosity,
                               int32_t inputs_on_device, const lbm_rheology* rheo, const lbm_porous* por,
                               const lbm_bc* bc, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    *out = c;
    if (!grid_ok(grid)) return fail(c, LBM_EINVAL, "grid: q must be 19 or 27, storage 0..2, sizes 2..1024");
    if (!flags || !porosity || !rheo || !por || !bc || !workspace)
        return fail(c, LBM_EINVAL, "null input pointer");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(c, LBM_EINVAL, "workspace not 256-byte aligned");
    if (!(rheo->mu0 > 0 && rheo->mu_inf > 0 && rheo->rho0 > 0 && rheo->dx > 0 && rheo->dt > 0 && rheo->a > 0 &&
          rheo->lambda >= 0))
        return fail(c, LBM_EINVAL, "rheology: mu0, mu_inf, rho0, dx, dt, a must be > 0 and lambda >= 0");
    if (!(por->k_const > 0) && !(por->d_p > 0)) return fail(c, LBM_EINVAL, "porous: d_p must be > 0 (or k_const > 0)");
    if (bc->inlet_axis < -1 || bc->inlet_axis > 2 || bc->outlet_axis < -1 || bc->outlet_axis > 2)
        return fail(c, LBM_EINVAL, "bc: axes must be -1, 0, 1 or 2");
    if (bc->inlet_axis >= 0 && !(bc->period > 0 && bc->inlet_radius > 0))
        return fail(c, LBM_EINVAL, "bc: inlet needs period > 0 and inlet_radius > 0");
    if (bc->outlet_axis >= 0 && !(bc->rho_out > 0)) return fail(c, LBM_EINVAL, "bc: rho_out must be > 0");
    c->grid = *grid;
    c->rheo = *rheo;
    c->por = *por;
    c->bc = *bc;
    c->stream = static_cast<cudaStream_t>(stream);
    c->ws = static_cast<char*>(workspace);
    c->ws_bytes = workspace_bytes;
    c->N = (long long)grid->nx * grid->ny * grid->nz;
    c->L = layout(grid, 0);
    if (workspace_bytes < c->L.fixed_end)
        return fail(c, LBM_ENOMEM, "workspace smaller than lbm_workspace_size(grid, 0)");
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    const int nrows = ny * nz;

    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LBM_CUDA(cudaMemcpyAsync(c->at<uint8_t>(c->L.flags), flags, (size_t)c->N, kind, c->stream), "copy flags");
    LBM_CUDA(cudaMemcpyAsync(c->at<float>(c->L.phi_dense), porosity, (size_t)c->N * 4, kind, c->stream),
             "copy porosity");
    uint32_t* errw = c->at<uint32_t>(c->L.err);
    LBM_CUDA(cudaMemsetAsync(errw, 0, 32, c->stream), "clear error words");

    // row spans (device), scanned on the host into the row bases
    LBM_CUDA(launch_setup_rows(c->at<uint8_t>(c->L.flags), nx, nrows, c->at<int>(c->L.xmin), c->at<int>(c->L.ext),
                               errw, c->stream),
             "setup_rows");
    std::vector<int> xmin(nrows), ext(nrows);
    uint32_t err0 = 0;
    LBM_CUDA(cudaMemcpyAsync(xmin.data(), c->at<int>(c->L.xmin), (size_t)nrows * 4, cudaMemcpyDeviceToHost, c->stream),
             "copy spans");
    LBM_CUDA(cudaMemcpyAsync(ext.data(), c->at<int>(c->L.ext), (size_t)nrows * 4, cudaMemcpyDeviceToHost, c->stream),
             "copy spans");
    LBM_CUDA(cudaMemcpyAsync(&err0, errw, 4, cudaMemcpyDeviceToHost, c->stream), "copy error word");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "setup sync");
    if (err0 & kErrFlag) return fail(c, LBM_EINVAL, "flags must be 0 (solid), 1 (fluid), 2 (inlet) or 3 (outlet)");
    long long total = 0;
    std::vector<int> rowbase(nrows, 0);
    for (int r = 0; r < nrows; ++r) {
        if (ext[r] > 0) {
            if (total - xmin[r] < INT32_MIN || total + nx > INT32_MAX)
                return fail(c, LBM_EINVAL, "too many non-solid cells for 32-bit slot indices");
            rowbase[r] = (int)(total - xmin[r]);
        }
        total += ext[r];
    }
    c->n_store = (int)total;
    c->plane_first.assign((size_t)nz + 1, 0);
    for (int z = 0; z < nz; ++z) {
        long long cnt = 0;
        for (int y = 0; y < ny; ++y) cnt += ext[y + ny * z];
        c->plane_first[z + 1] = c->plane_first[z] + cnt;
    }
    c->halo_lo = c->halo_hi = 0;
    c->L = layout(grid, c->n_store);
    if (workspace_bytes < c->L.end)
        return fail(c, LBM_ENOMEM, "workspace smaller than lbm_workspace_size(grid, " + std::to_string(c->n_store) +
                                       "), the packed length of these flags");
    // per row: the bases of its nine neighbour rows, wrapped on periodic axes
    // (0 outside the box: those links are never pulled), then y, z (device)
    LBM_CUDA(cudaMemcpyAsync(c->at<int>(c->L.rowbase), rowbase.data(), (size_t)nrows * 4, cudaMemcpyHostToDevice,
                             c->stream), "copy row bases");
    LBM_CUDA(launch_setup_rownb(c->at<int>(c->L.rowbase), ny, nz, grid->periodic[1] ? 1 : 0,
                                grid->periodic[2] ? 1 : 0, c->at<int>(c->L.rownb), c->stream),
             "setup_rownb");
    LBM_CUDA(launch_setup_slots(c->at<float>(c->L.phi_dense), nx, nrows, c->at<int>(c->L.rowbase),
                                c->at<int>(c->L.xmin), c->at<int>(c->L.ext), c->at<uint32_t>(c->L.rows),
                                c->at<float>(c->L.phi), c->stream),
             "setup_slots");

    SetupParams S{};
    S.nx = nx;
    S.ny = ny;
    S.nz = nz;
    for (int a = 0; a < 3; ++a) S.periodic[a] = grid->periodic[a] ? 1 : 0;
    S.n_store = c->n_store;
    S.flags = c->at<uint8_t>(c->L.flags);
    S.phi = c->at<float>(c->L.phi_dense);
    S.rows = c->at<uint32_t>(c->L.rows);
    S.rowbase = c->at<int>(c->L.rowbase);
    S.mask = c->at<uint32_t>(c->L.mask);
    S.bnd_prof = c->at<float>(c->L.bnd_prof);
    S.bnd_nbmask = c->at<uint32_t>(c->L.bnd_nbmask);
    S.in_axis = bc->inlet_axis;
    S.in_side = bc->inlet_side;
    S.out_axis = bc->outlet_axis;
    S.out_side = bc->outlet_side;
    for (int a = 0; a < 3; ++a) S.in_center[a] = bc->inlet_center[a];
    S.in_radius = bc->inlet_radius;
    S.err = errw;
    LBM_CUDA(launch_setup_mask(grid->q, S, c->stream), "setup_mask");
    // slot classes per chunk of slots (device), for the host tables below;
    // the staging area is free until the first host-output call
    const bool wide = (unsigned long long)grid->q * (unsigned long long)c->n_store >= (1ull << 32);
    const int nch = classify_chunks(c->n_store);
    int4* cls_d = c->at<int4>(c->L.staging);
    int2* off_d = reinterpret_cast<int2*>(cls_d + nch);
    uint32_t* outl_d = reinterpret_cast<uint32_t*>(off_d + nch);
    LBM_CUDA(launch_classify_count(S.mask, c->n_store, wide ? 1 : 0, cls_d, c->stream), "classify slots");
    std::vector<int4> cls(nch);
    uint32_t errv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    LBM_CUDA(cudaMemcpyAsync(errv, errw, 32, cudaMemcpyDeviceToHost, c->stream), "copy error words");
    if (nch > 0)
        LBM_CUDA(cudaMemcpyAsync(cls.data(), cls_d, (size_t)nch * sizeof(int4), cudaMemcpyDeviceToHost, c->stream),
                 "copy slot classes");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "setup sync");
    if (errv[0]) {
        float bad_phi;
        std::memcpy(&bad_phi, &errv[3], 4);
        char where[256];
        const uint32_t why = errv[4];
        std::snprintf(where, sizeof(where), " (first at cell x=%u y=%u z=%u, porosity %.9g%s%s%s%s)",
                      errv[2] & 1023u, (errv[2] >> 10) & 1023u, errv[2] >> 20, (double)bad_phi,
                      (why & 1u) ? "; no inlet axis" : "", (why & 2u) ? "; inlet axis is periodic" : "",
                      (why & 4u) ? "; not on the inlet face" : "", (why & 8u) ? "; porosity is not 1" : "");
        if (errv[0] & kErrPorosity)
            return fail(c, LBM_EINVAL, std::string("porosity must lie in (0, 1] on every non-solid cell") + where);
        if (errv[0] & kErrInlet)
            return fail(c, LBM_EINVAL,
                        std::string("inlet cells must lie on the inlet face, with an inlet configured and porosity 1") +
                            where);
        return fail(c, LBM_EINVAL,
                    std::string("outlet cells must lie on the outlet face with porosity 1 and a fluid interior "
                                "neighbour of porosity 1") + where);
    }
    // host tables: ghost count, outlet slots, general list (the dense index of
    // every slot is built on the first call that scatters to host memory)
    c->host_idx.clear();
    c->n_ghost = 0;
    c->n_in = 0;
    std::vector<int2> off(nch);
    int ngen = 0, nout = 0;
    for (int k = 0; k < nch; ++k) {
        off[k] = make_int2(ngen, nout);
        ngen += cls[k].x;
        nout += cls[k].y;
        c->n_ghost += cls[k].z;
        c->n_in += cls[k].w;
    }
    c->general.assign((size_t)ngen, 0u);
    c->out_slots.assign((size_t)nout, 0u);
    if (nch > 0 && (ngen > 0 || nout > 0)) {
        LBM_CUDA(cudaMemcpyAsync(off_d, off.data(), (size_t)nch * sizeof(int2), cudaMemcpyHostToDevice, c->stream),
                 "copy class offsets");
        LBM_CUDA(launch_classify_write(S.mask, c->n_store, wide ? 1 : 0, off_d, c->at<uint32_t>(c->L.general),
                                       outl_d, c->stream),
                 "list general and outlet slots");
        if (ngen > 0)
            LBM_CUDA(cudaMemcpyAsync(c->general.data(), c->at<uint32_t>(c->L.general), (size_t)ngen * 4,
                                     cudaMemcpyDeviceToHost, c->stream), "copy general list");
        if (nout > 0)
            LBM_CUDA(cudaMemcpyAsync(c->out_slots.data(), outl_d, (size_t)nout * 4, cudaMemcpyDeviceToHost,
                                     c->stream), "copy outlet list");
        LBM_CUDA(cudaStreamSynchronize(c->stream), "slot lists sync");
    }
    c->n_out = (int)c->out_slots.size();
    c->all_general = c->general;
    c->halo_masks.clear();

    // Lattice units from the Table 1 scales (Sec. 4): nu = mu / rho0 * dt / dx^2.
    const double scale = rheo->dt / (rheo->dx * rheo->dx);
    const double mu0 = rheo->mu0 / rheo->rho0 * scale;
    const double mui = rheo->mu_inf / rheo->rho0 * scale;
    const double nu_d = por->nu_darcy > 0 ? por->nu_darcy * scale : mu0;  // nu = mu0 / rho0 (Sec. 4)
    Params& P = c->base;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.N = c->N;
    P.n_store = c->n_store;
    // the lean path indexes the distribution buffers with 32-bit element
    // offsets; larger layouts run every cell through the general path
    P.wide = wide ? 1 : 0;
    P.n_general = (int)c->general.size();
    // general cells per block: one warp's worth while the lean grid is under
    // about four waves of LBM_MIN_BLOCKS blocks on 152 SMs, full blocks beyond
    P.gen_block = (c->n_store + kBlock - 1) / kBlock < 4 * LBM_MIN_BLOCKS * 152 ? 32 : kBlock;
    P.general = c->at<uint32_t>(c->L.general);
    P.rows = S.rows;
    P.rownb = c->at<int4>(c->L.rownb);
    P.rowbase = S.rowbase;
    P.mask = S.mask;
    P.phi = c->at<float>(c->L.phi);
    P.bnd_prof = S.bnd_prof;
    P.bnd_nbmask = S.bnd_nbmask;
    P.gx = (float)bc->body_force[0];
    P.gy = (float)bc->body_force[1];
    P.gz = (float)bc->body_force[2];
    if (por->k_const > 0) {
        const double kc = por->k_const / (rheo->dx * rheo->dx);
        P.drag_kc = 0;
        P.drag_a = (float)(nu_d / kc);
        P.drag_b = por->forchheimer ? (float)(1.75 / std::sqrt(150.0 * kc)) : 0.0f;
    } else {
        const double d = por->d_p / rheo->dx;
        P.drag_kc = 1;
        P.drag_a = (float)(150.0 * nu_d / (d * d));
        P.drag_b = por->forchheimer ? (float)(1.75 / d) : 0.0f;
    }
    P.mu0 = (float)mu0;
    P.mu_inf = (float)mui;
    P.lam = (float)(rheo->lambda / rheo->dt);
    P.cy_a = (float)rheo->a;
    P.cy_e = (float)((rheo->n - 1.0) / rheo->a);
    P.cy_a_two = rheo->a == 2.0 ? 1 : 0;
    P.in_axis = bc->inlet_axis;
    P.in_side = bc->inlet_side;
    P.out_axis = bc->outlet_axis;
    P.out_side = bc->outlet_side;
    P.u0 = bc->u0;
    P.amp = bc->amp;
    P.period = bc->period > 0 ? bc->period : 1.0;
    P.ramp = bc->ramp_steps;
    P.rho_out = (float)bc->rho_out;
    P.omega = c->at<float>(c->L.omega);
    c->omega0 = (float)(2.0 / (6.0 * mu0 + 1.0));  // omega(mu0) at rho = 1
    LBM_CUDA(l2_window(c, -1), "L2 residency window");

    // initial state: rest equilibrium (zero deviations)
    const size_t fb = (size_t)grid->q * c->n_store * elem_size(grid->storage);
    LBM_CUDA(cudaMemsetAsync(c->f(0), 0, fb, c->stream), "initial state");
    LBM_CUDA(launch_fill_f32(P.omega, c->n_store, c->omega0, c->stream), "initial omega");
    c->cur = 0;
    c->t = 0;
    c->ready = true;
    return LBM_OK;
}

// Time steps per captured graph (even: the state ends in the buffer it
// started from).
constexpr int kGraphSteps = 32;

// The graph of kGraphSteps time steps from the current buffer, captured on a
// private stream (capture does not run anything) the first time it is needed
// and again after any change of the step's parameters.  Without a velocity
// inlet no kernel reads the time, so one graph serves every later run.
// nullptr if capture or instantiation fails (the caller launches steps one
// by one from then on).
static cudaGraphExec_t step_graph(lbm_ctx* c)
{
    const int k = c->cur;
    if (c->graph[k] && c->graph_gen[k] == c->params_gen) return c->graph[k];
    if (c->graph[k]) {
        cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
    }
    if (!c->capture_stream && cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        c->graphs_ok = false;
        return nullptr;
    }
    if (cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        c->graphs_ok = false;
        return nullptr;
    }
    bool ok = true;
    int cur = k;
    for (int s = 0; s < kGraphSteps && ok; ++s) {
        Params P = c->base;
        P.fsrc = c->f(cur);
        P.fdst = c->f(1 - cur);
        P.t = 0;  // not read: no velocity inlet
        ok = launch(c->grid, kModeStep, P, c->capture_stream) == cudaSuccess;
        cur ^= 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
    cudaGraphExec_t x = nullptr;
    if (ok && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
        c->graph[k] = x;
        c->graph_gen[k] = c->params_gen;
    } else {
        (void)cudaGetLastError();
        c->graphs_ok = false;
    }
    if (g) cudaGraphDestroy(g);
    return c->graph[k];
}

extern "C" lbm_status lbm_step(lbm_ctx* c, int32_t n)
{
    if (!c) return LBM_EINVAL;
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    if (n > 0) LBM_CUDA(l2_claim(c), "claim the persisting L2");
    // problems without a velocity inlet run whole graphs of steps where the
    // steps up to the next instability check allow
    const bool graphs = c->graphs_ok && c->bc.inlet_axis < 0;
    for (int32_t s = 0; s < n;) {
        const long long to_check = c->check_every > 0 ? c->check_every - c->since_check : LLONG_MAX;
        cudaGraphExec_t x = (graphs && n - s >= kGraphSteps && to_check >= kGraphSteps) ? step_graph(c) : nullptr;
        if (x) {
            LBM_CUDA(cudaGraphLaunch(x, c->stream), "step graph");
            c->t += kGraphSteps;
            s += kGraphSteps;
            if (c->check_every > 0) c->since_check += kGraphSteps;
        } else {
            Params P = c->base;
            P.fsrc = c->f(c->cur);
            P.fdst = c->f(1 - c->cur);
            P.t = c->t;
            LBM_CUDA(launch(c->grid, kModeStep, P, c->stream), "step kernel");
            c->cur ^= 1;
            c->t += 1;
            s += 1;
            if (c->check_every > 0) c->since_check += 1;
        }
        if (c->check_every > 0 && c->since_check >= c->check_every) {
            c->since_check = 0;
            double d[8];
            lbm_status st = run_diag(c, nullptr, d);
            if (st != LBM_OK) return st;
            if (d[7] > 0) return fail(c, LBM_EUNSTABLE, "non-finite state at step " + std::to_string(c->t));
        }
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_moments(lbm_ctx* c, float* rho, float* u, float* shear_rate, float* omega,
                                  int32_t dst_on_device)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    Params P = c->base;
    P.fsrc = c->f(c->cur);
    P.fdst = nullptr;
    P.t = c->t;
    const size_t N = (size_t)c->N;
    if (dst_on_device) {
        float* outs[6] = {rho, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr, shear_rate, omega};
        for (float* o : outs)
            if (o) LBM_CUDA(cudaMemsetAsync(o, 0, N * 4, c->stream), "clear moments");
        P.o_rho = outs[0];
        P.o_ux = outs[1];
        P.o_uy = outs[2];
        P.o_uz = outs[3];
        P.o_gdot = outs[4];
        P.o_omega = outs[5];
        P.o_compact = 0;
        return launch(c->grid, kModeMoments, P, c->stream) == cudaSuccess ? LBM_OK
                                                                          : fail(c, LBM_ECUDA, "moments kernel");
    }
    const size_t n = (size_t)c->n_store;
    float* st = c->at<float>(c->L.staging);
    P.o_rho = st;
    P.o_ux = st + n;
    P.o_uy = st + 2 * n;
    P.o_uz = st + 3 * n;
    P.o_gdot = st + 4 * n;
    P.o_omega = st + 5 * n;
    P.o_compact = 1;
    std::vector<float> h(6 * n);
    const lbm_status hs = ensure_host_idx(c);
    if (hs != LBM_OK) return hs;
    if (n > 0) {
        LBM_CUDA(launch(c->grid, kModeMoments, P, c->stream), "moments kernel");
        LBM_CUDA(cudaMemcpyAsync(h.data(), st, 6 * n * 4, cudaMemcpyDeviceToHost, c->stream), "moments copy");
    }
    LBM_CUDA(cudaStreamSynchronize(c->stream), "moments sync");
    float* outs[6] = {rho, u, u ? u + N : nullptr, u ? u + 2 * N : nullptr, shear_rate, omega};
    for (int k = 0; k < 6; ++k) {
        if (!outs[k]) continue;
        std::memset(outs[k], 0, N * 4);
        for (size_t p = 0; p < n; ++p)
            if (c->host_idx[p] >= 0) outs[k][c->host_idx[p]] = h[k * n + p];
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_diag(lbm_ctx* c, const uint8_t* region, int32_t region_on_device, double out[8])
{
    if (!c || !out) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    const uint8_t* reg = nullptr;
    if (region) {
        if (region_on_device) {
            reg = region;
        } else {
            LBM_CUDA(cudaMemcpyAsync(c->at<uint8_t>(c->L.region), region, (size_t)c->N, cudaMemcpyHostToDevice,
                                     c->stream), "copy region");
            reg = c->at<uint8_t>(c->L.region);
        }
    }
    return run_diag(c, reg, out);
}

extern "C" lbm_status lbm_wall_shear(lbm_ctx* c, float* wss, int32_t dst_on_device)
{
    if (!c || !wss) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    Params P = c->base;
    P.fsrc = c->f(c->cur);
    P.fdst = nullptr;
    P.t = c->t;
    const size_t N = (size_t)c->N;
    if (dst_on_device) {
        LBM_CUDA(cudaMemsetAsync(wss, 0, N * 4, c->stream), "clear wall shear");
        LBM_CUDA(launch_wall_shear(c->grid.q, c->grid.storage, P, wss, 0, c->stream), "wall shear kernel");
        return LBM_OK;
    }
    const size_t n = (size_t)c->n_store;
    float* st = c->at<float>(c->L.staging);
    std::vector<float> h(n);
    const lbm_status hs = ensure_host_idx(c);
    if (hs != LBM_OK) return hs;
    if (n > 0) {
        LBM_CUDA(cudaMemsetAsync(st, 0, n * 4, c->stream), "clear wall shear");
        LBM_CUDA(launch_wall_shear(c->grid.q, c->grid.storage, P, st, 1, c->stream), "wall shear kernel");
        LBM_CUDA(cudaMemcpyAsync(h.data(), st, n * 4, cudaMemcpyDeviceToHost, c->stream), "wall shear copy");
    }
    LBM_CUDA(cudaStreamSynchronize(c->stream), "wall shear sync");
    std::memset(wss, 0, N * 4);
    for (size_t p = 0; p < n; ++p)
        if (c->host_idx[p] >= 0) wss[c->host_idx[p]] = h[p];
    return LBM_OK;
}

extern "C" size_t lbm_anisotropy_buffer_size(const lbm_ctx* c)
{
    if (!c || !c->ready) return 0;
    return align256(12 * sizeof(float) * (size_t)c->n_store);
}

extern "C" lbm_status lbm_set_anisotropy(lbm_ctx* c, const float* shape, void* buffer, size_t bytes, int32_t max_iter,
                                         float tol)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    ++c->params_gen;  // the captured step graphs hold the old parameters
    if (!shape) {
        c->base.aniso = nullptr;
        return LBM_OK;
    }
    if (!buffer || reinterpret_cast<uintptr_t>(buffer) % 256 != 0)
        return fail(c, LBM_EINVAL, "anisotropy buffer null or not 256-byte aligned");
    if (bytes < lbm_anisotropy_buffer_size(c)) return fail(c, LBM_ENOMEM, "anisotropy buffer too small");
    if (max_iter < 1 || max_iter > 1000 || !(tol >= 0.0f && tol < 1.0f))
        return fail(c, LBM_EINVAL, "max_iter must be 1..1000 and 0 <= tol < 1");
    uint32_t* errw = c->at<uint32_t>(c->L.err) + 5;
    LBM_CUDA(cudaMemsetAsync(errw, 0, 4, c->stream), "clear error word");
    Params P = c->base;
    LBM_CUDA(launch_setup_aniso(P, shape, (long long)c->N, static_cast<float*>(buffer), errw, c->stream),
             "anisotropy set-up kernel");
    uint32_t e = 0;
    LBM_CUDA(cudaMemcpyAsync(&e, errw, 4, cudaMemcpyDeviceToHost, c->stream), "copy error word");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "anisotropy set-up sync");
    if (e) {
        c->base.aniso = nullptr;
        return fail(c, LBM_EINVAL, "shape tensor not finite or not positive definite at a cell with phi < 1");
    }
    c->base.aniso = static_cast<const float*>(buffer);
    c->base.aniso_iters = max_iter;
    c->base.aniso_tol = tol;
    return LBM_OK;
}

static bool porosity_dims_ok(int32_t nx, int32_t ny, int32_t nz)
{
    return nx >= 1 && ny >= 1 && nz >= 1 && nx <= kPorosityMaxNx && (long long)nx * ny * nz <= (1ll << 40);
}

extern "C" size_t lbm_porosity_workspace_size(int32_t nx, int32_t ny, int32_t nz)
{
    if (!porosity_dims_ok(nx, ny, nz)) return 0;
    const size_t N = (size_t)nx * ny * nz;
    return align256(N) + align256(2 * N);
}

extern "C" lbm_status lbm_porosity_average(int32_t nx, int32_t ny, int32_t nz, const uint8_t* wire,
                                           const uint8_t* flags, int32_t window, float phi_min, float* phi,
                                           void* workspace, size_t workspace_bytes, void* cuda_stream)
{
    if (!porosity_dims_ok(nx, ny, nz) || !wire || !phi || !workspace) return LBM_EINVAL;
    if (window < 1 || window > kPorosityMaxWindow || !(phi_min >= 0.0f && phi_min <= 1.0f)) return LBM_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return LBM_EINVAL;
    if (workspace_bytes < lbm_porosity_workspace_size(nx, ny, nz)) return LBM_ENOMEM;
    const size_t N = (size_t)nx * ny * nz;
    uint8_t* ws_x = static_cast<uint8_t*>(workspace);
    uint16_t* ws_y = reinterpret_cast<uint16_t*>(ws_x + align256(N));
    const cudaError_t e = launch_porosity_average(wire, flags, nx, ny, nz, window, phi_min, phi, ws_x, ws_y,
                                                  static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" lbm_status lbm_set_l2_window(lbm_ctx* c, int64_t max_bytes)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    LBM_CUDA(l2_window(c, max_bytes), "L2 residency window");
    return LBM_OK;
}

extern "C" int64_t lbm_l2_window_bytes(const lbm_ctx* c) { return c && c->ready ? (int64_t)c->base.l2_bytes : -1; }

extern "C" lbm_status lbm_set_l2_group(lbm_ctx* c, int64_t group)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    c->l2_group = group;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_check(lbm_ctx* c, int32_t check_every)
{
    if (!c) return LBM_EINVAL;
    if (check_every < 0) return fail(c, LBM_EINVAL, "check_every must be >= 0");
    c->check_every = check_every;
    c->since_check = 0;
    return LBM_OK;
}

namespace {
struct StateHeader {
    uint64_t magic;
    int64_t t;
    int64_t n_store;
    int32_t q, storage;
};
}  // namespace

// Checkpoint: header, then the distributions [Q][n_store] in the storage type
// and omega [n_store], both exactly as they sit in the workspace.
extern "C" size_t lbm_state_size(const lbm_ctx* c)
{
    if (!c || !c->ready) return 0;
    return kHeader + (size_t)c->n_store * ((size_t)c->grid.q * elem_size(c->grid.storage) + 4);
}

extern "C" lbm_status lbm_save(lbm_ctx* c, void* dst, size_t bytes, int32_t dst_on_device)
{
    if (!c || !dst) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    const size_t need = lbm_state_size(c);
    if (bytes < need) return fail(c, LBM_ENOMEM, "destination smaller than lbm_state_size");
    StateHeader h{kStateMagic, c->t, c->n_store, c->grid.q, c->grid.storage};
    const size_t fbytes = (size_t)c->n_store * c->grid.q * elem_size(c->grid.storage);
    const cudaMemcpyKind k = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    char* d = static_cast<char*>(dst);
    LBM_CUDA(cudaMemcpyAsync(d + kHeader, c->f(c->cur), fbytes, k, c->stream), "save state");
    LBM_CUDA(cudaMemcpyAsync(d + kHeader + fbytes, c->base.omega, (size_t)c->n_store * 4, k, c->stream), "save omega");
    if (dst_on_device)
        LBM_CUDA(cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream), "save header");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "save sync");
    if (!dst_on_device) std::memcpy(d, &h, sizeof(h));
    return LBM_OK;
}

extern "C" lbm_status lbm_load(lbm_ctx* c, const void* src, size_t bytes, int32_t src_on_device)
{
    if (!c || !src) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    const size_t need = lbm_state_size(c);
    if (bytes < need) return fail(c, LBM_EINVAL, "source smaller than lbm_state_size");
    StateHeader h{};
    const char* s = static_cast<const char*>(src);
    if (src_on_device) {
        LBM_CUDA(cudaMemcpyAsync(&h, s, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "load header");
        LBM_CUDA(cudaStreamSynchronize(c->stream), "load sync");
    } else {
        std::memcpy(&h, s, sizeof(h));
    }
    if (h.magic != kStateMagic || h.n_store != c->n_store || h.q != c->grid.q || h.storage != c->grid.storage)
        return fail(c, LBM_EINVAL, "checkpoint does not match this context");
    const size_t fbytes = (size_t)c->n_store * c->grid.q * elem_size(c->grid.storage);
    const cudaMemcpyKind k = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LBM_CUDA(cudaMemcpyAsync(c->f(c->cur), s + kHeader, fbytes, k, c->stream), "load state");
    LBM_CUDA(cudaMemcpyAsync(c->base.omega, s + kHeader + fbytes, (size_t)c->n_store * 4, k, c->stream), "load omega");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "load sync");
    c->t = h.t;
    return LBM_OK;
}

extern "C" int64_t lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }
extern "C" int64_t lbm_fluid_count(const lbm_ctx* c) { return c ? c->n_store - c->n_ghost : -1; }
extern "C" const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }
extern "C" void lbm_destroy(lbm_ctx* c)
{
    if (c) {
        l2_release(c);
        for (cudaGraphExec_t& g : c->graph)
            if (g) cudaGraphExecDestroy(g);
        if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    }
    delete c;
}

// ---------------------------------------------------------------------------
// Discrete adjoint: d J / d phi of the sac kinetic-energy objective by a
// checkpointed reverse sweep (kernels in adjoint.cuh).
//
// Pass 1 runs the T forward steps from the rest state and keeps the state
// S(kK-1), omega(kK-1) and rho(kK-1) - 1 at the start of every segment k of K
// steps; the last segment writes all its states straight into the history
// slots.  The reverse sweep then visits the segments from last to first:
// it replays a segment from its checkpoint into the history slots (states,
// omega and the dense density deviation of every step), and runs the reverse steps
// t = e-1 .. s of the segment (after the objective-only step t = T for the
// last one).  Nothing is copied apart from the small omega arrays; every
// state buffer is written in place by the step kernel.
// ---------------------------------------------------------------------------
namespace {

struct AdjLayout {
    int nseg = 0, Kh = 0;  // segments; history slots H[1..Kh]
    size_t sbytes = 0, wbytes = 0, lbytes = 0;
    size_t ck = 0, hist = 0, wck = 0, whist = 0, rck = 0, rhist = 0, lam[2] = {0, 0};
    size_t mu = 0, gphi = 0, region = 0, jpart = 0, outs = 0, ord = 0, bdelta = 0, bdphi = 0, count = 0, end = 0;
};

AdjLayout adj_layout(const lbm_ctx* c, int T, int K)
{
    AdjLayout A;
    A.nseg = (T + K - 1) / K;
    A.Kh = K < T ? K : T;
    const size_t N = (size_t)c->N, Q = (size_t)c->grid.q;
    const size_t n = (size_t)(c->n_store > 0 ? c->n_store : 1);
    const size_t no = (size_t)(c->n_out > 0 ? c->n_out : 1);
    A.sbytes = align256(Q * n * elem_size(c->grid.storage));
    A.wbytes = align256(n * 4);
    A.lbytes = align256(Q * n * 4);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    A.ck = take((size_t)A.nseg * A.sbytes);
    A.hist = take((size_t)A.Kh * A.sbytes);
    A.wck = take((size_t)A.nseg * A.wbytes);
    A.whist = take((size_t)A.Kh * A.wbytes);
    A.rck = take((size_t)A.nseg * A.wbytes);
    A.rhist = take((size_t)A.Kh * A.wbytes);
    A.lam[0] = take(A.lbytes);
    A.lam[1] = take(A.lbytes);
    A.mu = take(n * 4);
    A.gphi = take(n * 8);
    A.region = take(N);
    A.jpart = take((size_t)(total_blocks(c->base) + 1) * (kBlock / 32) * 8);
    A.outs = take(no * 4);
    A.ord = take(n * 4);
    A.bdelta = take(Q * no * 4);
    A.bdphi = take(no * 8);
    A.count = take(8);
    A.end = o;
    return A;
}

cudaError_t launch_adj(const lbm_grid& g, int what, const AdjParams& A, cudaStream_t s)
{
    if (g.q == 19) {
        if (g.storage == LBM_F32) return launch_adjoint_19_f32(what, A, s);
        if (g.storage == LBM_F16DEV) return launch_adjoint_19_f16(what, A, s);
        return launch_adjoint_19_bf16(what, A, s);
    }
    if (g.storage == LBM_F32) return launch_adjoint_27_f32(what, A, s);
    if (g.storage == LBM_F16DEV) return launch_adjoint_27_f16(what, A, s);
    return launch_adjoint_27_bf16(what, A, s);
}

}  // namespace

extern "C" size_t lbm_adjoint_workspace_size(const lbm_ctx* c, int32_t T, int32_t K)
{
    if (!c || !c->ready || T < 1 || K < 1) return 0;
    return adj_layout(c, T, K).end;
}

extern "C" lbm_status lbm_adjoint(lbm_ctx* c, int32_t T, int32_t K, int32_t objective, const uint8_t* region,
                                  int32_t region_on_device, void* workspace, size_t workspace_bytes, double* grad,
                                  double* J)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    if (T < 1 || K < 1) return fail(c, LBM_EINVAL, "T and K must be >= 1");
    if (objective != 0 && objective != 1) return fail(c, LBM_EINVAL, "objective must be 0 (kinetic energy) or 1 (wall shear)");
    if (c->halo_lo || c->halo_hi) return fail(c, LBM_EINVAL, "the adjoint runs on a whole box, not on a z-slab");
    if (!region || !workspace || !grad || !J) return fail(c, LBM_EINVAL, "null pointer argument");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(c, LBM_EINVAL, "adjoint workspace not 256-byte aligned");
    const AdjLayout AL = adj_layout(c, T, K);
    if (workspace_bytes < AL.end) return fail(c, LBM_ENOMEM, "workspace smaller than lbm_adjoint_workspace_size");
    char* w = static_cast<char*>(workspace);
    const cudaStream_t st = c->stream;
    const size_t N = (size_t)c->N;
    const size_t n = (size_t)c->n_store;
    auto Cs = [&](int k) { return static_cast<void*>(w + AL.ck + (size_t)k * AL.sbytes); };
    auto Hs = [&](int j) { return static_cast<void*>(w + AL.hist + (size_t)(j - 1) * AL.sbytes); };
    auto Wc = [&](int k) { return reinterpret_cast<float*>(w + AL.wck + (size_t)k * AL.wbytes); };
    auto Wh = [&](int j) { return reinterpret_cast<float*>(w + AL.whist + (size_t)(j - 1) * AL.wbytes); };
    auto Rc = [&](int k) { return reinterpret_cast<float*>(w + AL.rck + (size_t)k * AL.wbytes); };
    auto Rh = [&](int j) { return reinterpret_cast<float*>(w + AL.rhist + (size_t)(j - 1) * AL.wbytes); };
    float* lam[2] = {reinterpret_cast<float*>(w + AL.lam[0]), reinterpret_cast<float*>(w + AL.lam[1])};
    float* mu = reinterpret_cast<float*>(w + AL.mu);
    double* gphi = reinterpret_cast<double*>(w + AL.gphi);
    uint8_t* reg = reinterpret_cast<uint8_t*>(w + AL.region);
    double* jpart = reinterpret_cast<double*>(w + AL.jpart);
    uint32_t* outs = reinterpret_cast<uint32_t*>(w + AL.outs);
    const Params B = c->base;

    LBM_CUDA(cudaMemcpyAsync(reg, region, N, region_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
             "copy region");
    if (c->n_out > 0)
        LBM_CUDA(cudaMemcpyAsync(outs, c->out_slots.data(), (size_t)c->n_out * 4, cudaMemcpyHostToDevice, st),
                 "copy outlet slots");
    unsigned long long* cnt_dev = reinterpret_cast<unsigned long long*>(w + AL.count);
    unsigned long long cnt = 0;
    // objective 1 averages over the region's plain fluid cells with a wall link
    const uint32_t wall_bits = objective == 1 ? ((1u << c->grid.q) - 2u) : 0u;
    LBM_CUDA(launch_region_count(B.rows, B.rowbase, B.mask, c->n_store, c->grid.nx, reg, wall_bits, cnt_dev, st),
             "region count");
    LBM_CUDA(cudaMemcpyAsync(&cnt, cnt_dev, sizeof(cnt), cudaMemcpyDeviceToHost, st), "copy region count");
    LBM_CUDA(cudaStreamSynchronize(st), "region count sync");
    if (cnt == 0)
        return fail(c, LBM_EINVAL, objective == 1 ? "the objective region holds no fluid cell next to a wall"
                                                  : "the objective region holds no fluid cell");
    const int nblk = total_blocks(B);
    LBM_CUDA(l2_claim(c), "claim the persisting L2");
    LBM_CUDA(cudaMemsetAsync(grad, 0, N * 8, st), "clear gradient");
    LBM_CUDA(cudaMemsetAsync(gphi, 0, n * 8, st), "clear packed gradient");
    LBM_CUDA(cudaMemsetAsync(Cs(0), 0, AL.sbytes, st), "rest state");
    const size_t nparts = (size_t)nblk * (kBlock / 32);
    LBM_CUDA(cudaMemsetAsync(jpart, 0, (nparts + 1) * 8, st), "clear objective partials");
    LBM_CUDA(launch_fill_f32(Wc(0), (long long)n, c->omega0, st), "initial omega");

    auto step = [&](long long t, const void* src, void* dst, float* om, float* drho) {
        Params P = B;
        P.fsrc = src;
        P.fdst = dst;
        P.omega = om;
        P.o_drho = drho;
        P.t = t;
        return launch(c->grid, kModeStep, P, st);
    };
    auto copy_omega = [&](float* dst, const float* src) {
        return n ? cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
    };

    // pass 1: forward with checkpoints
    const int nseg = AL.nseg, kl = nseg - 1;
    const void* src = Cs(0);
    float* wcur = Wc(0);
    for (int t = 0; t < T; ++t) {
        const int k = t / K;
        void* dst;
        float* wdst;
        float* rdst = nullptr;
        if (k + 1 < nseg && t == (k + 1) * K - 1) {
            dst = Cs(k + 1);
            wdst = Wc(k + 1);
            rdst = Rc(k + 1);
        } else if (k == kl) {
            const int j = t - k * K + 1;
            dst = Hs(j);
            wdst = Wh(j);
            rdst = Rh(j);
        } else {
            dst = lam[t & 1];
            wdst = mu;
        }
        if (wdst != wcur) LBM_CUDA(copy_omega(wdst, wcur), "omega copy");
        LBM_CUDA(step(t, src, dst, wdst, rdst), "adjoint forward step");
        src = dst;
        wcur = wdst;
    }

    // reverse sweep
    AdjParams A{};
    A.F = B;
    A.mu = mu;
    A.gphi = gphi;
    A.region = reg;
    A.kappa = (float)(1.0 / ((double)T * (double)cnt));
    A.obj_kind = objective;
    A.out_slots = outs;
    A.out_ord = reinterpret_cast<uint32_t*>(w + AL.ord);
    A.n_out = c->n_out;
    A.bnd_delta = reinterpret_cast<float*>(w + AL.bdelta);
    A.bnd_dphi = reinterpret_cast<double*>(w + AL.bdphi);
    A.jpart = jpart;
    LBM_CUDA(launch_adj(c->grid, 2, A, st), "outlet ordinals");
    int li = 0;  // lam[li] holds lambda(t), lam[1 - li] receives lambda(t-1)
    for (int k = kl; k >= 0; --k) {
        const int s = k * K;
        const int e = s + K < T ? s + K : T;
        auto Sat = [&](int j) { return j == 0 ? Cs(k) : Hs(j); };
        auto Wat = [&](int j) { return j == 0 ? Wc(k) : Wh(j); };
        auto Rat = [&](int j) { return j == 0 ? Rc(k) : Rh(j); };
        if (k < kl) {
            // replay: S(t), omega(t), rho(t) - 1 for t = s .. e-2 (S(e-1) is the next checkpoint)
            for (int t = s; t <= e - 2; ++t) {
                const int j = t - s + 1;
                LBM_CUDA(copy_omega(Wh(j), Wat(j - 1)), "omega copy");
                LBM_CUDA(step(t, Sat(j - 1), Hs(j), Wh(j), Rh(j)), "adjoint replay step");
            }
        }
        auto reverse = [&](int t, int first) {
            const int j = t - s;
            A.F.fsrc = Sat(j);
            A.F.omega = Wat(j);
            A.F.t = t;
            A.drho_prev = Rat(j);
            A.lam_in = lam[li];
            A.lam_out = lam[1 - li];
            A.first = first;
            A.objective = t >= 1;
            A.last = t == 0;
            cudaError_t e1 = launch_adj(c->grid, 0, A, st);
            if (e1 == cudaSuccess && c->n_out > 0) e1 = launch_adj(c->grid, 1, A, st);
            li = 1 - li;
            return e1;
        };
        if (k == kl) LBM_CUDA(reverse(T, 1), "adjoint objective step");
        for (int t = e - 1; t >= s; --t) LBM_CUDA(reverse(t, 0), "adjoint reverse step");
    }
    LBM_CUDA(launch_scatter_f64(B.rows, B.rowbase, B.mask, c->n_store, c->grid.nx, gphi, grad, st), "gradient scatter");
    std::vector<double> hp(nparts + 1, 0.0);
    if (nparts > 0)
        LBM_CUDA(cudaMemcpyAsync(hp.data(), jpart, nparts * 8, cudaMemcpyDeviceToHost, st), "copy objective");
    LBM_CUDA(cudaStreamSynchronize(st), "adjoint sync");
    double sum = 0.0;
    for (size_t b = 0; b < nparts; ++b) sum += hp[b];
    *J = sum;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// z-slab decomposition: one context per slab of z-planes plus one halo plane on
// each side that has a neighbour.  A step pulls across a slab face only the
// directions with c_z pointing into the slab, from the neighbour's plane next
// to the face; those populations are copied into the halo plane after every
// step (directly on one device, or packed for a message between processes).
// ---------------------------------------------------------------------------
namespace {

// Directions whose c_z equals cz, in increasing index order (the order of a
// packed halo message).
int dirs_with_cz(int q, int cz, int* out)
{
    int n = 0;
    for (int i = 0; i < q; ++i) {
        const int c = q == 19 ? Lattice<19>::cz(i) : Lattice<27>::cz(i);
        if (c == cz) out[n++] = i;
    }
    return n;
}

// Slots of every z-plane of a box (host form of the packed layout).
bool plane_counts(const lbm_grid* g, const uint8_t* flags, std::vector<long long>& cnt)
{
    std::vector<int> ext;
    host_spans(g, flags, nullptr, &ext);
    cnt.assign((size_t)g->nz, 0);
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y) cnt[z] += ext[(size_t)y + (size_t)g->ny * z];
    return true;
}

// The plane a side of the face sends (interior) and the plane it receives
// (halo), and the direction set of each.  side 0: the lower face, side 1: the
// upper face.
struct FaceSpec {
    int send_plane, recv_plane, send_cz, recv_cz;
};
FaceSpec face_of(const lbm_ctx* c, int side)
{
    const int nz = c->grid.nz;
    if (side == 0) return {c->halo_lo, 0, -1, +1};
    return {nz - 1 - c->halo_hi, nz - 1, +1, -1};
}

size_t elem_of(const lbm_ctx* c) { return elem_size(c->grid.storage); }

}  // namespace

extern "C" lbm_status lbm_plane_slots(const lbm_grid* grid, const uint8_t* flags, int32_t z, int64_t* first,
                                      int64_t* count)
{
    if (!grid_ok(grid) || !flags || !first || !count || z < 0 || z >= grid->nz) return LBM_EINVAL;
    std::vector<long long> cnt;
    plane_counts(grid, flags, cnt);
    long long f = 0;
    for (int k = 0; k < z; ++k) f += cnt[k];
    *first = f;
    *count = cnt[z];
    return LBM_OK;
}

extern "C" lbm_status lbm_slab_bounds(const lbm_grid* grid, const uint8_t* flags, int32_t nslabs, int32_t* z_bounds)
{
    if (!grid_ok(grid) || !flags || !z_bounds || nslabs < 1 || nslabs > grid->nz) return LBM_EINVAL;
    std::vector<long long> cnt;
    plane_counts(grid, flags, cnt);
    long long total = 0;
    for (long long v : cnt) total += v;
    // boundary k at the first plane whose cumulative slot count reaches k/nslabs
    // of the total, kept strictly increasing so that every slab owns a plane
    z_bounds[0] = 0;
    long long acc = 0;
    int z = 0;
    for (int k = 1; k < nslabs; ++k) {
        const long long target = (total * k + nslabs / 2) / nslabs;
        while (z < grid->nz && acc + cnt[z] <= target) acc += cnt[z++];
        int b = z;
        if (b <= z_bounds[k - 1]) b = z_bounds[k - 1] + 1;
        if (b > grid->nz - (nslabs - k)) b = grid->nz - (nslabs - k);
        while (z < b) acc += cnt[z++];
        z_bounds[k] = b;
    }
    z_bounds[nslabs] = grid->nz;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_halo(lbm_ctx* c, int32_t lo_planes, int32_t hi_planes)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    if (lo_planes < 0 || lo_planes > 1 || hi_planes < 0 || hi_planes > 1)
        return fail(c, LBM_EINVAL, "halo planes: 0 or 1 on each side");
    if (c->grid.nz - lo_planes - hi_planes < 1) return fail(c, LBM_EINVAL, "a slab needs an interior plane");
    if ((lo_planes || hi_planes) && c->grid.periodic[2])
        return fail(c, LBM_EINVAL, "halo planes need a box that is not periodic in z");
    // Halo slots become ghost slots without zero stores: every kernel skips
    // them, so the step neither updates them nor do moments and diagnostics
    // count them, at no cost to the cells.  The previous halo planes get their
    // masks back first.
    const int nz = c->grid.nz;
    uint32_t* mask = c->at<uint32_t>(c->L.mask);
    auto ranges = [&](int lo, int hi, long long r[2][2]) {
        r[0][0] = c->plane_first[0];
        r[0][1] = c->plane_first[lo];
        r[1][0] = c->plane_first[nz - hi];
        r[1][1] = c->plane_first[nz];
    };
    long long old_r[2][2], new_r[2][2];
    ranges(c->halo_lo, c->halo_hi, old_r);
    size_t at = 0;
    for (auto& r : old_r) {
        const size_t cnt = (size_t)(r[1] - r[0]);
        if (cnt)
            LBM_CUDA(cudaMemcpyAsync(mask + r[0], c->halo_masks.data() + at, cnt * 4, cudaMemcpyHostToDevice,
                                     c->stream), "restore halo masks");
        at += cnt;
    }
    LBM_CUDA(cudaStreamSynchronize(c->stream), "restore halo masks");
    ranges(lo_planes, hi_planes, new_r);
    c->halo_masks.assign((size_t)(new_r[0][1] - new_r[0][0] + new_r[1][1] - new_r[1][0]), 0u);
    at = 0;
    for (auto& r : new_r) {
        const size_t cnt = (size_t)(r[1] - r[0]);
        if (cnt) {
            LBM_CUDA(cudaMemcpyAsync(c->halo_masks.data() + at, mask + r[0], cnt * 4, cudaMemcpyDeviceToHost,
                                     c->stream), "save halo masks");
            LBM_CUDA(launch_fill_u32(mask + r[0], (long long)cnt, kGhostBit, c->stream), "mark halo slots");
        }
        at += cnt;
    }
    c->general.clear();
    for (uint32_t p : c->all_general)
        if (!((long long)p < new_r[0][1] || (long long)p >= new_r[1][0])) c->general.push_back(p);
    if (!c->general.empty())
        LBM_CUDA(cudaMemcpyAsync(c->at<uint32_t>(c->L.general), c->general.data(), c->general.size() * 4,
                                 cudaMemcpyHostToDevice, c->stream), "copy general list");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "halo set-up sync");
    c->base.n_general = (int)c->general.size();
    c->host_idx.clear();  // halo slots scatter nothing to host outputs
    ++c->params_gen;
    c->halo_lo = lo_planes;
    c->halo_hi = hi_planes;
    return LBM_OK;
}

extern "C" size_t lbm_halo_message_size(const lbm_ctx* c, int32_t side)
{
    if (!c || !c->ready || (side != 0 && side != 1)) return 0;
    if ((side == 0 && !c->halo_lo) || (side == 1 && !c->halo_hi)) return 0;
    const FaceSpec f = face_of(c, side);
    int d[27];
    const int nd = dirs_with_cz(c->grid.q, f.send_cz, d);
    return (size_t)nd * (size_t)(c->plane_first[f.send_plane + 1] - c->plane_first[f.send_plane]) * elem_of(c);
}

static lbm_status halo_pack_unpack(lbm_ctx* c, int side, void* dst, const void* src, bool pack)
{
    if (!c) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    if (side != 0 && side != 1) return fail(c, LBM_EINVAL, "side must be 0 (lower face) or 1 (upper face)");
    if ((side == 0 && !c->halo_lo) || (side == 1 && !c->halo_hi))
        return fail(c, LBM_EINVAL, "no halo plane on this side (lbm_set_halo)");
    if (pack ? !dst : !src) return fail(c, LBM_EINVAL, "null buffer");
    const FaceSpec f = face_of(c, side);
    const int plane = pack ? f.send_plane : f.recv_plane;
    int d[27];
    const int nd = dirs_with_cz(c->grid.q, pack ? f.send_cz : f.recv_cz, d);
    const long long first = c->plane_first[plane], count = c->plane_first[plane + 1] - first;
    const size_t es = elem_of(c), n = (size_t)c->n_store;
    char* state = static_cast<char*>(c->f(c->cur));
    HaloCopy H{};
    H.ntask = nd;
    H.elem = (int)es;
    for (int k = 0; k < nd; ++k) {
        char* slot = state + ((size_t)d[k] * n + (size_t)first) * es;
        H.count[k] = count;
        if (pack) {
            H.src[k] = slot;
            H.dst[k] = static_cast<char*>(dst) + (size_t)k * count * es;
        } else {
            H.src[k] = static_cast<const char*>(src) + (size_t)k * count * es;
            H.dst[k] = slot;
        }
    }
    LBM_CUDA(launch_halo_copy(H, c->stream), pack ? "halo pack" : "halo unpack");
    return LBM_OK;
}

extern "C" lbm_status lbm_halo_pack(lbm_ctx* c, int32_t side, void* dst)
{
    return halo_pack_unpack(c, side, dst, nullptr, true);
}

extern "C" lbm_status lbm_halo_unpack(lbm_ctx* c, int32_t side, const void* src)
{
    return halo_pack_unpack(c, side, nullptr, src, false);
}

static lbm_status halo_exchange_on(lbm_ctx* lower, lbm_ctx* upper, cudaStream_t s);

extern "C" lbm_status lbm_halo_exchange(lbm_ctx* lower, lbm_ctx* upper)
{
    if (!lower || !upper || lower == upper) return LBM_EINVAL;
    if (!lower->ready || !upper->ready) return fail(lower, LBM_ESTATE, "context not initialised");
    if (!lower->halo_hi || !upper->halo_lo)
        return fail(lower, LBM_EINVAL, "the lower slab needs an upper halo plane and the upper slab a lower one");
    if (lower->grid.q != upper->grid.q || lower->grid.storage != upper->grid.storage ||
        lower->grid.nx != upper->grid.nx || lower->grid.ny != upper->grid.ny)
        return fail(lower, LBM_EINVAL, "slabs of different lattices, storage types or x-y extents");
    if (lower->stream != upper->stream) return fail(lower, LBM_EINVAL, "the two slabs must share one stream");
    return halo_exchange_on(lower, upper, lower->stream);
}

// The copies of lbm_halo_exchange, launched on stream s (the caller orders
// them after both slabs' steps).
static lbm_status halo_exchange_on(lbm_ctx* lower, lbm_ctx* upper, cudaStream_t s)
{
    const FaceSpec fl = face_of(lower, 1), fu = face_of(upper, 0);
    const long long a = lower->plane_first[fl.send_plane + 1] - lower->plane_first[fl.send_plane];
    const long long b = upper->plane_first[fu.recv_plane + 1] - upper->plane_first[fu.recv_plane];
    const long long c2 = upper->plane_first[fu.send_plane + 1] - upper->plane_first[fu.send_plane];
    const long long d2 = lower->plane_first[fl.recv_plane + 1] - lower->plane_first[fl.recv_plane];
    if (a != b || c2 != d2)
        return fail(lower, LBM_EINVAL, "the planes at the face differ between the slabs (not adjacent slabs of one box)");
    const size_t es = elem_of(lower);
    const size_t nl = (size_t)lower->n_store, nu = (size_t)upper->n_store;
    char* sl = static_cast<char*>(lower->f(lower->cur));
    char* su = static_cast<char*>(upper->f(upper->cur));
    int up[27], dn[27];
    const int nup = dirs_with_cz(lower->grid.q, +1, up), ndn = dirs_with_cz(lower->grid.q, -1, dn);
    HaloCopy H{};
    H.elem = (int)es;
    for (int k = 0; k < nup; ++k) {  // lower's top interior plane -> upper's lower halo, c_z = +1
        H.src[H.ntask] = sl + ((size_t)up[k] * nl + (size_t)lower->plane_first[fl.send_plane]) * es;
        H.dst[H.ntask] = su + ((size_t)up[k] * nu + (size_t)upper->plane_first[fu.recv_plane]) * es;
        H.count[H.ntask++] = a;
    }
    for (int k = 0; k < ndn; ++k) {  // upper's first interior plane -> lower's upper halo, c_z = -1
        H.src[H.ntask] = su + ((size_t)dn[k] * nu + (size_t)upper->plane_first[fu.send_plane]) * es;
        H.dst[H.ntask] = sl + ((size_t)dn[k] * nl + (size_t)lower->plane_first[fl.recv_plane]) * es;
        H.count[H.ntask++] = c2;
    }
    const cudaError_t e = launch_halo_copy(H, s);
    return e == cudaSuccess ? LBM_OK : cuda_fail(lower, e, "halo exchange");
}

extern "C" lbm_status lbm_step_slabs(lbm_ctx** slabs, int32_t n, int32_t steps, void* join_stream)
{
    if (!slabs || n < 1 || steps < 0) return LBM_EINVAL;
    for (int k = 0; k < n; ++k) {
        if (!slabs[k]) return LBM_EINVAL;
        if (!slabs[k]->ready) return fail(slabs[k], LBM_ESTATE, "context not initialised");
    }
    for (int k = 0; k + 1 < n; ++k) {
        lbm_ctx* lo = slabs[k];
        lbm_ctx* up = slabs[k + 1];
        if (!lo->halo_hi || !up->halo_lo)
            return fail(lo, LBM_EINVAL, "the lower slab needs an upper halo plane and the upper slab a lower one");
        if (lo->grid.q != up->grid.q || lo->grid.storage != up->grid.storage || lo->grid.nx != up->grid.nx ||
            lo->grid.ny != up->grid.ny)
            return fail(lo, LBM_EINVAL, "slabs of different lattices, storage types or x-y extents");
    }
    if (steps == 0) return LBM_OK;
    lbm_ctx* c = slabs[0];  // errors of the events go to the first slab
    std::vector<cudaEvent_t> ev((size_t)2 * n + 1, nullptr);
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (cudaEvent_t& e : ev) {
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return fail(c, LBM_ECUDA, "event creation");
        }
    }
    cudaEvent_t* step_done = ev.data();        // [n]
    cudaEvent_t* exch_done = ev.data() + n;    // [n - 1] face k | k + 1
    cudaEvent_t start = ev[(size_t)2 * n];
    const cudaStream_t join = static_cast<cudaStream_t>(join_stream);
    lbm_status st = LBM_OK;
    auto check = [&](cudaError_t e, const char* where) {
        if (e != cudaSuccess && st == LBM_OK) st = cuda_fail(c, e, where);
        return st == LBM_OK;
    };
    // join_stream may be the legacy default stream (NULL): always join
    check(cudaEventRecord(start, join), "join");
    for (int k = 0; k < n && st == LBM_OK; ++k) check(cudaStreamWaitEvent(slabs[k]->stream, start, 0), "join");
    for (int t = 0; t < steps && st == LBM_OK; ++t) {
        // every slab steps on its own stream once the faces of the last
        // exchange that touched it are done
        for (int k = 0; k < n && st == LBM_OK; ++k) {
            if (t > 0 && k > 0 && !check(cudaStreamWaitEvent(slabs[k]->stream, exch_done[k - 1], 0), "wait")) break;
            if (t > 0 && k + 1 < n && !check(cudaStreamWaitEvent(slabs[k]->stream, exch_done[k], 0), "wait")) break;
            const lbm_status s1 = lbm_step(slabs[k], 1);
            if (s1 != LBM_OK) {
                if (slabs[k] != c) c->err = slabs[k]->err;
                st = s1;
                break;
            }
            check(cudaEventRecord(step_done[k], slabs[k]->stream), "record");
        }
        // then each face, on the lower slab's stream, after the upper slab's step
        for (int k = 0; k + 1 < n && st == LBM_OK; ++k) {
            if (!check(cudaStreamWaitEvent(slabs[k]->stream, step_done[k + 1], 0), "wait")) break;
            const lbm_status s2 = halo_exchange_on(slabs[k], slabs[k + 1], slabs[k]->stream);
            if (s2 != LBM_OK) {
                if (slabs[k] != c) c->err = slabs[k]->err;
                st = s2;
                break;
            }
            check(cudaEventRecord(exch_done[k], slabs[k]->stream), "record");
        }
    }
    for (int k = 0; k < n; ++k) {
        // the slabs' last work, whatever happened above, before the join stream's next
        if (cudaEventRecord(step_done[k], slabs[k]->stream) == cudaSuccess) cudaStreamWaitEvent(join, step_done[k], 0);
    }
    cleanup();
    return st;
}

// ---------------------------------------------------------------------------
// Diagnostics without any caller-provided scratch.
//
// lbm_diag reduces into per-block partial sums kept in the caller's workspace.
// lbm_diag_noalloc computes the same numbers with the same kernels, but keeps
// those partial sums and the device-side result in the fixed array below, so it
// needs no scratch from the caller and never allocates.  It serves callers that
// may not allocate device memory at the point of the call: a monitoring thread
// attached to a running simulation whose allocator belongs to another framework,
// or code running where allocation is forbidden or unsafe.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds kNoAllocBytes for it until the process exits.  Its device
// address is looked up with cudaGetSymbolAddress on every call made outside
// stream capture (the name in host code is only a host-side stand-in and must
// never be handed to a kernel); calls during a capture reuse the address of
// the last uncaptured call on the device, so make the first call on a device
// before any stream capture begins.  All calls share the one
// array: calls that overlap on the GPU (other streams, other threads) race and
// must be serialised by the caller.  Every slot a call reads is written earlier
// in the same call, so leftover contents of a previous call do no harm.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr long long kNoAllocMaxCells = 8LL * 1024 * 1024;  // slots of the packed layout
// lean blocks for kNoAllocMaxCells slots plus up to 32768 blocks of general-path cells
constexpr long long kNoAllocMaxBlocks = kNoAllocMaxCells / kBlock + 32768;
constexpr size_t kNoAllocSlots = (size_t)(kNoAllocMaxBlocks + 1) * kDiagSlots + 8;  // partials + result
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  Looked up on
// every call whose stream is not capturing (the module may be reloaded at
// another address after a device reset); a capturing stream reuses the address
// of the last uncaptured call on this device, so the first call on a device
// must come before any capture.
cudaError_t noalloc_scratch(int dev, cudaStream_t s, double** out)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    } else if (!g_noalloc_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_diag_noalloc(lbm_ctx* c, const uint8_t* region, double out[8])
{
    if (!c || !out) return LBM_EINVAL;
    if (!c->ready) return fail(c, LBM_ESTATE, "context not initialised");
    if (c->n_store > kNoAllocMaxCells)
        return fail(c, LBM_EINVAL, "lbm_diag_noalloc handles at most " + std::to_string(kNoAllocMaxCells) +
                                       " packed cells, this context has " + std::to_string(c->n_store) +
                                       "; use lbm_diag");
    cudaPointerAttributes attr{};
    LBM_CUDA(cudaPointerGetAttributes(&attr, c->ws), "workspace attributes");
    int dev = -1;
    LBM_CUDA(cudaGetDevice(&dev), "current device");
    if (dev < 0 || dev >= kMaxDevices) return fail(c, LBM_EINVAL, "device ordinal out of range");
    if (attr.type == cudaMemoryTypeDevice && attr.device != dev)
        return fail(c, LBM_EINVAL, "make the context's device current before lbm_diag_noalloc");
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(c, LBM_EINVAL, "the context's workspace is not device or managed memory");
    if (region) {
        cudaPointerAttributes ra{};
        LBM_CUDA(cudaPointerGetAttributes(&ra, region), "region attributes");
        if (ra.type != cudaMemoryTypeDevice && ra.type != cudaMemoryTypeManaged)
            return fail(c, LBM_EINVAL, "lbm_diag_noalloc needs the region in device memory (or NULL)");
        if (ra.type == cudaMemoryTypeDevice && ra.device != dev)
            return fail(c, LBM_EINVAL, "the region lies on another device than the current one");
    }
    if (c->n_store == 0) {
        for (int k = 0; k < 8; ++k) out[k] = 0.0;
        return LBM_OK;
    }
    if (total_blocks(c->base) > kNoAllocMaxBlocks + 1)
        return fail(c, LBM_EINVAL, "lbm_diag_noalloc handles launches of at most " +
                                       std::to_string(kNoAllocMaxBlocks + 1) + " blocks, this context needs " +
                                       std::to_string(total_blocks(c->base)) + " (" +
                                       std::to_string(c->base.n_general) + " general-path cells, " +
                                       std::to_string(c->base.gen_block) + " per block); use lbm_diag");
    double* scratch = nullptr;
    LBM_CUDA(noalloc_scratch(dev, c->stream, &scratch), "address of the diagnostics scratch");
    double* partials = scratch;
    double* result = scratch + (size_t)(kNoAllocMaxBlocks + 1) * kDiagSlots;
    Params P = c->base;
    P.fsrc = c->f(c->cur);
    P.fdst = nullptr;
    P.t = c->t;
    P.region = region;
    P.partials = partials;
    LBM_CUDA(launch(c->grid, kModeDiag, P, c->stream), "diag kernel");
    const int nblk = total_blocks(P);
    LBM_CUDA(launch_diag_finish(partials, nblk, result, c->stream), "diag reduction");
    LBM_CUDA(cudaMemcpyAsync(out, result, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "diag copy");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "diag sync");
    return LBM_OK;
}
