// Declarations of the set-up and utility kernels (setup.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kSetupThreads = 256;

// Error bits raised by the set-up kernels.
constexpr uint32_t kErrPorosity = 1u;  // porosity outside (0, 1] on a non-solid cell
constexpr uint32_t kErrInlet = 2u;     // inlet cell off its face, no inlet, or phi != 1
constexpr uint32_t kErrOutlet = 4u;    // outlet cell off its face, or without a fluid phi = 1 neighbour
constexpr uint32_t kErrFlag = 8u;      // a flag value outside 0..3

struct SetupParams {
    int nx, ny, nz;
    int periodic[3];
    int n_store;
    const uint8_t* flags;     // dense
    const float* phi;         // dense
    const uint32_t* rows;     // [n_store] row id of each slot
    const int* rowbase;       // [ny nz]
    uint32_t* mask;           // [n_store]
    float* bnd_prof;          // [n_store]
    uint32_t* bnd_nbmask;     // [n_store]
    int in_axis, in_side, out_axis, out_side;
    double in_center[3];
    double in_radius;
    uint32_t* err;
};

// Host launchers (setup.cu).  setup_rows: span [xmin, xmin + ext) of the
// non-solid cells of every row; setup_slots: row id and porosity of every slot
// (rowbase from the host scan of ext); setup_mask: link masks, boundary data
// and input validation of every slot.
cudaError_t launch_setup_rows(const uint8_t* flags, int nx, int nrows, int* xmin, int* ext, uint32_t* err,
                              cudaStream_t s);
cudaError_t launch_setup_slots(const float* phi, int nx, int nrows, const int* rowbase, const int* xmin,
                               const int* ext, uint32_t* rows, float* phi_s, cudaStream_t s);
cudaError_t launch_setup_rownb(const int* rowbase, int ny, int nz, int py, int pz, int* out, cudaStream_t s);
cudaError_t launch_setup_mask(int q, const SetupParams& S, cudaStream_t s);
cudaError_t launch_diag_finish(const double* partials, int nblk, double* out, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, long long n, float v, cudaStream_t s);
cudaError_t launch_fill_u32(uint32_t* p, long long n, uint32_t v, cudaStream_t s);
// Host tables of a layout: classify_count gives each chunk of slots its
// counts (general, outlet, ghost, inlet); classify_write, from the chunks'
// exclusive offsets (general, outlet), the ascending general and outlet lists.
int classify_chunks(int n);
cudaError_t launch_classify_count(const uint32_t* mask, int n, int wide, int4* counts, cudaStream_t s);
cudaError_t launch_classify_write(const uint32_t* mask, int n, int wide, const int2* offsets, uint32_t* general,
                                  uint32_t* outlets, cudaStream_t s);
cudaError_t launch_region_count(const uint32_t* rows, const int* rowbase, const uint32_t* mask, int n_store, int nx,
                                const uint8_t* region, uint32_t wall_bits, unsigned long long* out, cudaStream_t s);
cudaError_t launch_scatter_f64(const uint32_t* rows, const int* rowbase, const uint32_t* mask, int n_store, int nx,
                               const double* src, double* dst, cudaStream_t s);

// Copies of the populations that cross a z-slab face (api.cu: lbm_halo_pack,
// lbm_halo_unpack, lbm_halo_exchange): task k copies count[k] elements of
// elem bytes (2 or 4) from src[k] to dst[k]; up to 18 tasks in one launch.
constexpr int kHaloTasks = 18;
struct HaloCopy {
    const void* src[kHaloTasks];
    void* dst[kHaloTasks];
    long long count[kHaloTasks];
    int ntask;
    int elem;
};
cudaError_t launch_halo_copy(const HaloCopy& H, cudaStream_t s);

// Volume-averaged porosity of a wire mask (porosity.cu): three sliding-window
// passes through the caller's scratch (ws_x: N bytes, ws_y: N uint16).  The x
// pass stages up to kPorosityRowBytes of rows per block in shared memory.
constexpr int kPorosityRowBytes = 16384;
constexpr int kPorosityMaxNx = 16384;
constexpr int kPorosityMaxWindow = 255;  // window^2 fits uint16, window^3 < 2^24
size_t porosity_smem_bytes(int nx);
cudaError_t launch_porosity_average(const uint8_t* wire, const uint8_t* flags, int nx, int ny, int nz, int window,
                                    float phi_min, float* phi, uint8_t* ws_x, uint16_t* ws_y, cudaStream_t s);

}  // namespace lbm
