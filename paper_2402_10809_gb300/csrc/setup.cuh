// Declarations of the set-up and utility kernels (setup.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kSetupThreads = 256;
constexpr int kSetupCellsPerThread = 16;
constexpr int kSetupChunk = kSetupThreads * kSetupCellsPerThread;
constexpr int kCategories = 4;  // list groups: bulk, bulk on a periodic face, inlet, outlet
constexpr int kCounters = 5;    // the four group sizes and the number of ghost entries (part of group 0)
// Ghost entries: solid cells that share an aligned group of kGhostGroup cells
// with a bulk cell.  They sit in group 0 in index order and only store zeros
// into their (never read) distribution slots, so that every 32-byte sector a
// warp writes is written whole and the memory never has to merge a partial
// sector.  Marked by bit 31 of their cell-list entry.
constexpr int kGhostGroup = 16;
constexpr uint32_t kGhostFlag = 0x80000000u;
static_assert(kSetupCellsPerThread == kGhostGroup, "one set-up thread scans one ghost group");

// Error bits raised by setup_mask.
constexpr uint32_t kErrPorosity = 1u;  // porosity outside (0, 1] on a non-solid cell
constexpr uint32_t kErrInlet = 2u;     // inlet cell off its face, no inlet, or phi != 1
constexpr uint32_t kErrOutlet = 4u;    // outlet cell off its face, or without a fluid phi = 1 neighbour

struct SetupParams {
    int nx, ny, nz;
    int periodic[3];
    int n_cells, n_bulk;
    const uint8_t* flags;
    const float* phi;
    const uint32_t* cells;
    uint32_t* mask;
    float* bnd_prof;
    uint32_t* bnd_nbmask;
    int in_axis, in_side, out_axis, out_side;
    double in_center[3];
    double in_radius;
    uint32_t* err;
};

// Host launchers (setup.cu).  phase 0 of launch_setup_cells counts and scans,
// phase 1 emits the list of dense cell indices in four consecutive groups:
// bulk cells away from periodic faces, bulk cells on a periodic face, inlet
// cells, outlet cells (totals[0..3]).
struct CellGrid {
    int nx, ny, nz;
    int periodic[3];
};
cudaError_t launch_setup_cells(const uint8_t* flags, long long N, const CellGrid& G, uint32_t* counts,
                               uint32_t* offsets, uint32_t* totals, cudaStream_t s, int phase, uint32_t* cells);
cudaError_t launch_setup_mask(int q, const SetupParams& S, cudaStream_t s);
cudaError_t launch_init_state(int storage, const uint32_t* cells, int n_cells, int nx, int ny, long long N, int Q,
                              void* f, float* omega, float omega0, cudaStream_t s);
cudaError_t launch_pack_state(int storage, const uint32_t* cells, int n_cells, int nx, int ny, long long N, int Q,
                              void* f, void* state, int unpack, cudaStream_t s);
cudaError_t launch_diag_finish(const double* partials, int nblk, double* out, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, long long n, float v, cudaStream_t s);
cudaError_t launch_region_count(const uint32_t* cells, int n_cells, const uint8_t* region, unsigned long long* out,
                                cudaStream_t s);

}  // namespace lbm
