// One translation unit per (velocity set, storage type): compiled several
// times with -DLBM_Q=19|27 and -DLBM_STORE=0|1|2 so the large unrolled
// kernels build in parallel.  Exports a host launcher per instantiation.
#include <cuda_runtime.h>

#include "kernels.cuh"

#ifndef LBM_Q
#error "LBM_Q must be defined"
#endif
#ifndef LBM_STORE
#error "LBM_STORE must be defined"
#endif

#if LBM_STORE == 0
#define LBM_T float
#define LBM_TNAME f32
#elif LBM_STORE == 1
#define LBM_T __half
#define LBM_TNAME f16
#else
#define LBM_T __nv_bfloat16
#define LBM_TNAME bf16
#endif

#define LBM_CAT2(a, b, c) launch_step_##a##_##b
#define LBM_CAT(a, b) LBM_CAT2(a, b, 0)
#define LBM_LAUNCHER LBM_CAT(LBM_Q, LBM_TNAME)

namespace lbm {

namespace {
// A time-step launch with the L2 access-policy window of P: the row records
// and per-slot words it covers are read by every step, so they stay resident
// in the persisting part of L2 while the populations stream past them.
template <bool AN>
cudaError_t launch_step_window(int grid, const Params& P, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeAccessPolicyWindow;
    at[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(P.l2_base);
    at[0].val.accessPolicyWindow.num_bytes = P.l2_bytes;
    at[0].val.accessPolicyWindow.hitRatio = P.l2_hit;
    at[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, lbm_kernel<LBM_Q, LBM_T, kModeStep, AN>, P);
}
}  // namespace

cudaError_t LBM_LAUNCHER(int mode, const Params& P, cudaStream_t s)
{
    const int grid = total_blocks(P);
    if (grid == 0) return cudaSuccess;
    if (mode == kModeStep && P.l2_bytes > 0)
        return P.aniso ? launch_step_window<true>(grid, P, s) : launch_step_window<false>(grid, P, s);
    if (P.aniso) {
        switch (mode) {
            case kModeStep: lbm_kernel<LBM_Q, LBM_T, kModeStep, true><<<grid, kBlock, 0, s>>>(P); break;
            case kModeMoments: lbm_kernel<LBM_Q, LBM_T, kModeMoments, true><<<grid, kBlock, 0, s>>>(P); break;
            default: lbm_kernel<LBM_Q, LBM_T, kModeDiag, true><<<grid, kBlock, 0, s>>>(P); break;
        }
        return cudaGetLastError();
    }
    switch (mode) {
        case kModeStep: lbm_kernel<LBM_Q, LBM_T, kModeStep><<<grid, kBlock, 0, s>>>(P); break;
        case kModeMoments: lbm_kernel<LBM_Q, LBM_T, kModeMoments><<<grid, kBlock, 0, s>>>(P); break;
        default: lbm_kernel<LBM_Q, LBM_T, kModeDiag><<<grid, kBlock, 0, s>>>(P); break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
