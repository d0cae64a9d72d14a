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
// A time-step launch: programmatic stream serialization (the step's blocks may
// start while the previous kernel on the stream finishes; lbm_kernel waits
// for it before its first dependent access) and, when P has one, the L2
// access-policy window of the row records and per-slot words, which every
// step reads, so that they stay resident while the populations stream past.
template <bool AN>
cudaError_t launch_step(int grid, const Params& P, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (P.l2_bytes > 0) {
        at[1].id = cudaLaunchAttributeAccessPolicyWindow;
        at[1].val.accessPolicyWindow.base_ptr = const_cast<void*>(P.l2_base);
        at[1].val.accessPolicyWindow.num_bytes = P.l2_bytes;
        at[1].val.accessPolicyWindow.hitRatio = P.l2_hit;
        at[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        at[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, lbm_kernel<LBM_Q, LBM_T, kModeStep, AN>, P);
}
}  // namespace

cudaError_t LBM_LAUNCHER(int mode, const Params& P, cudaStream_t s)
{
    const int grid = total_blocks(P);
    if (grid == 0) return cudaSuccess;
    if (mode == kModeStep) return P.aniso ? launch_step<true>(grid, P, s) : launch_step<false>(grid, P, s);
    if (P.aniso) {
        switch (mode) {
            case kModeMoments: lbm_kernel<LBM_Q, LBM_T, kModeMoments, true><<<grid, kBlock, 0, s>>>(P); break;
            default: lbm_kernel<LBM_Q, LBM_T, kModeDiag, true><<<grid, kBlock, 0, s>>>(P); break;
        }
        return cudaGetLastError();
    }
    switch (mode) {
        case kModeMoments: lbm_kernel<LBM_Q, LBM_T, kModeMoments><<<grid, kBlock, 0, s>>>(P); break;
        default: lbm_kernel<LBM_Q, LBM_T, kModeDiag><<<grid, kBlock, 0, s>>>(P); break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
