// One translation unit per (velocity set, storage type), like step.cu: the
// reverse time step and the outlet fix-up of the discrete adjoint.
#include <cuda_runtime.h>

#include "adjoint.cuh"

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

#define LBM_CAT2(a, b, c) launch_adjoint_##a##_##b
#define LBM_CAT(a, b) LBM_CAT2(a, b, 0)
#define LBM_LAUNCHER LBM_CAT(LBM_Q, LBM_TNAME)

namespace lbm {

namespace {
// A reverse-step launch: programmatic stream serialization, as for the time
// steps, and the forward step's L2 window (the per-slot words every reverse
// step reads too) when the context has one.
template <int TPS, bool AN>
cudaError_t launch_reverse(int grid, size_t smem, const AdjParams& A, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (A.F.l2_bytes > 0) {
        at[1].id = cudaLaunchAttributeAccessPolicyWindow;
        at[1].val.accessPolicyWindow.base_ptr = const_cast<void*>(A.F.l2_base);
        at[1].val.accessPolicyWindow.num_bytes = A.F.l2_bytes;
        at[1].val.accessPolicyWindow.hitRatio = A.F.l2_hit;
        at[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        at[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, adjoint_kernel<LBM_Q, LBM_T, TPS, AN>, A);
}
}  // namespace

// what = 0: reverse time step; 1: outlet fix-up; 2: outlet ordinals (once per call).
cudaError_t LBM_LAUNCHER(int what, const AdjParams& A, cudaStream_t s)
{
    if (what == 0) {
        const int grid = total_blocks(A.F);
        if (grid == 0) return cudaSuccess;
        constexpr size_t smem = adjoint_smem_bytes<LBM_Q>();
        static const cudaError_t attr = [] {
            const void* k[4] = {(const void*)adjoint_kernel<LBM_Q, LBM_T, 512, false>,
                                (const void*)adjoint_kernel<LBM_Q, LBM_T, 384, false>,
                                (const void*)adjoint_kernel<LBM_Q, LBM_T, 512, true>,
                                (const void*)adjoint_kernel<LBM_Q, LBM_T, 384, true>};
            for (const void* f : k) {
                const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }();
        if (attr != cudaSuccess) return attr;
        // grids of up to two waves of the 512-thread variant (152 SMs) take
        // the 384-thread one
        const bool small = grid <= 2 * 152 * (512 / kBlock);
        if (A.F.aniso)
            return small ? launch_reverse<384, true>(grid, smem, A, s) : launch_reverse<512, true>(grid, smem, A, s);
        return small ? launch_reverse<384, false>(grid, smem, A, s) : launch_reverse<512, false>(grid, smem, A, s);
    } else if (what == 1) {
        if (A.n_out == 0) return cudaSuccess;
        adjoint_outlet_fixup<LBM_Q><<<(A.n_out + 127) / 128, 128, 0, s>>>(A);
    } else {
        if (A.n_out == 0) return cudaSuccess;
        adjoint_outlet_ordinals<LBM_Q><<<(A.n_out + 127) / 128, 128, 0, s>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace lbm
