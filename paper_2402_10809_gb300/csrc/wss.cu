// Voxel wall-shear-stress proxy of the current time (the quantity whose sac
// average the paper reports beside the velocity, Sec. 4 results: the wall
// shear stress tau = sigma n - (n . sigma n) n).
//
// Voxel form: at a bulk cell with links to the wall (directions whose
// neighbour is solid or outside the box, the links the step bounces back),
// n = sum over those links of w_i c_i, normalised (the direction of the wall
// as seen from the cell); sigma = -(1 - omega(t)/2) Pi is the viscous stress
// recovered from the corrected second moment Pi that also gives the shear rate
// (Sec. 3), with omega(t) the rate of the collision of time t.  The output is
// |tau| in lattice units; cells without wall links, inlet and outlet cells stay
// at the caller's zero.  One thread per slot; only wall cells do any work, so
// the pass uses the general-path addressing for all of them.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbm {

template <int Q, class T, bool AN>
__global__ void __launch_bounds__(kBlock) wall_shear_kernel(const Params P, float* __restrict__ out, int compact)
{
    using L = Lattice<Q>;
    const int p = (int)blockIdx.x * kBlock + (int)threadIdx.x;
    if (p >= P.n_store) return;
    const uint32_t mask = P.mask[p];
    if ((mask & kGhostBit) || ((mask >> kTypeShift) & 3u) != kBulk) return;
    float nx = 0.0f, ny = 0.0f, nz = 0.0f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if ((mask >> opp(i)) & 1u) {  // y + c_i cannot pull from y: wall link
            nx += L::w(i) * L::cx(i);
            ny += L::w(i) * L::cy(i);
            nz += L::w(i) * L::cz(i);
        }
    }
    const float nn = sqrtf(nx * nx + ny * ny + nz * nz);
    if (!(nn > 0.0f)) return;
    nx /= nn;
    ny /= nn;
    nz /= nn;
    const Coords c = coords_of(P, p);
    float g[Q];
    pull_general<Q, T>(P, static_cast<const T*>(P.fsrc), c, mask, g);
    const Moments<Q> m = moments<Q>(g);
    Macro M;
    if constexpr (AN)
        M = macroscopic_aniso(P, p, __ldg(P.phi + p), m.sd, m.mx, m.my, m.mz);
    else
        M = macroscopic(P, __ldg(P.phi + p), m.sd, m.mx, m.my, m.mz);
    // corrected second moment Pi (as for the shear rate of the step)
    const float sd3 = M.sd * (1.0f / 3.0f);
    const float pxx = fmaf(M.ux, fmaf(-M.sigma, M.ux, M.Fx), m.sxx - sd3);
    const float pyy = fmaf(M.uy, fmaf(-M.sigma, M.uy, M.Fy), m.syy - sd3);
    const float pzz = fmaf(M.uz, fmaf(-M.sigma, M.uz, M.Fz), m.szz - sd3);
    const float pxy = fmaf(M.ux, fmaf(-M.sigma, M.uy, 0.5f * M.Fy), fmaf(0.5f * M.Fx, M.uy, m.sxy));
    const float pxz = fmaf(M.ux, fmaf(-M.sigma, M.uz, 0.5f * M.Fz), fmaf(0.5f * M.Fx, M.uz, m.sxz));
    const float pyz = fmaf(M.uy, fmaf(-M.sigma, M.uz, 0.5f * M.Fz), fmaf(0.5f * M.Fy, M.uz, m.syz));
    const float pn = sqrtf(fmaf(pxx, pxx, fmaf(pyy, pyy, fmaf(pzz, pzz, 2.0f * fmaf(pxy, pxy, fmaf(pxz, pxz, pyz * pyz))))));
    const float gdot = 3.0f * P.omega[p] * pn / M.rho;
    const float om = relaxation_rate(P, M.rho, gdot);
    const float s = -(1.0f - 0.5f * om);
    // sigma n, its normal part, and the tangential remainder
    const float sx = s * fmaf(pxx, nx, fmaf(pxy, ny, pxz * nz));
    const float sy = s * fmaf(pxy, nx, fmaf(pyy, ny, pyz * nz));
    const float sz = s * fmaf(pxz, nx, fmaf(pyz, ny, pzz * nz));
    const float sn = fmaf(sx, nx, fmaf(sy, ny, sz * nz));
    const float tx = sx - sn * nx, ty = sy - sn * ny, tz = sz - sn * nz;
    out[compact ? (long long)p : c.idx] = sqrtf(fmaf(tx, tx, fmaf(ty, ty, tz * tz)));
}

template <int Q, class T>
void launch_wall_shear_t(const Params& P, float* out, int compact, int grid, cudaStream_t s)
{
    if (P.aniso)
        wall_shear_kernel<Q, T, true><<<grid, kBlock, 0, s>>>(P, out, compact);
    else
        wall_shear_kernel<Q, T, false><<<grid, kBlock, 0, s>>>(P, out, compact);
}

template <int Q>
cudaError_t launch_wall_shear_q(int storage, const Params& P, float* out, int compact, int grid, cudaStream_t s)
{
    if (storage == 0) launch_wall_shear_t<Q, float>(P, out, compact, grid, s);
    else if (storage == 1) launch_wall_shear_t<Q, __half>(P, out, compact, grid, s);
    else launch_wall_shear_t<Q, __nv_bfloat16>(P, out, compact, grid, s);
    return cudaGetLastError();
}

cudaError_t launch_wall_shear(int q, int storage, const Params& P, float* out, int compact, cudaStream_t s)
{
    const int grid = (P.n_store + kBlock - 1) / kBlock;
    if (grid == 0) return cudaSuccess;
    if (q == 19) return launch_wall_shear_q<19>(storage, P, out, compact, grid, s);
    return launch_wall_shear_q<27>(storage, P, out, compact, grid, s);
}

}  // namespace lbm
