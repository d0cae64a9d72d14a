// Set-up of the anisotropic permeability (Sec. 3 remark on the velocity
// solution): K = k(phi) S^{-1} with the isotropic closure k(phi) of the step
// (Kozeny-Carman or constant permeability, Ergun's C_F) and a per-cell
// symmetric positive definite shape tensor S.  Per slot with phi < 1 it stores
//     Ah = (phi nu / 2) K^{-1}    = (K1 / (2 phi)) S,
//     B  = (phi^2 C_F / 2) K^{-1/2} = (K2 / (2 phi)) S^{1/2},
// K1 = phi^2 nu / k and K2 = phi^3 C_F / sqrt(k) the isotropic drag
// coefficients, so S = Id gives back the isotropic drag exactly.  S^{1/2} comes
// from the eigendecomposition S = V diag(l) V^T by cyclic Jacobi rotations in
// FP64: S^{1/2} = V diag(sqrt(l)) V^T.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbm {
namespace {

// Cyclic Jacobi eigenvalue iteration for a symmetric 3x3 matrix: each rotation
// in the (p, q) plane, angle from theta = (a_qq - a_pp) / (2 a_pq) and
// t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), zeroes a_pq; V accumulates
// the rotations.  Converges quadratically; at most 16 sweeps.
__device__ void jacobi3(double a[3][3], double v[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 16; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double diag = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > 1e-32 * diag)) break;
        for (int k = 0; k < 3; ++k) {
            const int p = k == 2 ? 1 : 0, q = k == 0 ? 1 : 2, r = 3 - p - q;
            const double apq = a[p][q];
            if (apq == 0.0) continue;
            const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            const double arp = a[r][p], arq = a[r][q];
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
            for (int i = 0; i < 3; ++i) {
                const double vip = v[i][p], viq = v[i][q];
                v[i][p] = c * vip - s * viq;
                v[i][q] = s * vip + c * viq;
            }
        }
    }
}

__global__ void setup_aniso(const Params P, const float* __restrict__ S, long long N, float* __restrict__ out,
                            uint32_t* err)
{
    const int p = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (p >= P.n_store) return;
    float val[12];
    for (int k = 0; k < 12; ++k) val[k] = 0.0f;
    const float phi = P.phi[p];
    if (!(P.mask[p] & kGhostBit) && phi < 1.0f) {
        const long long idx = coords_of(P, p).idx;
        double s[6];
        bool finite = true;
        for (int k = 0; k < 6; ++k) {
            s[k] = (double)S[(long long)k * N + idx];
            finite = finite && isfinite(s[k]);
        }
        double a[3][3] = {{s[0], s[3], s[4]}, {s[3], s[1], s[5]}, {s[4], s[5], s[2]}};
        double v[3][3];
        if (finite) jacobi3(a, v);
        const double l[3] = {a[0][0], a[1][1], a[2][2]};
        if (!finite || !(l[0] > 0.0 && l[1] > 0.0 && l[2] > 0.0)) {
            atomicOr(err, 1u);
        } else {
            double h[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    h[i][j] = v[i][0] * sqrt(l[0]) * v[j][0] + v[i][1] * sqrt(l[1]) * v[j][1] +
                              v[i][2] * sqrt(l[2]) * v[j][2];
            float k1, k2;
            const float iphi = __frcp_rn(phi);
            darcy_coeffs(P, phi, iphi, k1, k2);
            const float ca = 0.5f * k1 * iphi, cb = 0.5f * k2 * iphi;
            const double hs[6] = {h[0][0], h[1][1], h[2][2], h[0][1], h[0][2], h[1][2]};
            for (int k = 0; k < 6; ++k) {
                val[k] = ca * (float)s[k];
                val[6 + k] = cb * (float)hs[k];
            }
        }
    }
    for (int k = 0; k < 12; ++k) out[(size_t)k * P.n_store + p] = val[k];
}

}  // namespace

cudaError_t launch_setup_aniso(const Params& P, const float* S, long long N, float* out, uint32_t* err,
                               cudaStream_t s)
{
    if (P.n_store == 0) return cudaSuccess;
    setup_aniso<<<(P.n_store + kBlock - 1) / kBlock, kBlock, 0, s>>>(P, S, N, out, err);
    return cudaGetLastError();
}

}  // namespace lbm
