// Velocity sets for the fused LBM kernels (Sec. 3: D3Q27, c_s^2 = 1/3; D3Q19
// for the 19-velocity workload).  Directions come in opposite pairs: index 0 is
// the rest velocity, then (2k-1, 2k) are c and -c, so opp(i) is i+1 / i-1.
// Everything is constexpr so that fully unrolled loops fold c_i and w_i.
#pragma once

namespace lbm {

template <int Q>
struct Lattice;

template <>
struct Lattice<27> {
    static constexpr int Q = 27;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                               1, -1, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                               1, -1, 1, -1, -1, 1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                               1, -1, -1, 1, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr float w(int i)
    {
        return i == 0 ? 8.0f / 27.0f : i < 7 ? 2.0f / 27.0f : i < 19 ? 1.0f / 54.0f : 1.0f / 216.0f;
    }
};

template <>
struct Lattice<19> {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int cx(int i) { return Lattice<27>::cx(i); }
    __host__ __device__ static constexpr int cy(int i) { return Lattice<27>::cy(i); }
    __host__ __device__ static constexpr int cz(int i) { return Lattice<27>::cz(i); }
    __host__ __device__ static constexpr float w(int i)
    {
        return i == 0 ? 1.0f / 3.0f : i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f;
    }
};

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

template <int Q>
__host__ __device__ constexpr int c_axis(int i, int a)
{
    return a == 0 ? Lattice<Q>::cx(i) : a == 1 ? Lattice<Q>::cy(i) : Lattice<Q>::cz(i);
}

// Index of the direction (cx, cy, cz) in the Q-velocity set, -1 if absent.
template <int Q>
__host__ __device__ constexpr int find_dir(int cx, int cy, int cz)
{
    for (int i = 0; i < Q; ++i)
        if (Lattice<Q>::cx(i) == cx && Lattice<Q>::cy(i) == cy && Lattice<Q>::cz(i) == cz) return i;
    return -1;
}

}  // namespace lbm
