// mg_device.cuh -- device-side helpers shared by the kernel translation units.
#pragma once

#include "mg_internal.cuh"

namespace mgp {

constexpr int kThreads = 256;

__host__ __device__ inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Deterministic block reduction of NS doubles; thread 0 stores the block's
// partial sums at partials[q * kRedBlocks + blockIdx.x].  The grid must have
// exactly kRedBlocks blocks (1-D grid) of kThreads threads (any block shape).
template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* __restrict__ partials)
{
    __shared__ double sh[NS][kThreads / 32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);  // 1-D or 2-D blocks
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            double x = (lane < kThreads / 32) ? sh[q][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) partials[q * kRedBlocks + blockIdx.x] = x;
        }
    }
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// (i, j, k) of a flattened x-fastest index
__device__ __forceinline__ void unflat(int t, int nx, int ny, int& i, int& j, int& k)
{
    i = t % nx;
    const int q = t / nx;
    j = q % ny;
    k = q / ny;
}

// a * b + c with one rounding.  The smoother and residual rows accumulate
// their off-diagonal terms through this, so every kernel that evaluates a row
// rounds the same chain the same way, whatever the compiler would contract.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T recip(T d);
// FP32 levels only precondition the FP64 refinement: the fast reciprocal
// (about 2 ulp) is accurate far beyond what the V-cycle needs.
template <>
__device__ __forceinline__ float recip<float>(float d) { return d != 0.f ? __fdividef(1.f, d) : 0.f; }
template <>
__device__ __forceinline__ double recip<double>(double d) { return d != 0.0 ? 1.0 / d : 0.0; }

}  // namespace mgp
