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
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* __restrict__ partials, int slot)
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
            if (lane == 0) partials[q * kRedBlocks + slot] = x;
        }
    }
}
template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* __restrict__ partials)
{
    block_reduce_store<NS>(v, partials, blockIdx.x);
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

// IEEE-754 conversions between binary64 and binary32 done with 32-bit integer
// operations.  GB300 issues about two FP64 operations per SM per clock and a
// hardware conversion occupies that pipe like an FMA, so in the FP64-bound
// kernels the conversions move to the integer pipe.  Normal results follow the
// format definition: binary64 -> binary32 keeps the top 23 fraction bits and
// rounds to nearest, ties to even, on the 29 bits dropped (a carry out of the
// fraction increments the exponent, up to infinity); binary32 -> binary64 is
// exact (exponent rebiased by 1023 - 127, fraction shifted left by 29).  Zeros
// are handled here; subnormal, infinite and NaN operands or results take the
// hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e - 897u <= 253u) {  // 897 <= e <= 1150: the binary32 exponent field e - 896 is 1 .. 254
        unsigned r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu, half = 0x10000000u;
        r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;
        return __uint_as_float(r | (hi & 0x80000000u));
    }
    if (e == 0 && ((hi & 0xfffffu) | lo) == 0) return __uint_as_float(hi & 0x80000000u);
    return __double2float_rn(v);
}
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e - 1u < 254u) {  // normal
        const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if ((u & 0x7fffffffu) == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
}

// f64_to_f32_rn(v * 2^s) with the exact power-of-two scaling folded into the
// exponent field, so the scaling costs no FP64 operation: the FP64 residual
// kernels scale r by a power of two near 1/||f|| this way.  Normal results are
// the format definition's (as above); zeros keep their sign; everything else
// (subnormal or non-finite operands, results outside the normal binary32
// range) takes scalbn and the hardware conversion.
__device__ __forceinline__ float f64_to_f32_pow2(double v, int s)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const int eo = e + s - 896;   // binary32 exponent field of v * 2^s
    if (e != 0 && e != 0x7ff && eo >= 1 && eo <= 254) {
        unsigned r = ((unsigned)eo << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu, half = 0x10000000u;
        r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;
        return __uint_as_float(r | (hi & 0x80000000u));
    }
    if (e == 0 && ((hi & 0xfffffu) | lo) == 0) return __uint_as_float(hi & 0x80000000u);
    return __double2float_rn(scalbn(v, s));
}
// -log2 p of a power of two p (the residual scale)
__device__ __forceinline__ int pow2_shift(double p)
{
    return 1023 - (int)(((unsigned)__double2hiint(p) >> 20) & 0x7ffu);
}
// the largest power of two <= x, for finite normal x > 0
__device__ __forceinline__ double pow2_floor(double x) { return __hiloint2double(__double2hiint(x) & 0x7ff00000, 0); }

// the residual scale of a solve from ||f||^2: the power of two <= ||f|| (1
// when f = 0) and the factor that turns sums of scaled squares into squared
// relative residuals
__device__ __forceinline__ void set_fscale(DevScalars* d)
{
    const double f2 = d->fnorm2;
    if (f2 > 0.0) {
        const double p = pow2_floor(sqrt(f2));
        d->fscale = p;
        d->rscale2 = (p * p) / f2;
    } else {
        d->fscale = 1.0;
        d->rscale2 = 1.0;
    }
}

// 1/d by Newton's method on g(y) = 1/y - d, whose step y <- y + y (1 - d y)
// squares the relative error.  The start is PTX rcp.approx.ftz.f32 of d rounded
// to binary32 (relative error below about 2^-22 in all); two steps bring it to
// the binary64 rounding level, so the result is within about one ulp of 1/d
// (not always the correctly rounded quotient).  That is four FP64 FMAs; the
// FP64 pipe is the bound of the kernels that divide (face coefficients,
// projection updates).  Operands outside [2^-125, 2^126), and zeros,
// infinities and NaNs, take the IEEE division.
__device__ __forceinline__ double recip_nr(double d)
{
    const unsigned e = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
    if (e - 898u > 250u) return 1.0 / d;
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(f64_to_f32_rn(d)));
    double y = f32_to_f64(y0);
    y = fmadd(y, fmadd(-d, y, 1.0), y);
    y = fmadd(y, fmadd(-d, y, 1.0), y);
    return y;
}

__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
template <typename T>
__device__ __forceinline__ T from_f64(double v);
template <>
__device__ __forceinline__ float from_f64<float>(double v) { return f64_to_f32_rn(v); }
template <>
__device__ __forceinline__ double from_f64<double>(double v) { return v; }

// Row r of x = Minv b (dense coarsest solve), summed by the 32 lanes of a warp:
// lane-strided partial sums, then a shuffle-down tree; every lane must call it.
template <typename T>
__device__ __forceinline__ double dense_row(const double* __restrict__ Minv, int N, const T* __restrict__ b, int r,
                                            int lane)
{
    double s = 0.0;
    for (int c = lane; c < N; c += 32) s = fmadd(Minv[(size_t)r * N + c], to_f64(b[c]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

template <typename T>
__device__ __forceinline__ T recip(T d);
// FP32 levels only precondition the FP64 refinement: the fast reciprocal
// (about 2 ulp) is accurate far beyond what the V-cycle needs.
template <>
__device__ __forceinline__ float recip<float>(float d) { return d != 0.f ? __fdividef(1.f, d) : 0.f; }
template <>
__device__ __forceinline__ double recip<double>(double d) { return d != 0.0 ? 1.0 / d : 0.0; }

// coarse value seen from fine cell index i along one axis (linear interpolation):
// parent P = i/2 with weight 3/4, the neighbour Q on the fine cell's side with 1/4;
// beyond a boundary the neighbour is the periodic image, the mirror (Neumann) or
// the odd reflection (Dirichlet).
struct Lin1D {
    int p, q;
    float sq;  // sign applied to the value at q (+1, or -1 for the Dirichlet ghost)
};

__device__ __forceinline__ Lin1D lin1d(int i, int nc, int bclo, int bchi)
{
    Lin1D r;
    r.p = i >> 1;
    r.sq = 1.f;
    if (i & 1) {
        r.q = r.p + 1;
        if (r.q >= nc) {
            if (bchi == BCP) r.q = 0;
            else { r.q = r.p; r.sq = (bchi == BCD) ? -1.f : 1.f; }
        }
    } else {
        r.q = r.p - 1;
        if (r.q < 0) {
            if (bclo == BCP) r.q = nc - 1;
            else { r.q = r.p; r.sq = (bclo == BCD) ? -1.f : 1.f; }
        }
    }
    return r;
}

}  // namespace mgp
