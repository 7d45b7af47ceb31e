// mg_probe.cu -- FP64 fused multiply-add throughput probe (measurement support).
//
// The FP64 kernels of the solve (the refinement residuals, right-hand sides,
// projection updates and coefficient setup) are bound by the FP64 pipe, whose
// rate on this GPU is a small fraction of the FP32 rate.  Their roofline needs
// that rate as measured, not as listed: this kernel issues only independent
// FP64 FMA chains, eight per thread, so that the pipe -- not latency, memory or
// issue slots -- sets its time.  The caller times the launch with CUDA events on
// the stream and divides the flop count returned here by the elapsed time.  It
// reads no memory and changes no GPU setting.
#include "../../include/mg.h"
#include "mg_internal.cuh"

namespace mgp {
namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma_probe(int iters, double* sink)
{
    // distinct starting values per thread and chain; multiplier and addend keep
    // every chain finite and away from denormals for any iteration count
    const double t = 1.0 + 1e-7 * (double)(blockIdx.x * blockDim.x + threadIdx.x);
    double a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = t + 0.125 * c;
    const double m = 0.999999, q = 1e-6;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], m, q);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    if (s == -1.0) sink[0] = s;   // never true: keeps the chains live
}

}  // namespace
}  // namespace mgp

using namespace mgp;

extern "C" mg_status mg_fp64_fma_probe(int blocks, int iters, double* sink, void* stream, double* flops)
{
    if (blocks <= 0 || iters <= 0 || !sink || !flops) {
        set_last_error("mg_fp64_fma_probe: blocks and iters must be positive, sink and flops non-null");
        return MG_ERR_INVALID_ARG;
    }
    MGP_LAUNCH(k_fp64_fma_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, sink));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    *flops = 2.0 * kProbeChains * (double)iters * (double)blocks * 256.0;
    return MG_OK;
}
