// mg_noalloc.cu -- the one entry point of the library that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need an
// answer: a time-stepping code inside a captured CUDA graph, a host with a hard
// device-memory budget already handed out, or a plug-in that runs inside
// another application's allocator.  mg_mac_constraint_noalloc lets them check
// the MAC constraint of a velocity field (the residual of Eq. 6 on cells) with
// no cudaMalloc at all: its reduction scratch is a fixed file-scope device
// array that every GPU loading this library holds until the process exits.
#include <mutex>

#include "../../include/mg.h"
#include "mg_device.cuh"

namespace mgp {
namespace {

// One block per kNaCellsPerBlock cells; three partial sums per block.
constexpr int kNaThreads = 256;
constexpr int kNaCellsPerBlock = kNaThreads * 8;
constexpr int kNaMaxBlocks = MG_NOALLOC_MAX_CELLS / kNaCellsPerBlock;

static __device__ __align__(256) double g_noalloc_partials[3 * kNaMaxBlocks];

struct Ptrs3 {
    const double* p[3];
};

// v = D(beta0 U) - beta0 S per cell (the same arithmetic as the projection's
// constraint check); partial sums {sum v, sum (beta0 S)^2, sum v^2} per block.
template <int DIM>
__global__ void __launch_bounds__(kNaThreads)
k_constraint_noalloc(int nx, int ny, int nz, double ihx, double ihy, double ihz, Ptrs3 U, Ptrs3 B0,
                     const double* __restrict__ b0c, const double* __restrict__ S, double* __restrict__ partials)
{
    const int total = nx * ny * nz;
    const int base = blockIdx.x * kNaCellsPerBlock;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < kNaCellsPerBlock; q += kNaThreads) {
        const int t = base + q;
        if (t >= total) break;
        int i, j, k;
        unflat(t, nx, ny, i, j, k);
        const size_t rx = ((size_t)k * ny + j) * (nx + 1) + i;
        double v = (B0.p[0][rx + 1] * U.p[0][rx + 1] - B0.p[0][rx] * U.p[0][rx]) * ihx;
        const size_t ry = ((size_t)k * (ny + 1) + j) * nx + i;
        v += (B0.p[1][ry + nx] * U.p[1][ry + nx] - B0.p[1][ry] * U.p[1][ry]) * ihy;
        if (DIM == 3) {
            const size_t rz = (size_t)t, pl = (size_t)nx * ny;
            v += (B0.p[2][rz + pl] * U.p[2][rz + pl] - B0.p[2][rz] * U.p[2][rz]) * ihz;
        }
        const double src = b0c[t] * S[t];
        v -= src;
        acc[0] += v;
        acc[1] += src * src;
        acc[2] += v * v;
    }
    __shared__ double sh[3][kNaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = 0; s < 3; ++s) {
        double x = acc[s];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[s][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) x += sh[threadIdx.x][w];
        partials[threadIdx.x * kNaMaxBlocks + blockIdx.x] = x;
    }
}

// out[s] = sum of the nblocks partials of slot s, in block order.
__global__ void k_constraint_noalloc_sum(const double* __restrict__ partials, int nblocks, double* __restrict__ out)
{
    __shared__ double sh[kNaThreads];
    for (int s = 0; s < 3; ++s) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) x += partials[s * kNaMaxBlocks + b];
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[s] = sh[0];
        __syncthreads();
    }
}

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = p;
    }
    *out = static_cast<double*>(g_scratch[dev]);
    return cudaSuccess;
}

}  // namespace
}  // namespace mgp

using namespace mgp;

extern "C" mg_status mg_mac_constraint_noalloc(const mg_geometry* g, const double* const U[3],
                                               const mg_beta0* beta0, const double* S, double* out, void* stream)
{
    bool ok = g && U && beta0 && beta0->cell && S && out && (g->dim == 2 || g->dim == 3) && g->loc == MG_LOC_CELL;
    for (int d = 0; ok && d < g->dim; ++d) ok = g->n[d] >= 1 && g->h[d] > 0.0 && U[d] && beta0->face[d];
    if (ok && g->dim == 2 && g->n[2] != 1) ok = false;
    if (!ok) {
        set_last_error("mg_mac_constraint_noalloc: null pointer or invalid cell grid");
        return MG_ERR_INVALID_ARG;
    }
    const long long cells = (long long)g->n[0] * g->n[1] * (g->dim == 3 ? g->n[2] : 1);
    if (cells > MG_NOALLOC_MAX_CELLS) {
        set_last_error("grid larger than MG_NOALLOC_MAX_CELLS: the fixed reduction scratch is too small");
        return MG_ERR_UNSUPPORTED;
    }
    double* scratch = nullptr;
    const cudaError_t se = scratch_for_current_device(&scratch);
    if (se != cudaSuccess) {
        set_last_error(cudaGetErrorString(se));
        return MG_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)((cells + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    const int nx = g->n[0], ny = g->n[1], nz = g->dim == 3 ? g->n[2] : 1;
    Ptrs3 u{{U[0], U[1], g->dim == 3 ? U[2] : nullptr}};
    Ptrs3 b{{beta0->face[0], beta0->face[1], g->dim == 3 ? beta0->face[2] : nullptr}};
    const double ihz = g->dim == 3 ? 1.0 / g->h[2] : 0.0;
    if (g->dim == 2)
        k_constraint_noalloc<2><<<nblocks, kNaThreads, 0, s>>>(nx, ny, nz, 1.0 / g->h[0], 1.0 / g->h[1], ihz, u, b,
                                                                beta0->cell, S, scratch);
    else
        k_constraint_noalloc<3><<<nblocks, kNaThreads, 0, s>>>(nx, ny, nz, 1.0 / g->h[0], 1.0 / g->h[1], ihz, u, b,
                                                                beta0->cell, S, scratch);
    note_launch();
    k_constraint_noalloc_sum<<<1, kNaThreads, 0, s>>>(scratch, nblocks, out);
    note_launch();
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        set_last_error(cudaGetErrorString(le));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}
