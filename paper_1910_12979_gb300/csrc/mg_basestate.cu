// mg_basestate.cu -- the base state on the device: beta0 of Eq. 5 and its
// mapping onto the grid (the step that feeds the coefficient setup).
//
// Keeping the one-dimensional base state and its mapping resident on the GPU
// removes the host round trips that the paper (S6) names as a growing cost of
// its GPU port.
#include "../../include/mg.h"
#include "mg_device.cuh"

namespace mgp {
namespace {

constexpr int kScanThreads = 1024;

// beta0_{k+1} = rho0_0 exp( sum_{m<=k} (1/2)(1/G_m + 1/G_{m+1}) (ln p0_{m+1} - ln p0_m) ):
// the trapezoid rule for the integral of (1/Gamma1) d(ln p0), which equals the
// integral of dp0/dr / (Gamma1 p0) in Eq. 5.  One CTA: every thread sums a
// contiguous segment, a block scan of the segment sums gives each segment's
// offset (fixed order: deterministic), then the segments are written.
__global__ void __launch_bounds__(kScanThreads) k_beta0_scan(const double* __restrict__ p0, const double* __restrict__ g,
                                                            double g1, double rho00, int nr, double* __restrict__ beta0)
{
    __shared__ double part[kScanThreads];
    const int t = threadIdx.x, m = nr - 1;  // m increments
    const int per = (m + kScanThreads - 1) / kScanThreads;
    const int a = t * per, e = min(a + per, m);
    auto inc = [&](int k) {
        const double ga = g ? g[k] : g1, gb = g ? g[k + 1] : g1;
        return 0.5 * (1.0 / ga + 1.0 / gb) * (log(p0[k + 1]) - log(p0[k]));
    };
    double s = 0.0;
    for (int k = a; k < e; ++k) s += inc(k);
    part[t] = s;
    __syncthreads();
    // inclusive scan of the segment sums (Hillis-Steele, fixed order)
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const double v = t >= o ? part[t - o] : 0.0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    double acc = t > 0 ? part[t - 1] : 0.0;
    if (t == 0) beta0[0] = rho00;
    for (int k = a; k < e; ++k) {
        acc += inc(k);
        beta0[k + 1] = rho00 * exp(acc);
    }
}

__device__ __forceinline__ double interp(const double* __restrict__ f, int nr, double r0, double dr, double r)
{
    const double s = (r - r0) / dr;
    if (s <= 0.0) return f[0];
    if (s >= (double)(nr - 1)) return f[nr - 1];
    const int k = (int)floor(s);
    const double w = s - k;
    return (1.0 - w) * f[k] + w * f[k + 1];
}

struct MapArgs {
    int dim, nx, ny, nz, spherical, nr;
    double hx, hy, hz, cx, cy, cz, r0, dr;
    const double* beta0_r;
    const double* rho0_r;
};

__device__ __forceinline__ double radius(const MapArgs& A, double x, double y, double z)
{
    if (!A.spherical) return A.dim == 3 ? z : y;
    const double dx = x - A.cx, dy = y - A.cy, dz = A.dim == 3 ? z - A.cz : 0.0;
    return sqrt(dx * dx + dy * dy + dz * dz);
}

// One warp per kWarpRows x-rows of the target array (row = j + my * k),
// kMapWarps warps per block.  The radius of a plane-parallel base state is the
// height, constant along a row, so lane q interpolates the values of the
// warp's row q once and the warp broadcasts them by shuffles (the
// interpolation and the divisions are latency-bound FP64 work, done for the
// warp's rows in parallel; the coalesced stores are the per-cell cost); a
// spherical base state is interpolated cell by cell.
constexpr int kMapWarps = 8, kWarpRows = 4;

__global__ void __launch_bounds__(32 * kMapWarps) k_map_cells(MapArgs A, long long rows, double* __restrict__ sigma,
                                                              double* __restrict__ b0c)
{
    const long long row0 = ((long long)blockIdx.x * kMapWarps + threadIdx.y) * kWarpRows;
    if (row0 >= rows) return;   // whole warp
    const int lane = threadIdx.x;
    auto values = [&](double r, double& b, double& sg) {
        b = interp(A.beta0_r, A.nr, A.r0, A.dr, r);
        sg = b / interp(A.rho0_r, A.nr, A.r0, A.dr, r);
    };
    double bq = 0.0, sq = 0.0;   // lane q < kWarpRows: the values of row row0 + q
    if (!A.spherical && lane < kWarpRows && row0 + lane < rows) {
        const long long row = row0 + lane;
        const int j = (int)(row % A.ny), k = (int)(row / A.ny);
        values(radius(A, 0.0, (j + 0.5) * A.hy, (k + 0.5) * A.hz), bq, sq);
    }
#pragma unroll
    for (int q = 0; q < kWarpRows; ++q) {
        const long long row = row0 + q;
        const double b = __shfl_sync(0xffffffffu, bq, q), sg = __shfl_sync(0xffffffffu, sq, q);
        if (row >= rows) break;   // warp-uniform
        const size_t base = (size_t)row * A.nx;
        if (!A.spherical) {
            for (int i = lane; i < A.nx; i += 32) {
                if (sigma) sigma[base + i] = sg;
                if (b0c) b0c[base + i] = b;
            }
            continue;
        }
        const int j = (int)(row % A.ny), k = (int)(row / A.ny);
        for (int i = lane; i < A.nx; i += 32) {
            double bc, sc;
            values(radius(A, (i + 0.5) * A.hx, (j + 0.5) * A.hy, (k + 0.5) * A.hz), bc, sc);
            if (sigma) sigma[base + i] = sc;
            if (b0c) b0c[base + i] = bc;
        }
    }
}

__global__ void __launch_bounds__(32 * kMapWarps) k_map_faces(MapArgs A, int d, long long rows,
                                                              double* __restrict__ out)
{
    const long long row0 = ((long long)blockIdx.x * kMapWarps + threadIdx.y) * kWarpRows;
    if (row0 >= rows) return;   // whole warp
    const int mx = A.nx + (d == 0), my = A.ny + (d == 1);
    const int lane = threadIdx.x;
    auto yz = [&](long long row, double& y, double& z) {
        const int j = (int)(row % my), k = (int)(row / my);
        y = (j + (d == 1 ? 0.0 : 0.5)) * A.hy;
        z = (k + (d == 2 ? 0.0 : 0.5)) * A.hz;
    };
    double bq = 0.0;
    if (!A.spherical && lane < kWarpRows && row0 + lane < rows) {
        double y, z;
        yz(row0 + lane, y, z);
        bq = interp(A.beta0_r, A.nr, A.r0, A.dr, radius(A, 0.0, y, z));
    }
#pragma unroll
    for (int q = 0; q < kWarpRows; ++q) {
        const long long row = row0 + q;
        const double b = __shfl_sync(0xffffffffu, bq, q);
        if (row >= rows) break;   // warp-uniform
        const size_t base = (size_t)row * mx;
        if (!A.spherical) {
            for (int i = lane; i < mx; i += 32) out[base + i] = b;
            continue;
        }
        double y, z;
        yz(row, y, z);
        for (int i = lane; i < mx; i += 32) {
            const double x = (i + (d == 0 ? 0.0 : 0.5)) * A.hx;
            out[base + i] = interp(A.beta0_r, A.nr, A.r0, A.dr, radius(A, x, y, z));
        }
    }
}

}  // namespace
}  // namespace mgp

using namespace mgp;

extern "C" mg_status mg_base_state_beta0(const double* p0, const double* gamma1, double gamma1_const, double rho0_base,
                                         int nr, double* beta0, void* stream)
{
    if (!p0 || !beta0 || nr < 1 || (!gamma1 && !(gamma1_const > 0.0))) {
        set_last_error("mg_base_state_beta0: null pointer, nr < 1 or no Gamma1");
        return MG_ERR_INVALID_ARG;
    }
    MGP_LAUNCH(k_beta0_scan<<<1, kScanThreads, 0, (cudaStream_t)stream>>>(p0, gamma1, gamma1_const, rho0_base, nr,
                                                                           beta0));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return MG_ERR_CUDA; }
    return MG_OK;
}

extern "C" mg_status mg_base_state_map(const mg_geometry* g, int spherical, const double center[3], double r0, double dr,
                                       int nr, const double* beta0_r, const double* rho0_r, double* sigma,
                                       double* beta0_cell, double* const beta0_face[3], void* stream)
{
    if (!g || (g->dim != 2 && g->dim != 3) || !beta0_r || !rho0_r || nr < 1 || !(dr > 0.0) ||
        (spherical && !center)) {
        set_last_error("mg_base_state_map: invalid argument");
        return MG_ERR_INVALID_ARG;
    }
    MapArgs A;
    A.dim = g->dim;
    A.nx = g->n[0];
    A.ny = g->n[1];
    A.nz = g->dim == 3 ? g->n[2] : 1;
    A.spherical = spherical;
    A.nr = nr;
    A.hx = g->h[0];
    A.hy = g->h[1];
    A.hz = g->dim == 3 ? g->h[2] : 1.0;
    A.cx = spherical ? center[0] : 0.0;
    A.cy = spherical ? center[1] : 0.0;
    A.cz = spherical && g->dim == 3 ? center[2] : 0.0;
    A.r0 = r0;
    A.dr = dr;
    A.beta0_r = beta0_r;
    A.rho0_r = rho0_r;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 block(32, kMapWarps);
    constexpr long long per = (long long)kMapWarps * kWarpRows;
    auto blocks = [](long long rows) { return (unsigned)((rows + per - 1) / per); };
    if ((long long)(A.ny + 1) * (A.nz + 1) > 0x7fffffffLL * per) {
        set_last_error("mg_base_state_map: too many grid rows");
        return MG_ERR_INVALID_ARG;
    }
    if (sigma || beta0_cell) {
        const long long rows = (long long)A.ny * A.nz;
        MGP_LAUNCH(k_map_cells<<<blocks(rows), block, 0, s>>>(A, rows, sigma, beta0_cell));
    }
    for (int d = 0; d < g->dim; ++d) {
        if (!beta0_face || !beta0_face[d]) continue;
        const long long rows = (long long)(A.ny + (d == 1)) * (A.nz + (d == 2));
        MGP_LAUNCH(k_map_faces<<<blocks(rows), block, 0, s>>>(A, d, rows, beta0_face[d]));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return MG_ERR_CUDA; }
    return MG_OK;
}
