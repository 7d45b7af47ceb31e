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

__global__ void k_map_cells(MapArgs A, double* __restrict__ sigma, double* __restrict__ b0c)
{
    const int total = A.nx * A.ny * A.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, A.nx, A.ny, i, j, k);
    const double r = radius(A, (i + 0.5) * A.hx, (j + 0.5) * A.hy, (k + 0.5) * A.hz);
    const double b = interp(A.beta0_r, A.nr, A.r0, A.dr, r);
    if (sigma) sigma[t] = b / interp(A.rho0_r, A.nr, A.r0, A.dr, r);
    if (b0c) b0c[t] = b;
}

__global__ void k_map_faces(MapArgs A, int d, double* __restrict__ out)
{
    const int mx = A.nx + (d == 0), my = A.ny + (d == 1), mz = A.nz + (d == 2);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mx * my * mz) return;
    int i, j, k;
    unflat(t, mx, my, i, j, k);
    const double x = (i + (d == 0 ? 0.0 : 0.5)) * A.hx, y = (j + (d == 1 ? 0.0 : 0.5)) * A.hy,
                 z = (k + (d == 2 ? 0.0 : 0.5)) * A.hz;
    out[t] = interp(A.beta0_r, A.nr, A.r0, A.dr, radius(A, x, y, z));
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
    const long long cells = (long long)A.nx * A.ny * A.nz;
    if (sigma || beta0_cell)
        MGP_LAUNCH(k_map_cells<<<ceil_div(cells, kThreads), kThreads, 0, s>>>(A, sigma, beta0_cell));
    for (int d = 0; d < g->dim; ++d) {
        if (!beta0_face || !beta0_face[d]) continue;
        const long long m = (long long)(A.nx + (d == 0)) * (A.ny + (d == 1)) * (A.nz + (d == 2));
        MGP_LAUNCH(k_map_faces<<<ceil_div(m, kThreads), kThreads, 0, s>>>(A, d, beta0_face[d]));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return MG_ERR_CUDA; }
    return MG_OK;
}
