// mg_rotation.cu -- Coriolis and centrifugal accelerations of the rotating
// velocity equation (S5): a = -2 Omega x U - Omega x (Omega x r), r = x - centre,
// accumulated as F += alpha a at cell centres.
//
// FP64 throughout; the kernel is bound by the FP64 pipe, so the centrifugal
// term uses the identity -Omega x (Omega x r) = |Omega|^2 r - Omega (Omega . r)
// (9 operations instead of 12) and the factor -2 is folded into Omega once.
// One thread per cell; each cell's components are read before any is written,
// so F may alias U.
#include "mg_device.cuh"

#include "../../include/mg.h"

namespace mgp {

struct RotArgs {
    int dim, nx, ny, nz;
    double hx, hy, hz;
    double w[3], m2w[3], w2;     // Omega, -2 Omega, |Omega|^2
    double r0[3];                // (0.5 h - centre) per axis: r_d = i_d h_d + r0_d
    double alpha;
    int centrifugal;
};

__global__ void k_rotation(RotArgs A, const double* __restrict__ U0, const double* __restrict__ U1,
                           const double* __restrict__ U2, double* F0, double* F1, double* F2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= A.nx) return;
    const size_t id = ((size_t)k * A.ny + j) * A.nx + i;
    const double u0 = U0[id], u1 = U1[id], u2 = A.dim == 3 ? U2[id] : 0.0;
    // -2 Omega x U
    double a0 = fmadd(A.m2w[1], u2, -(A.m2w[2] * u1));
    double a1 = fmadd(A.m2w[2], u0, -(A.m2w[0] * u2));
    double a2 = fmadd(A.m2w[0], u1, -(A.m2w[1] * u0));
    if (A.centrifugal) {
        const double r0 = fmadd((double)i, A.hx, A.r0[0]), r1 = fmadd((double)j, A.hy, A.r0[1]);
        const double r2 = A.dim == 3 ? fmadd((double)k, A.hz, A.r0[2]) : 0.0;
        const double wr = fmadd(A.w[0], r0, fmadd(A.w[1], r1, A.w[2] * r2));
        a0 += fmadd(A.w2, r0, -(A.w[0] * wr));
        a1 += fmadd(A.w2, r1, -(A.w[1] * wr));
        a2 += fmadd(A.w2, r2, -(A.w[2] * wr));
    }
    F0[id] = fmadd(A.alpha, a0, F0[id]);
    F1[id] = fmadd(A.alpha, a1, F1[id]);
    if (A.dim == 3) F2[id] = fmadd(A.alpha, a2, F2[id]);
}

}  // namespace mgp

using namespace mgp;

extern "C" mg_status mg_rotation_forces(const mg_geometry* g, const double omega[3], const double center[3],
                                        int centrifugal, double alpha, const double* const U[3],
                                        double* const F[3], void* stream)
{
    if (!g || (g->dim != 2 && g->dim != 3) || !omega || (centrifugal && !center) || !U || !F) {
        set_last_error("mg_rotation_forces: invalid argument");
        return MG_ERR_INVALID_ARG;
    }
    for (int d = 0; d < g->dim; ++d)
        if (!U[d] || !F[d] || g->n[d] < 1) {
            set_last_error("mg_rotation_forces: missing velocity or force component");
            return MG_ERR_INVALID_ARG;
        }
    RotArgs A{};
    A.dim = g->dim;
    A.nx = g->n[0];
    A.ny = g->n[1];
    A.nz = g->dim == 3 ? g->n[2] : 1;
    A.hx = g->h[0];
    A.hy = g->h[1];
    A.hz = g->dim == 3 ? g->h[2] : 1.0;
    for (int d = 0; d < 3; ++d) {
        A.w[d] = omega[d];
        A.m2w[d] = -2.0 * omega[d];
        const double h = d == 0 ? A.hx : d == 1 ? A.hy : A.hz;
        A.r0[d] = (d < g->dim && centrifugal) ? 0.5 * h - center[d] : 0.0;
    }
    A.w2 = omega[0] * omega[0] + omega[1] * omega[1] + omega[2] * omega[2];
    A.alpha = alpha;
    A.centrifugal = centrifugal ? 1 : 0;
    const dim3 block(256), grid(ceil_div(A.nx, 256), A.ny, A.nz);
    MGP_LAUNCH(k_rotation<<<grid, block, 0, (cudaStream_t)stream>>>(A, U[0], U[1], g->dim == 3 ? U[2] : nullptr,
                                                                     F[0], F[1], g->dim == 3 ? F[2] : nullptr));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}
