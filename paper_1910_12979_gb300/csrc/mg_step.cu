// mg_step.cu -- one time step around the two projections (S2-S3): face
// velocities from the cell velocities, MAC projection of them, upwind
// advection of the cell velocities by the projected face velocities (plus the
// rotation accelerations of S5 when an angular velocity is given), nodal
// projection of the result.  The projections are mg_project calls on the
// caller's two resident handles; the two kernels here are FP64 and bound by the
// FP64 pipe (about 2 and 40 operations per face and per cell).
#include "mg_device.cuh"

#include "../../include/mg.h"

#include <string.h>

namespace mgp {

namespace {

struct StepGrid {
    int dim, n[3];
    int lo[3], hi[3];
    double ih[3];
};

__device__ __forceinline__ size_t cidx(const StepGrid& G, int i, int j, int k)
{
    return ((size_t)k * G.n[1] + j) * G.n[0] + i;
}

// cell c moved by s along d: true and the wrapped index when that cell exists
__device__ __forceinline__ bool shift(const StepGrid& G, int d, int c, int s, int& out)
{
    out = c + s;
    if (out >= 0 && out < G.n[d]) return true;
    if (G.lo[d] != BCP) return false;
    out = out < 0 ? out + G.n[d] : out - G.n[d];
    return true;
}

// faces of direction D: mean of the normal velocity in the two cells beside the
// face; periodic faces use the wrap neighbour, wall faces carry 0, outflow
// (Dirichlet) faces the interior cell's value
template <int D>
__global__ void k_face_avg(StepGrid G, const double* __restrict__ Ud, double* __restrict__ Uf)
{
    const int mx = G.n[0] + (D == 0), my = G.n[1] + (D == 1), mz = G.n[2] + (D == 2);
    const int fi = blockIdx.x * blockDim.x + threadIdx.x, fj = blockIdx.y, fk = blockIdx.z;
    if (fi >= mx) return;
    int hi[3] = {fi, fj, fk}, lo[3] = {fi, fj, fk};
    const int f = hi[D];
    bool has_hi = f < G.n[D];
    int q;
    const bool has_lo = shift(G, D, f, -1, q);
    lo[D] = q;
    if (!has_hi && G.lo[D] == BCP) { hi[D] = 0; has_hi = true; }
    double v;
    if (has_hi && has_lo) {
        v = 0.5 * (Ud[cidx(G, lo[0], lo[1], lo[2])] + Ud[cidx(G, hi[0], hi[1], hi[2])]);
    } else {
        const int bc = has_hi ? G.lo[D] : G.hi[D];
        const int* c = has_hi ? hi : lo;
        v = bc == BCN ? 0.0 : Ud[cidx(G, c[0], c[1], c[2])];
    }
    Uf[((size_t)fk * my + fj) * mx + fi] = v;
}

// Unew_c = U_c - dt (U_adv . grad) U_c for every component, upwind values on
// the faces (zero gradient where the upwind cell is outside a boundary)
template <int DIM>
__global__ void k_advect(StepGrid G, double dt, const double* __restrict__ F0, const double* __restrict__ F1,
                         const double* __restrict__ F2, const double* __restrict__ U0, const double* __restrict__ U1,
                         const double* __restrict__ U2, double* __restrict__ N0, double* __restrict__ N1,
                         double* __restrict__ N2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= G.n[0]) return;
    const double* Uc[3] = {U0, U1, U2};
    double* Nc[3] = {N0, N1, N2};
    const size_t id = cidx(G, i, j, k);
    double qc[3], a[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < DIM; ++c) qc[c] = Uc[c][id];
    const int cc[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const int mx = G.n[0] + (d == 0), my = G.n[1] + (d == 1);
        int fl[3] = {i, j, k};
        const double* Fd = d == 0 ? F0 : (d == 1 ? F1 : F2);
        const double ul = Fd[((size_t)fl[2] * my + fl[1]) * mx + fl[0]];
        fl[d] += 1;
        const double uh = Fd[((size_t)fl[2] * my + fl[1]) * mx + fl[0]];
        int q, nb[3];
        const bool hl = shift(G, d, cc[d], -1, q);
        nb[0] = i; nb[1] = j; nb[2] = k; nb[d] = q;
        const size_t il = hl ? cidx(G, nb[0], nb[1], nb[2]) : id;
        const bool hh = shift(G, d, cc[d], +1, q);
        nb[0] = i; nb[1] = j; nb[2] = k; nb[d] = q;
        const size_t ih = hh ? cidx(G, nb[0], nb[1], nb[2]) : id;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double qlo = Uc[c][il], qhi = Uc[c][ih];
            const double th = uh >= 0.0 ? qc[c] : qhi, tl = ul >= 0.0 ? qlo : qc[c];
            a[c] = fmadd(uh * (th - qc[c]) - ul * (tl - qc[c]), G.ih[d], a[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) Nc[c][id] = fmadd(-dt, a[c], qc[c]);
}

}  // namespace

}  // namespace mgp

using namespace mgp;

extern "C" mg_status mg_step(mg_handle* mac, mg_handle* nodal, const double* const U[3], double* const Unew[3],
                             double* const Uadv[3], const mg_beta0* beta0, const double* S, double dt,
                             const double omega[3], const double center[3], int centrifugal, double tol,
                             mg_stats stats[2])
{
    if (!mac || !nodal || !U || !Unew || !Uadv || !beta0 || !S || !(dt >= 0.0)) {
        set_last_error("mg_step: invalid argument");
        return MG_ERR_INVALID_ARG;
    }
    mg_geometry gm, gn;
    mg_bc bc, bcn;
    cudaStream_t s = nullptr, sn = nullptr;
    handle_info(mac, &gm, &bc, &s);
    handle_info(nodal, &gn, &bcn, &sn);
    bool same = gm.loc == MG_LOC_CELL && gn.loc == MG_LOC_NODAL && gm.dim == gn.dim && s == sn;
    for (int d = 0; d < gm.dim; ++d)
        same = same && gm.n[d] == gn.n[d] && gm.h[d] == gn.h[d] && bc.lo[d] == bcn.lo[d] && bc.hi[d] == bcn.hi[d];
    if (!same) {
        set_last_error("mg_step: needs a MAC (cell) handle and a nodal handle of the same grid, boundaries and stream");
        return MG_ERR_INVALID_ARG;
    }
    const int dim = gm.dim;
    for (int d = 0; d < dim; ++d)
        if (!U[d] || !Unew[d] || !Uadv[d] || U[d] == Unew[d]) {
            set_last_error("mg_step: U, Unew and Uadv need every component, and Unew must not alias U");
            return MG_ERR_INVALID_ARG;
        }
    StepGrid G{};
    G.dim = dim;
    for (int d = 0; d < 3; ++d) {
        G.n[d] = d < dim ? gm.n[d] : 1;
        G.lo[d] = d < dim ? bc.lo[d] : MG_BC_NEUMANN;
        G.hi[d] = d < dim ? bc.hi[d] : MG_BC_NEUMANN;
        G.ih[d] = d < dim ? 1.0 / gm.h[d] : 0.0;
    }
    // face velocities from U^n
    for (int d = 0; d < dim; ++d) {
        const int mx = G.n[0] + (d == 0), my = G.n[1] + (d == 1), mz = G.n[2] + (d == 2);
        const dim3 grid(ceil_div(mx, 128), my, mz);
        if (d == 0) MGP_LAUNCH(k_face_avg<0><<<grid, 128, 0, s>>>(G, U[0], Uadv[0]));
        else if (d == 1) MGP_LAUNCH(k_face_avg<1><<<grid, 128, 0, s>>>(G, U[1], Uadv[1]));
        else MGP_LAUNCH(k_face_avg<2><<<grid, 128, 0, s>>>(G, U[2], Uadv[2]));
    }
    mg_stats local[2];
    memset(local, 0, sizeof local);
    mg_status rc = mg_project(mac, Uadv, beta0, S, nullptr, tol, &local[0]);
    if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED) return rc;
    // U* = U^n - dt (U_adv . grad) U^n (+ dt a_rotation(U^n))
    {
        const dim3 grid(ceil_div(G.n[0], 128), G.n[1], G.n[2]);
        if (dim == 2)
            MGP_LAUNCH(k_advect<2><<<grid, 128, 0, s>>>(G, dt, Uadv[0], Uadv[1], nullptr, U[0], U[1], nullptr, Unew[0],
                                                       Unew[1], nullptr));
        else
            MGP_LAUNCH(k_advect<3><<<grid, 128, 0, s>>>(G, dt, Uadv[0], Uadv[1], Uadv[2], U[0], U[1], U[2], Unew[0],
                                                       Unew[1], Unew[2]));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    if (omega) {
        const mg_status r = mg_rotation_forces(&gm, omega, center, centrifugal, dt, U, Unew, (void*)s);
        if (r != MG_OK) return r;
    }
    const mg_status rc2 = mg_project(nodal, Unew, beta0, S, nullptr, tol, &local[1]);
    if (stats) {
        stats[0] = local[0];
        stats[1] = local[1];
    }
    if (rc2 != MG_OK) return rc2;
    return rc;
}
