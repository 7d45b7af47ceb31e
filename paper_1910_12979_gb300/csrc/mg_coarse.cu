// mg_coarse.cu -- the coarse end of a cell-centred V-cycle in one CTA.
//
// Below a few thousand cells per level the multigrid kernels are latency-bound:
// each level's zeroing, colour passes, restriction and prolongation cost a
// launch and a dependency gap each, however few cells it touches.  From the
// first level of at most kCoarseCells cells down to the dense bottom solve and
// back, one CTA of 1024 threads does the whole sub-cycle in place -- the same
// steps in the same order as the launched kernels, separated by barriers, on
// the level arrays in global memory (they stay in L2) -- with the per-cell
// arithmetic of mg_cellops.cuh and the warp dot products of dense_row, so its
// result equals the launched sequence bit for bit.
#include "mg_cellops.cuh"
#include "mg_nodal.cuh"

namespace mgp {

template <int DIM, typename T>
__device__ __forceinline__ void coarse_body(const CoarseArgs<T>& A)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    auto cells = [&](int l) { return A.L[l].nx * A.L[l].ny * A.L[l].nz; };
    auto smooth = [&](int l, int nu) {
        const CellLevel<T>& V = A.L[l];
        T* x = A.x[l];
        const T* b = A.b[l];
        const int n = cells(l);
        for (int sweep = 0; sweep < nu; ++sweep)
            for (int color = 0; color < 2; ++color) {
                for (int t = tid; t < n; t += nt) {
                    int i, j, k;
                    unflat(t, V.nx, V.ny, i, j, k);
                    if (((i + j + k) & 1) == color) x[t] = gs_value<DIM>(V, x, b, i, j, k);
                }
                __syncthreads();
            }
    };
    for (int l = 0; l < A.nlev - 1; ++l) {
        if (l > 0 || A.zero_first) {
            for (int t = tid; t < cells(l); t += nt) A.x[l][t] = T(0);
            __syncthreads();
        }
        smooth(l, A.nu1);
        const CellLevel<T>& C = A.L[l + 1];
        for (int t = tid; t < cells(l + 1); t += nt) {
            int ci, cj, ck;
            unflat(t, C.nx, C.ny, ci, cj, ck);
            A.b[l + 1][t] = restrict_value<DIM>(A.L[l], A.x[l], A.b[l], ci, cj, ck);
        }
        __syncthreads();
    }
    {
        const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5, last = A.nlev - 1;
        for (int r = warp; r < A.Nd; r += nw) {
            const double s = dense_row(A.Minv, A.Nd, A.b[last], r, lane);
            if (lane == 0) A.x[last][r] = from_f64<T>(s);
        }
        __syncthreads();
    }
    for (int l = A.nlev - 2; l >= 0; --l) {
        const CellLevel<T>& F = A.L[l];
        for (int t = tid; t < cells(l); t += nt) {
            int i, j, k;
            unflat(t, F.nx, F.ny, i, j, k);
            A.x[l][t] += prolong_value<DIM>(F, A.L[l + 1], A.x[l + 1], i, j, k, A.order);
        }
        __syncthreads();
        smooth(l, A.nu2);
    }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle(CoarseArgs<T> A)
{
    coarse_body<DIM, T>(A);
}

// Batched coarse ends: CTA i runs solve i's while its run flag is set.
__global__ void __launch_bounds__(1024) k_coarse_batch(const CoarseArgs<float>* __restrict__ A,
                                                       const int* __restrict__ run)
{
    if (!run[blockIdx.x]) return;
    coarse_body<3, float>(A[blockIdx.x]);
}

void coarse_cycle_batch(const CoarseArgs<float>* A, int count, const int* run, cudaStream_t s)
{
    MGP_LAUNCH(k_coarse_batch<<<count, 1024, 0, s>>>(A, run));
}

template <typename T>
void coarse_cycle(int dim, int nlev, const CellLevel<T>* L, T* const* x, T* const* b, const double* Minv, int Nd,
                  int nu1, int nu2, int order, bool zero_first, cudaStream_t s)
{
    CoarseArgs<T> A{};
    A.nlev = nlev;
    for (int l = 0; l < nlev; ++l) {
        A.L[l] = L[l];
        A.x[l] = x[l];
        A.b[l] = b[l];
    }
    A.Minv = Minv;
    A.Nd = Nd;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.order = order;
    A.zero_first = zero_first ? 1 : 0;
    if (dim == 2) MGP_LAUNCH(k_coarse_cycle<2, T><<<1, 1024, 0, s>>>(A));
    else MGP_LAUNCH(k_coarse_cycle<3, T><<<1, 1024, 0, s>>>(A));
}

template void coarse_cycle<float>(int, int, const CellLevel<float>*, float* const*, float* const*, const double*, int,
                                  int, int, int, bool, cudaStream_t);
template void coarse_cycle<double>(int, int, const CellLevel<double>*, double* const*, double* const*,
                                   const double*, int, int, int, int, bool, cudaStream_t);

}  // namespace mgp

namespace mgp {

// The same for the nodal V-cycle: from the first level of at most
// kCoarseNodes stored nodes down to the dense bottom solve and back, one CTA
// runs the launched sequence -- zeroing, damped Jacobi sweeps ping-ponging
// between x and the level's temp vector (copied back after an odd count),
// residual, full-weighting restriction, prolongation -- with the per-node
// functions of mg_nodal.cuh, so the result equals the launched kernels'.
template <typename T>
struct NodeCoarseArgs {
    int nlev;
    NodeLevel<T> L[kCoarseMaxLevels];
    T* x[kCoarseMaxLevels];
    T* b[kCoarseMaxLevels];            // b[0]: the sub-cycle's right-hand side (read only)
    T* t[kCoarseMaxLevels];            // Jacobi temp
    T* r[kCoarseMaxLevels];            // residual
    const double* Minv;
    int Nd, nu1, nu2, zero_first;
    T omega;
};

template <int DIM, typename T>
__global__ void __launch_bounds__(1024) k_node_coarse_cycle(NodeCoarseArgs<T> A)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    auto nodes = [&](int l) { return A.L[l].Nx * A.L[l].Ny * A.L[l].Nz; };
    auto smooth = [&](int l, int nu) {
        const NodeLevel<T>& V = A.L[l];
        const T* b = A.b[l];
        const int n = nodes(l);
        for (int sweep = 0; sweep < nu; ++sweep) {
            const T* src = (sweep & 1) ? A.t[l] : A.x[l];
            T* dst = (sweep & 1) ? A.x[l] : A.t[l];
            for (int q = tid; q < n; q += nt) {
                int i, j, k;
                unflat(q, V.Nx, V.Ny, i, j, k);
                dst[q] = node_jacobi_value<DIM>(V, src, b, q, i, j, k, A.omega);
            }
            __syncthreads();
        }
        if (nu & 1) {
            for (int q = tid; q < n; q += nt) A.x[l][q] = A.t[l][q];
            __syncthreads();
        }
    };
    for (int l = 0; l < A.nlev - 1; ++l) {
        const NodeLevel<T>& V = A.L[l];
        if (l > 0 || A.zero_first) {
            for (int q = tid; q < nodes(l); q += nt) A.x[l][q] = T(0);
            __syncthreads();
        }
        smooth(l, A.nu1);
        for (int q = tid; q < nodes(l); q += nt) {
            int i, j, k;
            unflat(q, V.Nx, V.Ny, i, j, k);
            A.r[l][q] = node_resid_value<DIM>(V, A.x[l], A.b[l], q, i, j, k);
        }
        __syncthreads();
        const NodeLevel<T>& C = A.L[l + 1];
        for (int q = tid; q < nodes(l + 1); q += nt) {
            int i, j, k;
            unflat(q, C.Nx, C.Ny, i, j, k);
            A.b[l + 1][q] = node_restrict_value<DIM>(V, C, A.r[l], i, j, k);
        }
        __syncthreads();
    }
    {
        const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5, last = A.nlev - 1;
        for (int r = warp; r < A.Nd; r += nw) {
            const double s = dense_row(A.Minv, A.Nd, A.b[last], r, lane);
            if (lane == 0) A.x[last][r] = from_f64<T>(s);
        }
        __syncthreads();
    }
    for (int l = A.nlev - 2; l >= 0; --l) {
        const NodeLevel<T>& F = A.L[l];
        for (int q = tid; q < nodes(l); q += nt) {
            int i, j, k;
            unflat(q, F.Nx, F.Ny, i, j, k);
            if (!node_dirichlet(F, i, j, k, DIM)) A.x[l][q] += node_prolong_value<DIM>(F, A.L[l + 1], A.x[l + 1], i, j, k);
        }
        __syncthreads();
        smooth(l, A.nu2);
    }
}

template <typename T>
void node_coarse_cycle(int dim, int nlev, const NodeLevel<T>* L, T* const* x, T* const* b, T* const* t, T* const* r,
                       const double* Minv, int Nd, int nu1, int nu2, T omega, bool zero_first, cudaStream_t s)
{
    NodeCoarseArgs<T> A{};
    A.nlev = nlev;
    for (int l = 0; l < nlev; ++l) {
        A.L[l] = L[l];
        A.x[l] = x[l];
        A.b[l] = b[l];
        A.t[l] = t[l];
        A.r[l] = r[l];
    }
    A.Minv = Minv;
    A.Nd = Nd;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.omega = omega;
    A.zero_first = zero_first ? 1 : 0;
    if (dim == 2) MGP_LAUNCH(k_node_coarse_cycle<2, T><<<1, 1024, 0, s>>>(A));
    else MGP_LAUNCH(k_node_coarse_cycle<3, T><<<1, 1024, 0, s>>>(A));
}

template void node_coarse_cycle<float>(int, int, const NodeLevel<float>*, float* const*, float* const*,
                                       float* const*, float* const*, const double*, int, int, int, float, bool,
                                       cudaStream_t);
template void node_coarse_cycle<double>(int, int, const NodeLevel<double>*, double* const*, double* const*,
                                        double* const*, double* const*, const double*, int, int, int, double, bool,
                                        cudaStream_t);

}  // namespace mgp
