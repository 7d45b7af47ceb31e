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

namespace mgp {

template <typename T>
struct CoarseArgs {
    int nlev;                          // levels of the sub-cycle; the last is the coarsest
    CellLevel<T> L[kCoarseMaxLevels];
    T* x[kCoarseMaxLevels];
    T* b[kCoarseMaxLevels];            // b[0]: the sub-cycle's right-hand side (read only)
    const double* Minv;
    int Nd, nu1, nu2, order, zero_first;
};

template <int DIM, typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle(CoarseArgs<T> A)
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
