// mg_cellops.cuh -- per-cell arithmetic of the cell-centred (MAC) system shared
// by every kernel that evaluates it: the row of the operator, one Gauss-Seidel
// update, the residual averaged over a coarse cell's children, and the
// prolongation of a coarse correction.  Kernels that differ only in how they
// stage data or map threads call these, so they compute identical bits.
#pragma once

#include "mg_device.cuh"

namespace mgp {

// off and diag of row (i,j,k); phi(ii,jj,kk) returns the neighbour value.
template <int DIM, typename T, typename Phi>
__device__ __forceinline__ void cell_row(const CellLevel<T>& L, int i, int j, int k, const Phi& phi, T& off, T& dg)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    off = T(0);
    dg = T(0);
    {
        const size_t r = ((size_t)k * ny + j) * (nx + 1) + i;
        const T bl = L.bx[r], bh = L.bx[r + 1];
        if (i > 0) { off = fmadd(bl, phi(i - 1, j, k), off); dg += bl; }
        else if (L.bc.lo[0] == BCP) { off = fmadd(bl, phi(nx - 1, j, k), off); dg += bl; }
        else if (L.bc.lo[0] == BCD) { dg += T(2) * bl; }
        if (i < nx - 1) { off = fmadd(bh, phi(i + 1, j, k), off); dg += bh; }
        else if (L.bc.hi[0] == BCP) { off = fmadd(bh, phi(0, j, k), off); dg += bh; }
        else if (L.bc.hi[0] == BCD) { dg += T(2) * bh; }
    }
    {
        const size_t r = ((size_t)k * (ny + 1) + j) * nx + i;
        const T bl = L.by[r], bh = L.by[r + nx];
        if (j > 0) { off = fmadd(bl, phi(i, j - 1, k), off); dg += bl; }
        else if (L.bc.lo[1] == BCP) { off = fmadd(bl, phi(i, ny - 1, k), off); dg += bl; }
        else if (L.bc.lo[1] == BCD) { dg += T(2) * bl; }
        if (j < ny - 1) { off = fmadd(bh, phi(i, j + 1, k), off); dg += bh; }
        else if (L.bc.hi[1] == BCP) { off = fmadd(bh, phi(i, 0, k), off); dg += bh; }
        else if (L.bc.hi[1] == BCD) { dg += T(2) * bh; }
    }
    if (DIM == 3) {
        const size_t r = ((size_t)k * ny + j) * nx + i;
        const size_t pl = (size_t)nx * ny;
        const T bl = L.bz[r], bh = L.bz[r + pl];
        if (k > 0) { off = fmadd(bl, phi(i, j, k - 1), off); dg += bl; }
        else if (L.bc.lo[2] == BCP) { off = fmadd(bl, phi(i, j, nz - 1), off); dg += bl; }
        else if (L.bc.lo[2] == BCD) { dg += T(2) * bl; }
        if (k < nz - 1) { off = fmadd(bh, phi(i, j, k + 1), off); dg += bh; }
        else if (L.bc.hi[2] == BCP) { off = fmadd(bh, phi(i, j, 0), off); dg += bh; }
        else if (L.bc.hi[2] == BCD) { dg += T(2) * bh; }
    }
}

template <typename T>
struct GlobalPhi {
    const T* p;
    int nx, ny;
    __device__ __forceinline__ T operator()(int i, int j, int k) const { return p[((size_t)k * ny + j) * nx + i]; }
};

struct UnitPhi {  // phi = e_col
    int col, nx, ny;
    __device__ __forceinline__ double operator()(int i, int j, int k) const
    {
        return (((k * ny + j) * nx + i) == col) ? 1.0 : 0.0;
    }
};

template <typename T>
__device__ __forceinline__ T inv_diag(const CellLevel<T>& L, int idx, T dg)
{
    return L.invd ? L.invd[idx] : recip(dg);
}

// Gauss-Seidel value of cell (i,j,k): x = (off - b) / diag
template <int DIM, typename T>
__device__ __forceinline__ T gs_value(const CellLevel<T>& L, const T* x, const T* b, int i, int j, int k)
{
    T off, dg;
    cell_row<DIM>(L, i, j, k, GlobalPhi<T>{x, L.nx, L.ny}, off, dg);
    const size_t t = ((size_t)k * L.ny + j) * L.nx + i;
    return (off - b[t]) * inv_diag(L, (int)t, dg);
}

// residual b - L x averaged over the 2^dim children of coarse cell (ci,cj,ck):
// x pairs, then y, then z
template <int DIM, typename T>
__device__ __forceinline__ T restrict_value(const CellLevel<T>& F, const T* x, const T* b, int ci, int cj, int ck)
{
    const GlobalPhi<T> ph{x, F.nx, F.ny};
    T r[1 << DIM];
#pragma unroll
    for (int q = 0; q < (1 << DIM); ++q) {
        const int i = 2 * ci + (q & 1), j = 2 * cj + ((q >> 1) & 1), k = DIM == 3 ? 2 * ck + ((q >> 2) & 1) : 0;
        T off, dg;
        cell_row<DIM>(F, i, j, k, ph, off, dg);
        const size_t id = ((size_t)k * F.ny + j) * F.nx + i;
        r[q] = b[id] - fmadd(-dg, x[id], off);
    }
    T s = (r[0] + r[1]) + (r[2] + r[3]);
    if (DIM == 3) s = s + ((r[4] + r[5]) + (r[6] + r[7]));
    return s * (T(1) / T(1 << DIM));
}

// prolongation of coarse xc to fine cell (i,j,k): piecewise constant (order 0)
// or linear (order 1, weights 3/4 and 1/4 per axis, see lin1d)
template <int DIM, typename T>
__device__ __forceinline__ T prolong_value(const CellLevel<T>& F, const CellLevel<T>& C, const T* xc, int i, int j,
                                           int k, int order)
{
    auto X = [&](int a, int b2, int c) { return xc[((size_t)c * C.ny + b2) * C.nx + a]; };
    if (order == 0) return X(i >> 1, j >> 1, DIM == 3 ? (k >> 1) : 0);
    const Lin1D lx = lin1d(i, C.nx, F.bc.lo[0], F.bc.hi[0]);
    const Lin1D ly = lin1d(j, C.ny, F.bc.lo[1], F.bc.hi[1]);
    const T w1 = T(0.75), w2 = T(0.25);
    const T ax = w2 * T(lx.sq), ay = w2 * T(ly.sq);
    auto plane = [&](int c) {
        const T lo = fmadd(ax, X(lx.q, ly.p, c), w1 * X(lx.p, ly.p, c));
        const T hi = fmadd(ax, X(lx.q, ly.q, c), w1 * X(lx.p, ly.q, c));
        return fmadd(ay, hi, w1 * lo);
    };
    if (DIM == 2) return plane(0);
    const Lin1D lz = lin1d(k, C.nz, F.bc.lo[2], F.bc.hi[2]);
    return fmadd(w2 * T(lz.sq), plane(lz.q), w1 * plane(lz.p));
}

}  // namespace mgp
