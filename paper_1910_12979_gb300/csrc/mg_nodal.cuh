// mg_nodal.cuh -- helpers shared by the nodal (Q1 finite element) kernels.
//
// phi lives on nodes, sigma = beta0/rho is constant per cell, U is cell-centred.
// With equal spacing h the Q1 operator at node I, assembled on the fly from the
// sigma of the 2^dim cells touching I (cells outside a non-periodic boundary
// contribute nothing: the natural boundary condition), is
//   3-D: h^2 (L phi)_I = sum_cells sigma_c [ -phi_I/3
//            + (phi_{2 axes moved} x3 + phi_{opposite corner}) / 12 ]
//        (face-adjacent corners have zero weight: 21 non-zeros at constant sigma)
//   2-D: h^2 (L phi)_I = sum_cells sigma_c [ -2 phi_I/3 + (phi_x + phi_y)/6 + phi_diag/3 ]
// written as (L phi)_I = off_I + diag_I phi_I.  Dirichlet nodes hold 0 and are not
// unknowns; periodic node n_d is node 0.
#pragma once

#include "mg_device.cuh"

namespace mgp {

__device__ __forceinline__ bool cell_ok(int c, int n, int bc, int& w)
{
    if (c >= 0 && c < n) { w = c; return true; }
    if (bc != BCP) return false;
    w = c < 0 ? c + n : c - n;
    return true;
}

// fine node position q on an axis of n cells: wrapped when periodic, absent outside 0 .. n otherwise
__device__ __forceinline__ bool fine_pos(int q, int n, int bc, int& w)
{
    if (bc == BCP) { w = wrap(q, n); return true; }
    if (q < 0 || q > n) return false;
    w = q;
    return true;
}

__device__ __forceinline__ int node_nb(int p, int N, int bc)  // periodic wrap of a node index
{
    return bc == BCP ? wrap(p, N) : p;
}

template <typename T>
__device__ __forceinline__ bool node_dirichlet(const NodeLevel<T>& L, int i, int j, int k, int dim)
{
    if ((L.bc.lo[0] == BCD && i == 0) || (L.bc.hi[0] == BCD && i == L.nx)) return true;
    if ((L.bc.lo[1] == BCD && j == 0) || (L.bc.hi[1] == BCD && j == L.ny)) return true;
    if (dim == 3 && ((L.bc.lo[2] == BCD && k == 0) || (L.bc.hi[2] == BCD && k == L.nz))) return true;
    return false;
}

template <int DIM, typename T, typename Phi>
__device__ __forceinline__ void node_row(const NodeLevel<T>& L, int i, int j, int k, const Phi& phi, T& off, T& dg)
{
    T acc = T(0), ssum = T(0);
    if (DIM == 3) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1, sz = (c & 4) ? 1 : -1;
            int ci, cj, ck;
            if (!cell_ok(sx > 0 ? i : i - 1, L.nx, L.bc.lo[0], ci)) continue;
            if (!cell_ok(sy > 0 ? j : j - 1, L.ny, L.bc.lo[1], cj)) continue;
            if (!cell_ok(sz > 0 ? k : k - 1, L.nz, L.bc.lo[2], ck)) continue;
            const T sg = L.sigma[((size_t)ck * L.ny + cj) * L.nx + ci];
            const int a = node_nb(i + sx, L.Nx, L.bc.lo[0]);
            const int b = node_nb(j + sy, L.Ny, L.bc.lo[1]);
            const int e = node_nb(k + sz, L.Nz, L.bc.lo[2]);
            acc = fmadd(sg, ((phi(a, b, k) + phi(a, j, e)) + phi(i, b, e)) + phi(a, b, e), acc);
            ssum += sg;
        }
        off = acc * (L.ih2 / T(12));
        dg = -ssum * (L.ih2 / T(3));
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1;
            int ci, cj;
            if (!cell_ok(sx > 0 ? i : i - 1, L.nx, L.bc.lo[0], ci)) continue;
            if (!cell_ok(sy > 0 ? j : j - 1, L.ny, L.bc.lo[1], cj)) continue;
            const T sg = L.sigma[(size_t)cj * L.nx + ci];
            const int a = node_nb(i + sx, L.Nx, L.bc.lo[0]);
            const int b = node_nb(j + sy, L.Ny, L.bc.lo[1]);
            acc = fmadd(sg, fmadd(phi(a, j, 0) + phi(i, b, 0), T(0.5), phi(a, b, 0)), acc);
            ssum += sg;
        }
        off = acc * (L.ih2 / T(3));
        dg = -ssum * (L.ih2 * T(2) / T(3));
    }
}

template <typename T>
struct NodePhi {
    const T* p;
    int Nx, Ny;
    __device__ __forceinline__ T operator()(int i, int j, int k) const { return p[((size_t)k * Ny + j) * Nx + i]; }
};

// Per-node arithmetic shared by the plain kernels and the one-CTA coarse
// cycle, so both compute the same bits.  t is the flat index of (i, j, k).

// damped Jacobi value: x + omega (b - L x) / diag; Dirichlet nodes 0
template <int DIM, typename T>
__device__ __forceinline__ T node_jacobi_value(const NodeLevel<T>& L, const T* x, const T* b, size_t t, int i, int j,
                                               int k, T omega)
{
    if (node_dirichlet(L, i, j, k, DIM)) return T(0);
    T off, dg;
    node_row<DIM>(L, i, j, k, NodePhi<T>{x, L.Nx, L.Ny}, off, dg);
    const T xi = x[t];
    const T id = L.invd ? L.invd[t] : recip(dg);
    return fmadd(omega * (b[t] - fmadd(dg, xi, off)), id, xi);
}

// residual b - L x; Dirichlet nodes 0
template <int DIM, typename T>
__device__ __forceinline__ T node_resid_value(const NodeLevel<T>& L, const T* x, const T* b, size_t t, int i, int j,
                                              int k)
{
    if (node_dirichlet(L, i, j, k, DIM)) return T(0);
    T off, dg;
    node_row<DIM>(L, i, j, k, NodePhi<T>{x, L.Nx, L.Ny}, off, dg);
    return b[t] - fmadd(dg, x[t], off);
}

// full weighting R = 2^-dim P^T at coarse node (i, j, k); Dirichlet nodes 0
template <int DIM, typename T>
__device__ __forceinline__ T node_restrict_value(const NodeLevel<T>& F, const NodeLevel<T>& C, const T* rf, int i,
                                                 int j, int k)
{
    if (node_dirichlet(C, i, j, k, DIM)) return T(0);
    T s = T(0);
    for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz) {
        int c = 0;
        if (DIM == 3 && !fine_pos(2 * k + oz, F.nz, F.bc.lo[2], c)) continue;
        const T wz = (oz == 0) ? T(1) : T(0.5);
        for (int oy = -1; oy <= 1; ++oy) {
            int b;
            if (!fine_pos(2 * j + oy, F.ny, F.bc.lo[1], b)) continue;
            const T wy = (oy == 0) ? T(1) : T(0.5);
            for (int ox = -1; ox <= 1; ++ox) {
                int a;
                if (!fine_pos(2 * i + ox, F.nx, F.bc.lo[0], a)) continue;
                const T wx = (ox == 0) ? T(1) : T(0.5);
                s = fmadd(wz * wy * wx, rf[((size_t)c * F.Ny + b) * F.Nx + a], s);
            }
        }
    }
    return s * (T(1) / T(1 << DIM));
}

// trilinear prolongation of the coarse correction to fine node (i, j, k)
// (callers leave Dirichlet nodes unchanged)
template <int DIM, typename T>
__device__ __forceinline__ T node_prolong_value(const NodeLevel<T>& F, const NodeLevel<T>& C, const T* xc, int i,
                                                int j, int k)
{
    int lo[3] = {i >> 1, j >> 1, k >> 1}, cnt[3] = {1 + (i & 1), 1 + (j & 1), DIM == 3 ? 1 + (k & 1) : 1};
    const int Nc[3] = {C.Nx, C.Ny, C.Nz};
    T s = T(0);
    for (int c = 0; c < cnt[2]; ++c)
        for (int b = 0; b < cnt[1]; ++b)
            for (int a = 0; a < cnt[0]; ++a) {
                int q[3] = {lo[0] + a, lo[1] + b, lo[2] + c};
                T w = T(1);
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    if (cnt[d] == 2) w *= T(0.5);
                    if (C.bc.lo[d] == BCP && q[d] >= Nc[d]) q[d] -= Nc[d];
                }
                s = fmadd(w, xc[((size_t)q[2] * C.Ny + q[1]) * C.Nx + q[0]], s);
            }
    return s;
}

// tile of the shared-memory nodal kernels (nodes in x, y)
constexpr int kNTX = 32, kNTY = 8;

__device__ __forceinline__ void cp_async_commit_n() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ncp_async(void* smem, const void* gmem, bool valid, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? bytes : 0;
    if (bytes == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}

__device__ __forceinline__ int npos(int g, int n, bool periodic)
{
    if (g >= 0 && g < n) return g;
    if (!periodic) return -1;
    return g < 0 ? g + n : g - n;
}

static inline int nb(long long n) { return ceil_div(n, kThreads); }
template <typename T>
static inline long long nnod(const NodeLevel<T>& L) { return (long long)L.Nx * L.Ny * L.Nz; }

}  // namespace mgp
