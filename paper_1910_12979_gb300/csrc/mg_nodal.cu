// mg_nodal.cu -- nodal (Q1 finite element) projection kernels.
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
#include "mg_device.cuh"

namespace mgp {

__device__ __forceinline__ bool cell_ok(int c, int n, int bc, int& w)
{
    if (c >= 0 && c < n) { w = c; return true; }
    if (bc != BCP) return false;
    w = c < 0 ? c + n : c - n;
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
            acc += sg * (phi(a, b, k) + phi(a, j, e) + phi(i, b, e) + phi(a, b, e));
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
            acc += sg * ((phi(a, j, 0) + phi(i, b, 0)) * T(0.5) + phi(a, b, 0));
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

// ----------------------------------------------------------------- setup

template <int DIM>
__global__ void k_coarsen_sigma(NodeLevel<double> F, NodeLevel<double> C, double* __restrict__ sc)
{
    const int total = C.nx * C.ny * C.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, C.nx, C.ny, i, j, k);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < (1 << DIM); ++q) {
        const int a = 2 * i + (q & 1), b = 2 * j + ((q >> 1) & 1), c = DIM == 3 ? 2 * k + ((q >> 2) & 1) : 0;
        s += F.sigma[((size_t)c * F.ny + b) * F.nx + a];
    }
    sc[t] = s / (1 << DIM);
}

// The diagonal of node row (i,j,k) alone: node_row's dg, same order of sums.
template <int DIM>
__device__ __forceinline__ double node_dg(const NodeLevel<double>& L, int i, int j, int k)
{
    double ssum = 0.0;
#pragma unroll
    for (int c = 0; c < (1 << DIM); ++c) {
        const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1, sz = (c & 4) ? 1 : -1;
        int ci, cj, ck = 0;
        if (!cell_ok(sx > 0 ? i : i - 1, L.nx, L.bc.lo[0], ci)) continue;
        if (!cell_ok(sy > 0 ? j : j - 1, L.ny, L.bc.lo[1], cj)) continue;
        if (DIM == 3 && !cell_ok(sz > 0 ? k : k - 1, L.nz, L.bc.lo[2], ck)) continue;
        ssum += L.sigma[((size_t)ck * L.ny + cj) * L.nx + ci];
    }
    return DIM == 3 ? -ssum * (L.ih2 / 3.0) : -ssum * (L.ih2 * 2.0 / 3.0);
}

template <int DIM>
__global__ void k_node_invdiag(NodeLevel<double> L, double* __restrict__ invd)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    invd[t] = node_dirichlet(L, i, j, k, DIM) ? 0.0 : recip(node_dg<DIM>(L, i, j, k));
}

// ------------------------------------------------------------- smoothing

// damped Jacobi: xo = x + omega (b - L x) / diag; Dirichlet nodes stay 0
template <int DIM, typename T>
__global__ void k_jacobi(NodeLevel<T> L, const T* __restrict__ x, T* __restrict__ xo, const T* __restrict__ b,
                         T omega)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    if (node_dirichlet(L, i, j, k, DIM)) { xo[t] = T(0); return; }
    T off, dg;
    node_row<DIM>(L, i, j, k, NodePhi<T>{x, L.Nx, L.Ny}, off, dg);
    const T xi = x[t];
    const T id = L.invd ? L.invd[t] : recip(dg);
    xo[t] = xi + omega * (b[t] - (off + dg * xi)) * id;
}

template <int DIM, typename T>
__global__ void k_node_resid(NodeLevel<T> L, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    if (node_dirichlet(L, i, j, k, DIM)) { r[t] = T(0); return; }
    T off, dg;
    node_row<DIM>(L, i, j, k, NodePhi<T>{x, L.Nx, L.Ny}, off, dg);
    r[t] = b[t] - (off + dg * x[t]);
}

// fine lattice position q on an axis: wrapped when periodic; false outside
__device__ __forceinline__ bool fine_pos(int q, int n, int bc, int& w)
{
    if (bc == BCP) { w = wrap(q, n); return true; }
    if (q < 0 || q > n) return false;
    w = q;
    return true;
}

// full weighting, R = 2^-dim P^T
template <int DIM, typename T>
__global__ void k_node_restrict(NodeLevel<T> F, NodeLevel<T> C, const T* __restrict__ rf, T* __restrict__ bc)
{
    const int total = C.Nx * C.Ny * C.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, C.Nx, C.Ny, i, j, k);
    if (node_dirichlet(C, i, j, k, DIM)) { bc[t] = T(0); return; }
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
                s += wz * wy * wx * rf[((size_t)c * F.Ny + b) * F.Nx + a];
            }
        }
    }
    bc[t] = s * (T(1) / T(1 << DIM));
}

// trilinear prolongation and correction
template <int DIM, typename T>
__global__ void k_node_prolong(NodeLevel<T> F, NodeLevel<T> C, T* __restrict__ xf, const T* __restrict__ xc)
{
    const int total = F.Nx * F.Ny * F.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, F.Nx, F.Ny, i, j, k);
    if (node_dirichlet(F, i, j, k, DIM)) return;
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
                s += w * xc[((size_t)q[2] * C.Ny + q[1]) * C.Nx + q[0]];
            }
    xf[t] += s;
}

// ------------------------------------------------------ tiled node sweeps
//
// The Jacobi sweep and the residual of k_jacobi / k_node_resid, one CTA per
// 32 x 8 tile of node columns marching through a chunk of z-planes.  A 4-slot
// shared-memory ring receives, two planes ahead of use and by cp.async, the
// phi plane with a 1-node halo, the sigma plane of the cells around the tile's
// nodes (0 outside the domain), b and (FP64) the inverse diagonal, so phi,
// sigma and b are read and the result written once per node while the HBM
// latency of later planes overlaps the arithmetic.  The cell loop visits the
// cells in node_row's order; a missing cell adds 0 * (...), which leaves both
// sums unchanged: the results equal k_jacobi's / k_node_resid's.  3-D only.
constexpr int kNTX = 32, kNTY = 8, kNSlots = 4;

template <typename T>
struct NodePipeSlot {
    T xs[kNTY + 2][kNTX + 2];   // phi, nodes x0-1 .. x0+32, y0-1 .. y0+8
    T ss[kNTY + 1][kNTX + 1];   // sigma of cells x0-1 .. x0+31, y0-1 .. y0+7 (cell plane p)
    T bb[kNTY][kNTX];           // b of the tile
    T iv[kNTY][kNTX];           // 1/diagonal (FP64 levels)
};

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

template <typename T, bool RESID>
__global__ void __launch_bounds__(kNTX * kNTY)
k_node_tiled(NodeLevel<T> L, const T* __restrict__ x, T* __restrict__ out, const T* __restrict__ b, T omega, int kz)
{
    constexpr int TX = kNTX, TY = kNTY, NT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NodePipeSlot<T>* slot = reinterpret_cast<NodePipeSlot<T>*>(smem_raw);
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * kz, z1 = min(z0 + kz, Nz);
    const int tid = threadIdx.y * TX + threadIdx.x;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const bool has_iv = !RESID && L.invd != nullptr;
    const size_t nplane = (size_t)Nx * Ny, cplane = (size_t)nx * ny;

    // plane-independent copy offsets (-1: outside the domain -> zero fill)
    int ox[2], os[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int q = tid + e * NT;
        ox[e] = -2;
        if (q < (TX + 2) * (TY + 2)) {
            const int ly = q / (TX + 2), lx = q - ly * (TX + 2);
            const int gx = npos(x0 - 1 + lx, Nx, px), gy = npos(y0 - 1 + ly, Ny, py);
            ox[e] = (gx >= 0 && gy >= 0) ? gy * Nx + gx : -1;
        }
        os[e] = -2;
        if (q < (TX + 1) * (TY + 1)) {
            const int ly = q / (TX + 1), lx = q - ly * (TX + 1);
            const int gx = npos(x0 - 1 + lx, nx, px), gy = npos(y0 - 1 + ly, ny, py);
            os[e] = (gx >= 0 && gy >= 0) ? gy * nx + gx : -1;
        }
    }
    const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
    const bool own = i < Nx && j < Ny;
    const int ob = own ? j * Nx + i : 0;

    // stage node plane p (phi, b, 1/diag) and cell plane p (sigma); p may be
    // -1 or Nz (wrapped when z is periodic, else zero)
    auto issue = [&](int p) {
        if (p >= -1 && p <= Nz) {
            NodePipeSlot<T>& S = slot[(p + kNSlots) % kNSlots];
            int pn = p, pc = p;
            bool nok = true, cok = true;
            if (pn < 0 || pn >= Nz) { if (pz) pn = pn < 0 ? pn + Nz : pn - Nz; else nok = false; }
            if (pc < 0 || pc >= nz) { if (pz) pc = pc < 0 ? pc + nz : pc - nz; else cok = false; }
            const T* xp = x + (nok ? pn * nplane : 0);
            const T* sp = L.sigma + (cok ? pc * cplane : 0);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int q = tid + e * NT;
                if (ox[e] >= -1) ncp_async(&S.xs[0][0] + q, xp + (ox[e] < 0 ? 0 : ox[e]), nok && ox[e] >= 0, sizeof(T));
                if (os[e] >= -1) ncp_async(&S.ss[0][0] + q, sp + (os[e] < 0 ? 0 : os[e]), cok && os[e] >= 0, sizeof(T));
            }
            const bool bok = own && p >= 0 && p < Nz;
            ncp_async(&S.bb[threadIdx.y][threadIdx.x], b + (bok ? p * nplane + ob : 0), bok, sizeof(T));
            if (has_iv)
                ncp_async(&S.iv[threadIdx.y][threadIdx.x], L.invd + (bok ? p * nplane + ob : 0), bok, sizeof(T));
        }
        cp_async_commit_n();
    };

    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);
    issue(z0 + 2);
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    for (int k = z0; k < z1; ++k) {
        cp_async_wait_n<1>();  // planes <= k + 1 have landed
        __syncthreads();
        if (own) {
            const size_t id = (size_t)k * nplane + ob;
            if (node_dirichlet(L, i, j, k, 3)) {
                out[id] = T(0);
            } else {
                const NodePipeSlot<T>& Sk = slot[(k + kNSlots) % kNSlots];
                const NodePipeSlot<T>& Sm = slot[(k - 1 + kNSlots) % kNSlots];
                const NodePipeSlot<T>& Sp = slot[(k + 1 + kNSlots) % kNSlots];
                T acc = T(0), ssum = T(0);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1, sz = (c & 4) ? 1 : -1;
                    const NodePipeSlot<T>& Sc = sz > 0 ? Sk : Sm;   // cell plane k or k-1
                    const NodePipeSlot<T>& Se = sz > 0 ? Sp : Sm;   // node plane k+sz
                    const T sg = Sc.ss[ly + (sy > 0 ? 0 : -1)][lx + (sx > 0 ? 0 : -1)];
                    const int a = lx + sx, bb2 = ly + sy;
                    acc += sg * (Sk.xs[bb2][a] + Se.xs[ly][a] + Se.xs[bb2][lx] + Se.xs[bb2][a]);
                    ssum += sg;
                }
                const T off = acc * (L.ih2 / T(12));
                const T dg = -ssum * (L.ih2 / T(3));
                const T xi = Sk.xs[ly][lx];
                const T bv = Sk.bb[threadIdx.y][threadIdx.x];
                if (RESID) {
                    out[id] = bv - (off + dg * xi);
                } else {
                    const T inv = has_iv ? Sk.iv[threadIdx.y][threadIdx.x] : recip(dg);
                    out[id] = xi + omega * (bv - (off + dg * xi)) * inv;
                }
            }
        }
        __syncthreads();
        issue(k + 3);
    }
    cp_async_wait_n<0>();
}

// -------------------------------------------------------- FP64 residuals

template <int DIM, bool HAS_DIAG>
__global__ void k_node_resid64(NodeLevel<double> L, const double* __restrict__ x, const double* __restrict__ b,
                               float* __restrict__ r32, const double* __restrict__ scale,
                               double* __restrict__ partials)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const double inv = 1.0 / *scale;
    float acc = 0.f;
    const NodePhi<double> ph{x, L.Nx, L.Ny};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int i, j, k;
        unflat(t, L.Nx, L.Ny, i, j, k);
        float rs = 0.f;
        if (!node_dirichlet(L, i, j, k, DIM)) {
            double off, dg;
            node_row<DIM>(L, i, j, k, ph, off, dg);
            const double d = HAS_DIAG ? L.diag[t] : dg;
            rs = (float)((b[t] - (off + d * x[t])) * inv);
        }
        acc = fmaf(rs, rs, acc);
        if (r32) r32[t] = rs;
    }
    double a[1] = {(double)acc};
    block_reduce_store<1>(a, partials);
}

template <int DIM>
__global__ void k_node_diag(NodeLevel<double> L, double* __restrict__ diag)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    diag[t] = node_dirichlet(L, i, j, k, DIM) ? 0.0 : node_dg<DIM>(L, i, j, k);
}

template <int DIM>
__global__ void k_node_apply64(NodeLevel<double> L, const double* __restrict__ x, double* __restrict__ out)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    if (node_dirichlet(L, i, j, k, DIM)) { out[t] = 0.0; return; }
    double off, dg;
    node_row<DIM>(L, i, j, k, NodePhi<double>{x, L.Nx, L.Ny}, off, dg);
    out[t] = off + dg * x[t];
}

// ------------------------------------------------------ RHS / projection

struct CPtr3 {
    const double* p[3];
};
struct MPtr3n {
    double* p[3];
};

// f_I = D_N(beta0 U)_I - sum_c (beta0 S)_c / 2^dim; partials {sum f, sum lump^2, sum f^2}
template <int DIM>
__global__ void k_node_rhs(NodeLevel<double> L, double h, CPtr3 U, const double* __restrict__ b0,
                           const double* __restrict__ S, double* __restrict__ f, double* __restrict__ partials)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const double wdiv = 1.0 / ((1 << (DIM - 1)) * h), wl = 1.0 / (1 << DIM);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int i, j, k;
        unflat(t, L.Nx, L.Ny, i, j, k);
        double v = 0.0, lump = 0.0;
        if (!node_dirichlet(L, i, j, k, DIM)) {
            for (int c = 0; c < (1 << DIM); ++c) {
                const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1, sz = (c & 4) ? 1 : -1;
                int ci, cj, ck = 0;
                if (!cell_ok(sx > 0 ? i : i - 1, L.nx, L.bc.lo[0], ci)) continue;
                if (!cell_ok(sy > 0 ? j : j - 1, L.ny, L.bc.lo[1], cj)) continue;
                if (DIM == 3 && !cell_ok(sz > 0 ? k : k - 1, L.nz, L.bc.lo[2], ck)) continue;
                const size_t id = ((size_t)ck * L.ny + cj) * L.nx + ci;
                const double bb = b0[id];
                double dv = sx * U.p[0][id] + sy * U.p[1][id];
                if (DIM == 3) dv += sz * U.p[2][id];
                v += bb * dv * wdiv;
                lump += bb * S[id] * wl;
            }
            v -= lump;
        }
        if (f) f[t] = v;
        acc[0] += v;
        acc[1] += lump * lump;
        acc[2] += v * v;
    }
    block_reduce_store<3>(acc, partials);
}

// Tiled 3-D version of k_node_rhs.  Per z-plane the cells around a 32 x 8 node
// tile get W = beta0 U (3 components) and beta0 S computed once into shared
// memory; each node then forms D_N from signed sums of its 8 cells (additions
// only) and the lumped source from their sum.  Cells outside a non-periodic
// boundary hold 0 (natural boundary condition).  The fixed kRedBlocks grid
// strides over (tile, z-chunk) work items, so the reduction stays deterministic.
struct NodeRhsShared {
    double w[2][4][kNTY + 1][kNTX + 1];  // [plane ring][Wx, Wy, Wz, beta0 S][y][x]
};

__global__ void __launch_bounds__(kNTX * kNTY)
k_node_rhs_tiled(NodeLevel<double> L, double h, CPtr3 U, const double* __restrict__ b0, const double* __restrict__ S,
                 double* __restrict__ f, double* __restrict__ partials, int kz)
{
    constexpr int TX = kNTX, TY = kNTY;
    __shared__ NodeRhsShared sh;
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const int tx_n = (Nx + TX - 1) / TX, ty_n = (Ny + TY - 1) / TY, tz_n = (Nz + kz - 1) / kz;
    const int items = tx_n * ty_n * tz_n;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const double wdiv = 1.0 / (4.0 * h), wl = 1.0 / 8.0;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int bx = it % tx_n, by = (it / tx_n) % ty_n, bz = it / (tx_n * ty_n);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * kz, z1 = min(z0 + kz, Nz);
        auto load = [&](int c) {  // cell plane c -> ring slot
            int gz = c;
            bool zok = true;
            if (gz < 0 || gz >= nz) { if (pz) gz = gz < 0 ? gz + nz : gz - nz; else zok = false; }
            const int slot = (c + 2) & 1;
            for (int q = tid; q < (TX + 1) * (TY + 1); q += TX * TY) {
                const int ly = q / (TX + 1), lx = q - ly * (TX + 1);
                int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
                bool ok = zok;
                if (gx < 0 || gx >= nx) { if (px) gx = gx < 0 ? gx + nx : gx - nx; else ok = false; }
                if (gy < 0 || gy >= ny) { if (py) gy = gy < 0 ? gy + ny : gy - ny; else ok = false; }
                if (gx >= nx || gy >= ny) ok = false;
                double w0 = 0.0, w1 = 0.0, w2 = 0.0, ws = 0.0;
                if (ok) {
                    const size_t id = ((size_t)gz * ny + gy) * nx + gx;
                    const double bb = b0[id];
                    w0 = bb * U.p[0][id];
                    w1 = bb * U.p[1][id];
                    w2 = bb * U.p[2][id];
                    ws = bb * S[id];
                }
                sh.w[slot][0][ly][lx] = w0;
                sh.w[slot][1][ly][lx] = w1;
                sh.w[slot][2][ly][lx] = w2;
                sh.w[slot][3][ly][lx] = ws;
            }
        };
        load(z0 - 1);
        for (int k = z0; k < z1; ++k) {
            load(k);
            __syncthreads();
            const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
            if (i < Nx && j < Ny) {
                const size_t id = ((size_t)k * Ny + j) * Nx + i;
                double v = 0.0, lump = 0.0;
                if (!node_dirichlet(L, i, j, k, 3)) {
                    const int lx = threadIdx.x, ly = threadIdx.y;  // cell (i-1, j-1) is at (lx, ly)
                    const int sp = (k + 2) & 1, sm = (k + 1) & 1;   // cell planes k and k-1
                    auto W = [&](int s, int q, int a, int b) { return sh.w[s][q][ly + b][lx + a]; };
                    const double dx = (W(sp, 0, 1, 1) + W(sp, 0, 1, 0) + W(sm, 0, 1, 1) + W(sm, 0, 1, 0)) -
                                      (W(sp, 0, 0, 1) + W(sp, 0, 0, 0) + W(sm, 0, 0, 1) + W(sm, 0, 0, 0));
                    const double dy = (W(sp, 1, 1, 1) + W(sp, 1, 0, 1) + W(sm, 1, 1, 1) + W(sm, 1, 0, 1)) -
                                      (W(sp, 1, 1, 0) + W(sp, 1, 0, 0) + W(sm, 1, 1, 0) + W(sm, 1, 0, 0));
                    const double dz = (W(sp, 2, 1, 1) + W(sp, 2, 0, 1) + W(sp, 2, 1, 0) + W(sp, 2, 0, 0)) -
                                      (W(sm, 2, 1, 1) + W(sm, 2, 0, 1) + W(sm, 2, 1, 0) + W(sm, 2, 0, 0));
                    lump = ((W(sp, 3, 1, 1) + W(sp, 3, 0, 1)) + (W(sp, 3, 1, 0) + W(sp, 3, 0, 0)) +
                            (W(sm, 3, 1, 1) + W(sm, 3, 0, 1)) + (W(sm, 3, 1, 0) + W(sm, 3, 0, 0))) * wl;
                    v = (dx + dy + dz) * wdiv - lump;
                }
                if (f) f[id] = v;
                acc[0] += v;
                acc[1] += lump * lump;
                acc[2] += v * v;
            }
            __syncthreads();
        }
    }
    block_reduce_store<3>(acc, partials);
}

// U_c -= (sigma_c / beta0_c) G_N(phi)_c
template <int DIM>
__global__ void k_node_project(NodeLevel<double> L, double h, const double* __restrict__ phi,
                               const double* __restrict__ b0, MPtr3n U)
{
    const int total = L.nx * L.ny * L.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.nx, L.ny, i, j, k);
    double g[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < (1 << DIM); ++c) {
        const int a = node_nb(i + (c & 1), L.Nx, L.bc.lo[0]);
        const int b = node_nb(j + ((c >> 1) & 1), L.Ny, L.bc.lo[1]);
        const int e = DIM == 3 ? node_nb(k + ((c >> 2) & 1), L.Nz, L.bc.lo[2]) : 0;
        const double v = phi[((size_t)e * L.Ny + b) * L.Nx + a];
        g[0] += (c & 1) ? v : -v;
        g[1] += (c & 2) ? v : -v;
        if (DIM == 3) g[2] += (c & 4) ? v : -v;
    }
    const double w = L.sigma[t] / b0[t] / ((1 << (DIM - 1)) * h);
    for (int d = 0; d < DIM; ++d) U.p[d][t] -= w * g[d];
}

template <int DIM, typename T>
__global__ void k_node_dense_assemble(NodeLevel<T> L, double* __restrict__ A, int lda)
{
    const int N = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * N) return;
    const int row = t / N, col = t % N;
    int i, j, k;
    unflat(row, L.Nx, L.Ny, i, j, k);
    double v;
    if (node_dirichlet(L, i, j, k, DIM)) {
        v = (row == col) ? 1.0 : 0.0;
    } else {
        T off, dg;
        const int Nx = L.Nx, Ny = L.Ny;
        node_row<DIM>(L, i, j, k, [&](int a, int b, int c) { return ((c * Ny + b) * Nx + a) == col ? T(1) : T(0); },
                      off, dg);
        v = (double)off + (row == col ? (double)dg : 0.0);
    }
    A[(size_t)row * lda + col] = v;
}

template <int DIM, typename T>
__global__ void k_node_zero_dirichlet(NodeLevel<T> L, T* __restrict__ x)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    if (node_dirichlet(L, i, j, k, DIM)) x[t] = T(0);
}

// ================================================================ launchers

static inline int nb(long long n) { return ceil_div(n, kThreads); }
template <typename T>
static inline long long nnod(const NodeLevel<T>& L) { return (long long)L.Nx * L.Ny * L.Nz; }

void node_coarsen_sigma(int dim, const NodeLevel<double>& F, const NodeLevel<double>& C, double* sc, cudaStream_t s)
{
    long long n = (long long)C.nx * C.ny * C.nz;
    if (dim == 2) MGP_LAUNCH(k_coarsen_sigma<2><<<nb(n), kThreads, 0, s>>>(F, C, sc));
    else MGP_LAUNCH(k_coarsen_sigma<3><<<nb(n), kThreads, 0, s>>>(F, C, sc));
}

void node_invdiag(int dim, const NodeLevel<double>& L, double* invd, cudaStream_t s)
{
    if (dim == 2) MGP_LAUNCH(k_node_invdiag<2><<<nb(nnod(L)), kThreads, 0, s>>>(L, invd));
    else MGP_LAUNCH(k_node_invdiag<3><<<nb(nnod(L)), kThreads, 0, s>>>(L, invd));
}

template <typename T>
static bool node_tiled_ok(int dim, const NodeLevel<T>& L, bool allow)
{
    return allow && dim == 3 && L.Nx >= kNTX && L.Ny >= kNTY && L.Nz >= 4;
}

template <typename T>
static dim3 node_tiled_grid(const NodeLevel<T>& L, int& kz)
{
    const long long tx = (L.Nx + kNTX - 1) / kNTX, ty = (L.Ny + kNTY - 1) / kNTY;
    kz = (int)((tx * ty * L.Nz + 152 * 7 - 1) / (152 * 7));
    kz = kz < 4 ? 4 : kz;
    return dim3((unsigned)tx, (unsigned)ty, (unsigned)((L.Nz + kz - 1) / kz));
}

template <typename T, bool RESID>
static void launch_node_tiled(const NodeLevel<T>& L, const T* x, T* out, const T* b, T omega, cudaStream_t s)
{
    const size_t smem = kNSlots * sizeof(NodePipeSlot<T>);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_node_tiled<T, RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    int kz;
    const dim3 g = node_tiled_grid(L, kz);
    MGP_LAUNCH(k_node_tiled<T, RESID><<<g, dim3(kNTX, kNTY), smem, s>>>(L, x, out, b, omega, kz));
}

template <typename T>
void node_jacobi(int dim, const NodeLevel<T>& L, const T* x, T* xo, const T* b, T omega, bool tiled, cudaStream_t s)
{
    if (node_tiled_ok(dim, L, tiled)) {
        launch_node_tiled<T, false>(L, x, xo, b, omega, s);
    } else if (dim == 2) {
        MGP_LAUNCH(k_jacobi<2, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, xo, b, omega));
    } else {
        MGP_LAUNCH(k_jacobi<3, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, xo, b, omega));
    }
}

template <typename T>
void node_resid(int dim, const NodeLevel<T>& L, const T* x, const T* b, T* r, bool tiled, cudaStream_t s)
{
    if (node_tiled_ok(dim, L, tiled)) {
        launch_node_tiled<T, true>(L, x, r, b, T(0), s);
    } else if (dim == 2) {
        MGP_LAUNCH(k_node_resid<2, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, b, r));
    } else {
        MGP_LAUNCH(k_node_resid<3, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, b, r));
    }
}

template <typename T>
void node_restrict(int dim, const NodeLevel<T>& F, const NodeLevel<T>& C, const T* rf, T* bc, cudaStream_t s)
{
    if (dim == 2) MGP_LAUNCH(k_node_restrict<2, T><<<nb(nnod(C)), kThreads, 0, s>>>(F, C, rf, bc));
    else MGP_LAUNCH(k_node_restrict<3, T><<<nb(nnod(C)), kThreads, 0, s>>>(F, C, rf, bc));
}

template <typename T>
void node_prolong_add(int dim, const NodeLevel<T>& F, const NodeLevel<T>& C, T* xf, const T* xc, cudaStream_t s)
{
    if (dim == 2) MGP_LAUNCH(k_node_prolong<2, T><<<nb(nnod(F)), kThreads, 0, s>>>(F, C, xf, xc));
    else MGP_LAUNCH(k_node_prolong<3, T><<<nb(nnod(F)), kThreads, 0, s>>>(F, C, xf, xc));
}

void node_resid64(int dim, const NodeLevel<double>& L, const double* x, const double* b, float* r32,
                  const double* scale, double* partials, cudaStream_t s)
{
    if (dim == 2) {
        if (L.diag) MGP_LAUNCH(k_node_resid64<2, true><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
        else MGP_LAUNCH(k_node_resid64<2, false><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
    } else {
        if (L.diag) MGP_LAUNCH(k_node_resid64<3, true><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
        else MGP_LAUNCH(k_node_resid64<3, false><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
    }
}

void node_diag(int dim, const NodeLevel<double>& L, double* diag, cudaStream_t s)
{
    if (dim == 2) MGP_LAUNCH(k_node_diag<2><<<nb(nnod(L)), kThreads, 0, s>>>(L, diag));
    else MGP_LAUNCH(k_node_diag<3><<<nb(nnod(L)), kThreads, 0, s>>>(L, diag));
}

void node_apply64(int dim, const NodeLevel<double>& L, const double* x, double* out, cudaStream_t s)
{
    if (dim == 2) MGP_LAUNCH(k_node_apply64<2><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, out));
    else MGP_LAUNCH(k_node_apply64<3><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, out));
}

void node_rhs(int dim, const NodeLevel<double>& L, double h, const double* const U[3], const double* b0,
              const double* S, double* f, double* partials, cudaStream_t s)
{
    CPtr3 u{{U[0], U[1], dim == 3 ? U[2] : nullptr}};
    if (dim == 3 && L.Nx >= kNTX && L.Ny >= kNTY) {
        // about 4 work items per block
        const long long tiles = (long long)((L.Nx + kNTX - 1) / kNTX) * ((L.Ny + kNTY - 1) / kNTY);
        int kz = (int)((tiles * L.Nz + kRedBlocks * 4 - 1) / (kRedBlocks * 4));
        kz = kz < 4 ? 4 : kz;
        MGP_LAUNCH(k_node_rhs_tiled<<<kRedBlocks, dim3(kNTX, kNTY), 0, s>>>(L, h, u, b0, S, f, partials, kz));
        return;
    }
    if (dim == 2) MGP_LAUNCH(k_node_rhs<2><<<kRedBlocks, kThreads, 0, s>>>(L, h, u, b0, S, f, partials));
    else MGP_LAUNCH(k_node_rhs<3><<<kRedBlocks, kThreads, 0, s>>>(L, h, u, b0, S, f, partials));
}

void node_project(int dim, const NodeLevel<double>& L, double h, const double* phi, const double* b0,
                  double* const U[3], cudaStream_t s)
{
    MPtr3n u{{U[0], U[1], dim == 3 ? U[2] : nullptr}};
    long long n = (long long)L.nx * L.ny * L.nz;
    if (dim == 2) MGP_LAUNCH(k_node_project<2><<<nb(n), kThreads, 0, s>>>(L, h, phi, b0, u));
    else MGP_LAUNCH(k_node_project<3><<<nb(n), kThreads, 0, s>>>(L, h, phi, b0, u));
}

template <typename T>
void node_dense_assemble(int dim, const NodeLevel<T>& L, double* A, int lda, cudaStream_t s)
{
    long long N = nnod(L);
    if (dim == 2) MGP_LAUNCH(k_node_dense_assemble<2, T><<<nb(N * N), kThreads, 0, s>>>(L, A, lda));
    else MGP_LAUNCH(k_node_dense_assemble<3, T><<<nb(N * N), kThreads, 0, s>>>(L, A, lda));
}

template <typename T>
void node_zero_dirichlet(int dim, const NodeLevel<T>& L, T* x, cudaStream_t s)
{
    if (dim == 2) MGP_LAUNCH(k_node_zero_dirichlet<2, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x));
    else MGP_LAUNCH(k_node_zero_dirichlet<3, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x));
}

template void node_jacobi<float>(int, const NodeLevel<float>&, const float*, float*, const float*, float, bool,
                                 cudaStream_t);
template void node_jacobi<double>(int, const NodeLevel<double>&, const double*, double*, const double*, double, bool,
                                  cudaStream_t);
template void node_resid<float>(int, const NodeLevel<float>&, const float*, const float*, float*, bool, cudaStream_t);
template void node_resid<double>(int, const NodeLevel<double>&, const double*, const double*, double*, bool,
                                 cudaStream_t);
template void node_restrict<float>(int, const NodeLevel<float>&, const NodeLevel<float>&, const float*, float*,
                                   cudaStream_t);
template void node_restrict<double>(int, const NodeLevel<double>&, const NodeLevel<double>&, const double*, double*,
                                    cudaStream_t);
template void node_prolong_add<float>(int, const NodeLevel<float>&, const NodeLevel<float>&, float*, const float*,
                                      cudaStream_t);
template void node_prolong_add<double>(int, const NodeLevel<double>&, const NodeLevel<double>&, double*,
                                       const double*, cudaStream_t);
template void node_dense_assemble<float>(int, const NodeLevel<float>&, double*, int, cudaStream_t);
template void node_dense_assemble<double>(int, const NodeLevel<double>&, double*, int, cudaStream_t);
template void node_zero_dirichlet<float>(int, const NodeLevel<float>&, float*, cudaStream_t);
template void node_zero_dirichlet<double>(int, const NodeLevel<double>&, double*, cudaStream_t);

}  // namespace mgp
