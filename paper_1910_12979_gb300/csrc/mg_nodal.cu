// mg_nodal.cu -- nodal (Q1 finite element) operator, smoother, transfers and FP64 residual.
#include "mg_nodal.cuh"

#include <type_traits>

namespace mgp {

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
    xo[t] = node_jacobi_value<DIM>(L, x, b, t, i, j, k, omega);
}

template <int DIM, typename T>
__global__ void k_node_resid(NodeLevel<T> L, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    r[t] = node_resid_value<DIM>(L, x, b, t, i, j, k);
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
    bc[t] = node_restrict_value<DIM>(F, C, rf, i, j, k);
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
    xf[t] += node_prolong_value<DIM>(F, C, xc, i, j, k);
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
constexpr int kNSlots = 4;

template <typename T>
struct NodePipeSlot {
    T xs[kNTY + 2][kNTX + 2];   // phi, nodes x0-1 .. x0+32, y0-1 .. y0+8
    T ss[kNTY + 1][kNTX + 1];   // sigma of cells x0-1 .. x0+31, y0-1 .. y0+7 (cell plane p)
    T bb[kNTY][kNTX];           // b of the tile
    T iv[kNTY][kNTX];           // 1/diagonal (FP64 levels)
};

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
                    acc = fmadd(sg, ((Sk.xs[bb2][a] + Se.xs[ly][a]) + Se.xs[bb2][lx]) + Se.xs[bb2][a], acc);
                    ssum += sg;
                }
                const T off = acc * (L.ih2 / T(12));
                const T dg = -ssum * (L.ih2 / T(3));
                const T xi = Sk.xs[ly][lx];
                const T bv = Sk.bb[threadIdx.y][threadIdx.x];
                if (RESID) {
                    out[id] = bv - fmadd(dg, xi, off);
                } else {
                    const T inv = has_iv ? Sk.iv[threadIdx.y][threadIdx.x] : recip(dg);
                    out[id] = fmadd(omega * (bv - fmadd(dg, xi, off)), inv, xi);
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
    const int sh = pow2_shift(*scale);
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
            rs = f64_to_f32_pow2(b[t] - (off + d * x[t]), sh);
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

// ------------------------------------- sum-factorised FP64 residual (3-D)
//
// GB300 issues about two FP64 operations per SM per clock, so the FP64
// residual is bound by its FP64 operation count, not by HBM.  With the cell
// sum s_c = (sum of the 8 phi of cell c), the 3-D row of node_row regroups as
//   h^2 (L phi)_I = (1/12) [ sum_c sigma_c s_c - sum_{6 nbrs n} W_In phi_n ]
//                   - (5/12) phi_I sum_c sigma_c
// (the 3 face-adjacent nodes of each cell carry weight 0 in the Q1 row, and
// s_c = phi_I + (face-adjacent) + (the 4 weighted nodes)), where W_In is the
// sum of sigma over the cells that contain the edge I-n.  W and the diagonal
// part are coefficient data, built once per coefficient update (k_node_edges).
// sum_c sigma_c s_c is formed with shared partial sums: per node plane the
// 2x2 phi sums at every cell position, per cell Q = sigma (lower + upper 2x2
// sums), per node the 2x2 sum of Q over each of the two cell planes.  About
// 20 FP64 operations per node instead of about 40 for the direct row.

// per node: cells around the +x, +y, +z edges and the scaled diagonal part
__global__ void k_node_edges(NodeLevel<double> L, NodeEdges E)
{
    const int total = L.Nx * L.Ny * L.Nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.Nx, L.Ny, i, j, k);
    auto sg = [&](int a, int b, int c) -> double {
        int ci, cj, ck;
        if (!cell_ok(a, L.nx, L.bc.lo[0], ci) || !cell_ok(b, L.ny, L.bc.lo[1], cj) || !cell_ok(c, L.nz, L.bc.lo[2], ck))
            return 0.0;
        return L.sigma[((size_t)ck * L.ny + cj) * L.nx + ci];
    };
    const double s00 = sg(i - 1, j - 1, k - 1), s10 = sg(i, j - 1, k - 1), s01 = sg(i - 1, j, k - 1),
                 s11 = sg(i, j, k - 1);
    const double u00 = sg(i - 1, j - 1, k), u10 = sg(i, j - 1, k), u01 = sg(i - 1, j, k), u11 = sg(i, j, k);
    E.w[0][t] = (s10 + s11) + (u10 + u11);   // x-edge (i, i+1): cells of column i
    E.w[1][t] = (s01 + s11) + (u01 + u11);   // y-edge (j, j+1): cells of row j
    E.w[2][t] = (u00 + u10) + (u01 + u11);   // z-edge (k, k+1): cells of plane k
    const double S = ((s00 + s10) + (s01 + s11)) + ((u00 + u10) + (u01 + u11));
    E.dq[t] = node_dirichlet(L, i, j, k, 3) ? 0.0 : -(5.0 / 12.0) * L.ih2 * S;
}

struct NodeSFShared {
    double xs[4][kNTY + 2][kNTX + 2];  // phi node planes (ring), nodes x0-1 .. x0+32, y0-1 .. y0+8
    double ss[2][kNTY + 1][kNTX + 1];  // sigma cell planes (ring), cells x0-1 .. x0+31, y0-1 .. y0+7
    double q[kNTY + 1][kNTX + 1];      // Q of the current cell plane
};

// One fixed grid of kRedBlocks blocks; block b takes an equal contiguous share
// of the (tile, node plane) sequence, tile-major, so the work is balanced to a
// plane and the partial sums are deterministic.
__global__ void __launch_bounds__(kNTX * kNTY, kRedBlocks / 152)
k_node_resid64_sf(NodeLevel<double> L, NodeEdges E, const double* __restrict__ x, const double* __restrict__ b,
                  float* __restrict__ r32, const double* __restrict__ scale, double* __restrict__ partials)
{
    constexpr int TX = kNTX, TY = kNTY, NT = TX * TY, QN = (TX + 1) * (TY + 1), XN = (TX + 2) * (TY + 2);
    __shared__ NodeSFShared sh;
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const int tx_n = (Nx + TX - 1) / TX, ty_n = (Ny + TY - 1) / TY;
    const long long G = (long long)tx_n * ty_n * Nz;
    const long long g0 = G * blockIdx.x / gridDim.x, g1 = G * (blockIdx.x + 1) / gridDim.x;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int rsh = pow2_shift(*scale);
    const double c12 = L.ih2 / 12.0;
    const size_t nplane = (size_t)Nx * Ny, cplane = (size_t)nx * ny;
    float acc = 0.f;

    for (long long g = g0; g < g1;) {
        const int tile = (int)(g / Nz);
        const int z0 = (int)(g - (long long)tile * Nz);
        const int z1 = (int)min((long long)Nz, (long long)z0 + (g1 - g));
        g += z1 - z0;
        const int x0 = (tile % tx_n) * TX, y0 = (tile / tx_n) * TY;

        int ox[2], os[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = tid + e * NT;
            ox[e] = -2;
            if (q < XN) {
                const int ly = q / (TX + 2), lx = q - ly * (TX + 2);
                const int gx = npos(x0 - 1 + lx, Nx, px), gy = npos(y0 - 1 + ly, Ny, py);
                ox[e] = (gx >= 0 && gy >= 0) ? gy * Nx + gx : -1;
            }
            os[e] = -2;
            if (q < QN) {
                const int ly = q / (TX + 1), lx = q - ly * (TX + 1);
                const int gx = npos(x0 - 1 + lx, nx, px), gy = npos(y0 - 1 + ly, ny, py);
                os[e] = (gx >= 0 && gy >= 0) ? gy * nx + gx : -1;
            }
        }
        auto issue_node = [&](int p) {  // node plane p (wrapped when z is periodic, else 0 outside)
            int pn = p;
            bool ok = true;
            if (pn < 0 || pn >= Nz) { if (pz) pn = pn < 0 ? pn + Nz : pn - Nz; else ok = false; }
            const double* xp = x + (ok ? pn * nplane : 0);
            double* dst = &sh.xs[(p + 4) & 3][0][0];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (ox[e] >= -1) ncp_async(dst + tid + e * NT, xp + (ox[e] < 0 ? 0 : ox[e]), ok && ox[e] >= 0, 8);
        };
        auto issue_cell = [&](int p) {  // cell plane p
            int pc = p;
            bool ok = true;
            if (pc < 0 || pc >= nz) { if (pz) pc = pc < 0 ? pc + nz : pc - nz; else ok = false; }
            const double* sp = L.sigma + (ok ? pc * cplane : 0);
            double* dst = &sh.ss[(p + 2) & 1][0][0];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (os[e] >= -1) ncp_async(dst + tid + e * NT, sp + (os[e] < 0 ? 0 : os[e]), ok && os[e] >= 0, 8);
        };
        // 2x2 phi sum of node plane slot s at cell position q (x then y pairs)
        auto bxy = [&](int s, int q) {
            const int qy = q / (TX + 1), qx = q - qy * (TX + 1);
            const double* r0 = &sh.xs[s][qy][qx];
            const double* r1 = &sh.xs[s][qy + 1][qx];
            return (r0[0] + r0[1]) + (r1[0] + r1[1]);
        };
        const int q0 = tid, q1 = tid + NT;  // owned cell positions (q1 valid when < QN)
        double bp0, bp1 = 0.0;

        // prologue: Q of cell plane z0-1 and its 2x2 sums
        issue_node(z0 - 1);
        issue_node(z0);
        issue_cell(z0 - 1);
        cp_async_commit_n();
        cp_async_wait_n<0>();
        __syncthreads();
        issue_node(z0 + 1);
        issue_cell(z0);
        cp_async_commit_n();
        {
            const int sl = (z0 - 1 + 4) & 3, sc = (z0 + 4) & 3, sg = (z0 - 1 + 2) & 1;
            const double a0 = bxy(sl, q0), c0 = bxy(sc, q0);
            (&sh.q[0][0])[q0] = (&sh.ss[sg][0][0])[q0] * (a0 + c0);
            bp0 = c0;
            if (q1 < QN) {
                const double a1 = bxy(sl, q1), c1 = bxy(sc, q1);
                (&sh.q[0][0])[q1] = (&sh.ss[sg][0][0])[q1] * (a1 + c1);
                bp1 = c1;
            }
        }
        __syncthreads();
        const int lx = threadIdx.x, ly = threadIdx.y;
        double qb_prev = (sh.q[ly][lx] + sh.q[ly][lx + 1]) + (sh.q[ly + 1][lx] + sh.q[ly + 1][lx + 1]);
        const int i = x0 + lx, j = y0 + ly;
        const bool own = i < Nx && j < Ny;
        // index of the -x / -y neighbour's edge weight (-1: no such edge)
        const int im = i > 0 ? i - 1 : (px ? Nx - 1 : -1);
        const int jm = j > 0 ? j - 1 : (py ? Ny - 1 : -1);
        double wz_prev = 0.0;
        if (own) {
            const int km = z0 > 0 ? z0 - 1 : (pz ? Nz - 1 : -1);
            if (km >= 0) wz_prev = E.w[2][(size_t)km * nplane + (size_t)j * Nx + i];
        }

        for (int k = z0; k < z1; ++k) {
            cp_async_wait_n<0>();  // node plane k+1 and cell plane k have landed
            __syncthreads();
            if (k + 1 < z1) {
                issue_node(k + 2);
                issue_cell(k + 1);
            }
            cp_async_commit_n();
            {
                const int sn = (k + 1 + 4) & 3, sg = (k + 2) & 1;
                const double c0 = bxy(sn, q0);
                (&sh.q[0][0])[q0] = (&sh.ss[sg][0][0])[q0] * (bp0 + c0);
                bp0 = c0;
                if (q1 < QN) {
                    const double c1 = bxy(sn, q1);
                    (&sh.q[0][0])[q1] = (&sh.ss[sg][0][0])[q1] * (bp1 + c1);
                    bp1 = c1;
                }
            }
            __syncthreads();
            const double qb = (sh.q[ly][lx] + sh.q[ly][lx + 1]) + (sh.q[ly + 1][lx] + sh.q[ly + 1][lx + 1]);
            const double P = qb_prev + qb;
            qb_prev = qb;
            if (own) {
                const size_t row = (size_t)k * nplane + (size_t)j * Nx;
                const double wz = E.w[2][row + i];
                float rs = 0.f;
                if (!node_dirichlet(L, i, j, k, 3)) {
                    const int sk = (k + 4) & 3, sm = (k + 3) & 3, sp = (k + 5) & 3;
                    const double wxp = E.w[0][row + i];
                    const double wxm = im >= 0 ? E.w[0][row + im] : 0.0;
                    const double wyp = E.w[1][row + i];
                    const double wym = jm >= 0 ? E.w[1][(size_t)k * nplane + (size_t)jm * Nx + i] : 0.0;
                    const double xi = sh.xs[sk][ly + 1][lx + 1];
                    double t = P;
                    t = fmadd(-wxm, sh.xs[sk][ly + 1][lx], t);
                    t = fmadd(-wxp, sh.xs[sk][ly + 1][lx + 2], t);
                    t = fmadd(-wym, sh.xs[sk][ly][lx + 1], t);
                    t = fmadd(-wyp, sh.xs[sk][ly + 2][lx + 1], t);
                    t = fmadd(-wz_prev, sh.xs[sm][ly + 1][lx + 1], t);
                    t = fmadd(-wz, sh.xs[sp][ly + 1][lx + 1], t);
                    const double Lx = fmadd(E.dq[row + i], xi, t * c12);
                    rs = f64_to_f32_pow2(b[row + i] - Lx, rsh);
                }
                wz_prev = wz;
                acc = fmaf(rs, rs, acc);
                if (r32) r32[row + i] = rs;
            }
        }
        __syncthreads();  // the next segment's prologue refills the rings
    }
    double a[1] = {(double)acc};
    block_reduce_store<1>(a, partials);
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

// quads per block row and planes per thread of the four-node kernel for a smoother kind
// autotuned kinds of the vectorised nodal kernel: 1..3 one node plane per thread, 5..7 four, 9..11
// eight, with 8/16/32 quads per block row; 0: the launcher's default shape
static int v4_width(int kind)
{
    return kind >= 1 && kind <= 3 ? 4 << kind : kind >= 5 && kind <= 7 ? 4 << (kind - 4)
                                              : kind >= 9 && kind <= 11 ? 4 << (kind - 8) : 0;
}
static int v4_planes(int kind)
{
    return kind >= 1 && kind <= 3 ? 1 : kind >= 5 && kind <= 7 ? 4 : kind >= 9 && kind <= 11 ? 8 : 0;
}

template <typename T>
void node_jacobi(int dim, const NodeLevel<T>& L, const T* x, T* xo, const T* b, T omega, bool tiled, cudaStream_t s,
                 int kind)
{
    if constexpr (std::is_same<T, float>::value) {
        if (tiled && kind != 4 && node_v4_ok(dim, L, x, xo, b)) {
            node_v4(L, x, xo, b, omega, false, s, v4_width(kind), v4_planes(kind));
            return;
        }
    }
    if (node_tiled_ok(dim, L, tiled)) {
        launch_node_tiled<T, false>(L, x, xo, b, omega, s);
    } else if (dim == 2) {
        MGP_LAUNCH(k_jacobi<2, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, xo, b, omega));
    } else {
        MGP_LAUNCH(k_jacobi<3, T><<<nb(nnod(L)), kThreads, 0, s>>>(L, x, xo, b, omega));
    }
}

template <typename T>
void node_resid(int dim, const NodeLevel<T>& L, const T* x, const T* b, T* r, bool tiled, cudaStream_t s, int kind)
{
    if constexpr (std::is_same<T, float>::value) {
        if (tiled && kind != 4 && node_v4_ok(dim, L, x, r, b)) {
            node_v4(L, x, r, b, 0.f, true, s, v4_width(kind), v4_planes(kind));
            return;
        }
    }
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
    if constexpr (std::is_same<T, float>::value) {
        if (node_restrict_v4_ok(dim, F, rf, bc)) {
            node_restrict_v4(F, C, rf, bc, s);
            return;
        }
    }
    if (dim == 2) MGP_LAUNCH(k_node_restrict<2, T><<<nb(nnod(C)), kThreads, 0, s>>>(F, C, rf, bc));
    else MGP_LAUNCH(k_node_restrict<3, T><<<nb(nnod(C)), kThreads, 0, s>>>(F, C, rf, bc));
}

template <typename T>
void node_prolong_add(int dim, const NodeLevel<T>& F, const NodeLevel<T>& C, T* xf, const T* xc, cudaStream_t s)
{
    if constexpr (std::is_same<T, float>::value) {
        if (node_prolong_v4_ok(dim, F, xf, xc)) {
            node_prolong_v4(F, C, xf, xc, s);
            return;
        }
    }
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

void node_edges(const NodeLevel<double>& L, const NodeEdges& E, cudaStream_t s)
{
    MGP_LAUNCH(k_node_edges<<<nb(nnod(L)), kThreads, 0, s>>>(L, E));
}

void node_resid64_sf(const NodeLevel<double>& L, const NodeEdges& E, const double* x, const double* b, float* r32,
                     const double* scale, double* partials, cudaStream_t s)
{
    MGP_LAUNCH(k_node_resid64_sf<<<kRedBlocks, dim3(kNTX, kNTY), 0, s>>>(L, E, x, b, r32, scale, partials));
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
                                 cudaStream_t, int);
template void node_jacobi<double>(int, const NodeLevel<double>&, const double*, double*, const double*, double, bool,
                                  cudaStream_t, int);
template void node_resid<float>(int, const NodeLevel<float>&, const float*, const float*, float*, bool, cudaStream_t,
                                int);
template void node_resid<double>(int, const NodeLevel<double>&, const double*, const double*, double*, bool,
                                 cudaStream_t, int);
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
