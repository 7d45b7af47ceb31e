// mg_nodal_rhs.cu -- right-hand side and velocity update of the nodal projection.
#include "mg_nodal.cuh"

namespace mgp {

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

// Tiled 3-D version of k_node_rhs with shared partial sums.  Per cell plane
// the cells around a 32 x 8 node tile get W = beta0 U (3 components) and
// beta0 S once (4 products per cell); then per plane the pair sums that the
// node terms share are formed once: y-pairs of W_x at every cell column,
// x-pairs of W_y, W_z and beta0 S at every node column.  A node then needs,
// per cell plane, one difference for each of dx and dy and one pair sum for
// the z and source terms; the plane below is carried in registers.  Cells
// outside a non-periodic boundary hold 0 (natural boundary condition).  About
// 24 FP64 operations per node instead of about 41 for the 8-cell form.  The
// fixed kRedBlocks grid splits the (tile, node plane) sequence into equal
// contiguous shares, so the reduction is deterministic and balanced.
template <typename C>
struct NodeRhsShared {
    C w[4][kNTY + 1][kNTX + 1];  // Wx, Wy, Wz, beta0 S of cells x0-1 .. x0+31, y0-1 .. y0+7
    C ya[kNTY][kNTX + 1];        // Wx(cell col, row ly) + Wx(cell col, row ly+1)
    C xa[3][kNTY + 1][kNTX];     // Wy, Wz, beta0 S: (col lx) + (col lx+1)
};

// C: the arithmetic type.  double for the right-hand side of the solve; float
// for the post-projection diagnostic of the (approximate) nodal projection,
// whose FP64 inputs are rounded to binary32 on the integer pipe as they are
// loaded (f must then be null).  The partial sums are accumulated in FP64.
template <typename C>
__global__ void __launch_bounds__(kNTX * kNTY, 4)
k_node_rhs_tiled(NodeLevel<double> L, double h, CPtr3 U, const double* __restrict__ b0, const double* __restrict__ S,
                 double* __restrict__ f, double* __restrict__ partials)
{
    constexpr int TX = kNTX, TY = kNTY, NT = TX * TY, QN = (TX + 1) * (TY + 1);
    static_assert(QN <= 2 * NT, "each thread stages at most two cells of a plane");
    __shared__ NodeRhsShared<C> sh;
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const int tx_n = (Nx + TX - 1) / TX, ty_n = (Ny + TY - 1) / TY;
    const long long G = (long long)tx_n * ty_n * Nz;
    const long long g0 = G * blockIdx.x / gridDim.x, g1 = G * (blockIdx.x + 1) / gridDim.x;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const C wdiv = from_f64<C>(1.0 / (4.0 * h)), wl = C(1.0 / 8.0);
    double acc[3] = {0.0, 0.0, 0.0};

    for (long long g = g0; g < g1;) {
        const int tile = (int)(g / Nz);
        const int z0 = (int)(g - (long long)tile * Nz);
        const int z1 = (int)min((long long)Nz, (long long)z0 + (g1 - g));
        g += z1 - z0;
        const int x0 = (tile % tx_n) * TX, y0 = (tile / tx_n) * TY;

        // cell plane c: each thread loads the FP64 fields of the (up to two)
        // staged cells it owns into registers -- a plane ahead of their use, so
        // the loads are in flight during the previous plane's barriers and
        // arithmetic -- then stage() forms W in shared memory and the shared
        // pair sums.  Absent cells (outside a non-periodic boundary) load 0.
        double rb[2], ru0[2], ru1[2], ru2[2], rs[2];
        auto load = [&](int c) {
            int gz = c;
            bool zok = true;
            if (gz < 0 || gz >= nz) { if (pz) gz = gz < 0 ? gz + nz : gz - nz; else zok = false; }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int q = tid + e * NT;
                rb[e] = ru0[e] = ru1[e] = ru2[e] = rs[e] = 0.0;
                if (q >= QN) continue;
                const int qy = q / (TX + 1), qx = q - qy * (TX + 1);
                int gx = x0 - 1 + qx, gy = y0 - 1 + qy;
                bool ok = zok;
                if (gx < 0 || gx >= nx) { if (px) gx = gx < 0 ? gx + nx : gx - nx; else ok = false; }
                if (gy < 0 || gy >= ny) { if (py) gy = gy < 0 ? gy + ny : gy - ny; else ok = false; }
                if (gx >= nx || gy >= ny) ok = false;
                if (ok) {
                    const size_t id = ((size_t)gz * ny + gy) * nx + gx;
                    rb[e] = b0[id];
                    ru0[e] = U.p[0][id];
                    ru1[e] = U.p[1][id];
                    ru2[e] = U.p[2][id];
                    rs[e] = S[id];
                }
            }
        };
        auto stage = [&]() {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int q = tid + e * NT;
                if (q >= QN) continue;
                const int qy = q / (TX + 1), qx = q - qy * (TX + 1);
                const C bb = from_f64<C>(rb[e]);
                sh.w[0][qy][qx] = bb * from_f64<C>(ru0[e]);
                sh.w[1][qy][qx] = bb * from_f64<C>(ru1[e]);
                sh.w[2][qy][qx] = bb * from_f64<C>(ru2[e]);
                sh.w[3][qy][qx] = bb * from_f64<C>(rs[e]);
            }
            __syncthreads();
            for (int q = tid; q < TY * (TX + 1); q += NT) {
                const int r = q / (TX + 1), cx = q - r * (TX + 1);
                sh.ya[r][cx] = sh.w[0][r][cx] + sh.w[0][r + 1][cx];
            }
            for (int q = tid; q < 3 * (TY + 1) * TX; q += NT) {
                const int e = q / ((TY + 1) * TX), rem = q - e * ((TY + 1) * TX);
                const int r = rem / TX, cx = rem - r * TX;
                sh.xa[e][r][cx] = sh.w[e + 1][r][cx] + sh.w[e + 1][r][cx + 1];
            }
            __syncthreads();
        };
        // the per-plane node terms: dx, dy (differences of pair sums), z and source pair sums
        C pdx, pdy, pz2, ps;
        auto terms = [&](C& dx, C& dy, C& bz, C& bs) {
            dx = sh.ya[ly][lx + 1] - sh.ya[ly][lx];
            dy = sh.xa[0][ly + 1][lx] - sh.xa[0][ly][lx];
            bz = sh.xa[1][ly][lx] + sh.xa[1][ly + 1][lx];
            bs = sh.xa[2][ly][lx] + sh.xa[2][ly + 1][lx];
        };
        load(z0 - 1);
        stage();
        terms(pdx, pdy, pz2, ps);
        load(z0);
        const int i = x0 + lx, j = y0 + ly;
        const bool own = i < Nx && j < Ny;
        for (int k = z0; k < z1; ++k) {
            stage();   // plane k (its first barrier follows every read of the previous plane's W)
            if (k + 1 < z1) load(k + 1);
            C dx, dy, bz, bs;
            terms(dx, dy, bz, bs);
            if (own) {
                const size_t id = ((size_t)k * Ny + j) * Nx + i;
                C v = C(0), lump = C(0);
                if (!node_dirichlet(L, i, j, k, 3)) {
                    lump = (bs + ps) * wl;
                    v = fmadd(((dx + pdx) + (dy + pdy)) + (bz - pz2), wdiv, -lump);
                }
                const double vd = to_f64(v), ld = to_f64(lump);
                if (f) f[id] = vd;
                acc[0] += vd;
                acc[1] = fmadd(ld, ld, acc[1]);
                acc[2] = fmadd(vd, vd, acc[2]);
            }
            pdx = dx;
            pdy = dy;
            pz2 = bz;
            ps = bs;
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

// Tiled 3-D k_node_project.  A CTA owns a 32 x 8 column of cells and marches
// up its cell planes; per node plane it forms once the x-differences and
// x-pair sums of phi at every cell column and node row, from which each cell
// takes its gradient components with one y-pair operation per plane (the
// lower node plane's values are carried in registers).  About 9 FP64
// operations per cell for G_N instead of 21.
struct NodeProjShared {
    double xs[kNTY + 1][kNTX + 1];  // phi, nodes x0 .. x0+32, y0 .. y0+8 of one node plane
    double dx[kNTY + 1][kNTX];      // phi(x+1) - phi(x)
    double ax[kNTY + 1][kNTX];      // phi(x) + phi(x+1)
};

__global__ void __launch_bounds__(kNTX * kNTY, 4)
k_node_project_tiled(NodeLevel<double> L, double h, const double* __restrict__ phi, const double* __restrict__ b0,
                     MPtr3n U, int kz)
{
    constexpr int TX = kNTX, TY = kNTY, NT = TX * TY, QN = (TX + 1) * (TY + 1);
    static_assert(QN <= 2 * NT, "each thread stages at most two nodes of a plane");
    __shared__ NodeProjShared sh;
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * kz, z1 = min(z0 + kz, nz);
    const int tid = threadIdx.y * TX + threadIdx.x, lx = threadIdx.x, ly = threadIdx.y;
    const double w4 = 1.0 / (4.0 * h);
    // node plane p: phi of the (up to two) staged nodes a thread owns, loaded
    // into registers a plane ahead of use (nodes past the grid edge of a
    // partial tile read as 0); stage() forms the shared partial sums
    double rx[2];
    auto load = [&](int p) {
        const int pn = p >= Nz ? p - Nz : p;  // p == Nz only when z is periodic (node nz is node 0)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = tid + e * NT;
            rx[e] = 0.0;
            if (q >= QN) continue;
            const int r = q / (TX + 1), c = q - r * (TX + 1);
            int gx = x0 + c, gy = y0 + r;
            if (gx >= Nx) gx = L.bc.lo[0] == BCP ? gx - Nx : -1;
            if (gy >= Ny) gy = L.bc.lo[1] == BCP ? gy - Ny : -1;
            if (gx >= 0 && gy >= 0) rx[e] = phi[((size_t)pn * Ny + gy) * Nx + gx];
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = tid + e * NT;
            if (q >= QN) continue;
            const int r = q / (TX + 1), c = q - r * (TX + 1);
            sh.xs[r][c] = rx[e];
        }
        __syncthreads();
        for (int q = tid; q < (TY + 1) * TX; q += NT) {
            const int r = q / TX, c = q - r * TX;
            sh.dx[r][c] = sh.xs[r][c + 1] - sh.xs[r][c];
            sh.ax[r][c] = sh.xs[r][c] + sh.xs[r][c + 1];
        }
        __syncthreads();
    };
    double gxl, gyl, bl;
    auto terms = [&](double& gxp, double& gyp, double& bp) {
        gxp = sh.dx[ly][lx] + sh.dx[ly + 1][lx];
        gyp = sh.ax[ly + 1][lx] - sh.ax[ly][lx];
        bp = sh.ax[ly][lx] + sh.ax[ly + 1][lx];
    };
    const int i = x0 + lx, j = y0 + ly;
    const bool own = i < nx && j < ny;
    // the owned cell's sigma, beta0 and U, also loaded a plane ahead
    double cs = 0.0, cb = 1.0, cu[3] = {0.0, 0.0, 0.0};
    auto load_cell = [&](int k) {
        if (!own) return;
        const size_t t = ((size_t)k * ny + j) * nx + i;
        cs = L.sigma[t];
        cb = b0[t];
        cu[0] = U.p[0][t];
        cu[1] = U.p[1][t];
        cu[2] = U.p[2][t];
    };
    load(z0);
    stage();
    terms(gxl, gyl, bl);
    load(z0 + 1);
    load_cell(z0);
    for (int k = z0; k < z1; ++k) {
        stage();  // node plane k + 1 (its first barrier follows every read of the previous plane's sums)
        if (k + 2 <= z1) load(k + 2);
        const double s0 = cs, b0k = cb, u0 = cu[0], u1 = cu[1], u2 = cu[2];
        if (k + 1 < z1) load_cell(k + 1);
        double gxu, gyu, bu;
        terms(gxu, gyu, bu);
        if (own) {
            const size_t t = ((size_t)k * ny + j) * nx + i;
            const double w = s0 * recip_nr(b0k) * w4;
            U.p[0][t] = fmadd(-w, gxl + gxu, u0);
            U.p[1][t] = fmadd(-w, gyl + gyu, u1);
            U.p[2][t] = fmadd(-w, bu - bl, u2);
        }
        gxl = gxu;
        gyl = gyu;
        bl = bu;
    }
}

// ================================================================ launchers

void node_rhs(int dim, const NodeLevel<double>& L, double h, const double* const U[3], const double* b0,
              const double* S, double* f, double* partials, cudaStream_t s)
{
    CPtr3 u{{U[0], U[1], dim == 3 ? U[2] : nullptr}};
    if (dim == 3 && L.Nx >= kNTX && L.Ny >= kNTY) {
        MGP_LAUNCH(k_node_rhs_tiled<double><<<kRedBlocks, dim3(kNTX, kNTY), 0, s>>>(L, h, u, b0, S, f, partials));
        return;
    }
    if (dim == 2) MGP_LAUNCH(k_node_rhs<2><<<kRedBlocks, kThreads, 0, s>>>(L, h, u, b0, S, f, partials));
    else MGP_LAUNCH(k_node_rhs<3><<<kRedBlocks, kThreads, 0, s>>>(L, h, u, b0, S, f, partials));
}

bool node_constraint32(int dim, const NodeLevel<double>& L, double h, const double* const U[3], const double* b0,
                       const double* S, double* partials, cudaStream_t s)
{
    if (!(dim == 3 && L.Nx >= kNTX && L.Ny >= kNTY)) return false;
    CPtr3 u{{U[0], U[1], U[2]}};
    MGP_LAUNCH(k_node_rhs_tiled<float><<<kRedBlocks, dim3(kNTX, kNTY), 0, s>>>(L, h, u, b0, S, nullptr, partials));
    return true;
}

void node_project(int dim, const NodeLevel<double>& L, double h, const double* phi, const double* b0,
                  double* const U[3], cudaStream_t s)
{
    MPtr3n u{{U[0], U[1], dim == 3 ? U[2] : nullptr}};
    long long n = (long long)L.nx * L.ny * L.nz;
    if (dim == 3 && L.nx >= kNTX && L.ny >= kNTY) {
        // z-chunks sized for about 4 CTAs per SM
        const long long cols = (long long)((L.nx + kNTX - 1) / kNTX) * ((L.ny + kNTY - 1) / kNTY);
        int kz = (int)((cols * L.nz + 608 * 2 - 1) / (608 * 2));
        kz = kz < 4 ? 4 : kz;
        const dim3 grid((L.nx + kNTX - 1) / kNTX, (L.ny + kNTY - 1) / kNTY, (L.nz + kz - 1) / kz);
        MGP_LAUNCH(k_node_project_tiled<<<grid, dim3(kNTX, kNTY), 0, s>>>(L, h, phi, b0, u, kz));
        return;
    }
    if (dim == 2) MGP_LAUNCH(k_node_project<2><<<nb(n), kThreads, 0, s>>>(L, h, phi, b0, u));
    else MGP_LAUNCH(k_node_project<3><<<nb(n), kThreads, 0, s>>>(L, h, phi, b0, u));
}

}  // namespace mgp
