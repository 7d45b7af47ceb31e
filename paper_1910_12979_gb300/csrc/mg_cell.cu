// mg_cell.cu -- cell-centred (MAC projection) kernels.
//
// Discrete system (the reading of Eq. 6 used throughout the library):
//   (L phi)_c = sum_d [ Bt_{c+1/2}(phi_{c+e_d} - phi_c) - Bt_{c-1/2}(phi_c - phi_{c-e_d}) ]
// with Bt = B / h_d^2 the face coefficient pre-scaled at setup and B the
// harmonic mean of sigma = beta0/rho on the face.  Written row-wise as
//   (L phi)_c = off_c - diag_c phi_c,
//   off  = sum over interior/periodic faces of Bt phi_neighbour,
//   diag = sum over interior/periodic faces of Bt + 2 Bt on Dirichlet faces,
// Neumann faces contributing nothing and a Dirichlet face (phi = 0 on the
// face) acting through the ghost value -phi_c.
#include "mg_cellops.cuh"

#include <type_traits>

namespace mgp {

// ------------------------------------------------------------------ setup

__device__ __forceinline__ double harmonic(double a, double b) { return (2.0 * a * b) * recip_nr(a + b); }

// face coefficient along axis d from cell sigma, scaled by 1/h_d^2
template <int D>
__global__ void k_faces_from_sigma(CellLevel<double> L, const double* __restrict__ sigma, double ih2,
                                   double* __restrict__ out)
{
    const int mx = L.nx + (D == 0), my = L.ny + (D == 1), mz = L.nz + (D == 2);
    const int total = mx * my * mz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int f[3];
    unflat(t, mx, my, f[0], f[1], f[2]);
    const int n = (D == 0) ? L.nx : (D == 1) ? L.ny : L.nz;
    int lo[3] = {f[0], f[1], f[2]}, hi[3] = {f[0], f[1], f[2]};
    lo[D] -= 1;
    auto S = [&](const int* c) { return sigma[((size_t)c[2] * L.ny + c[1]) * L.nx + c[0]]; };
    double v;
    if (f[D] == 0 || f[D] == n) {
        if (L.bc.lo[D] == BCP) {
            lo[D] = n - 1;
            hi[D] = 0;
            v = harmonic(S(lo), S(hi));
        } else if (f[D] == 0) {
            v = S(hi);
        } else {
            v = S(lo);
        }
    } else {
        v = harmonic(S(lo), S(hi));
    }
    out[t] = v * ih2;
}

__global__ void k_scale(const double* __restrict__ in, double s, double* __restrict__ out, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = in[t] * s;
}

// coarse face = mean of the 2^(dim-1) fine faces it covers, times h_f^2/h_c^2 = 1/4
template <int DIM, int D>
__global__ void k_coarsen_faces(CellLevel<double> F, CellLevel<double> C, const double* __restrict__ fine,
                                double* __restrict__ coarse)
{
    const int mx = C.nx + (D == 0), my = C.ny + (D == 1), mz = C.nz + (D == 2);
    const int total = mx * my * mz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int f[3];
    unflat(t, mx, my, f[0], f[1], f[2]);
    const int fx = F.nx + (D == 0), fy = F.ny + (D == 1);
    double s = 0.0;
    constexpr int nsub = 1 << (DIM - 1);
#pragma unroll
    for (int q = 0; q < nsub; ++q) {
        int g[3] = {2 * f[0], 2 * f[1], DIM == 3 ? 2 * f[2] : 0};
        int bit = 0;
#pragma unroll
        for (int e = 0; e < DIM; ++e) {
            if (e == D) continue;
            g[e] += (q >> bit) & 1;
            ++bit;
        }
        s += fine[((size_t)g[2] * fy + g[1]) * fx + g[0]];
    }
    coarse[t] = s * (0.25 / nsub);
}

// The diagonal of row (i,j,k) alone: the dg sum of cell_row, in the same order.
template <int DIM>
__device__ __forceinline__ double cell_dg(const CellLevel<double>& L, int i, int j, int k)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    double dg = 0.0;
    auto term = [&](double b, bool inside, int bc) {
        if (inside || bc == BCP) dg += b;
        else if (bc == BCD) dg += 2.0 * b;
    };
    const size_t rx = ((size_t)k * ny + j) * (nx + 1) + i;
    term(L.bx[rx], i > 0, L.bc.lo[0]);
    term(L.bx[rx + 1], i < nx - 1, L.bc.hi[0]);
    const size_t ry = ((size_t)k * (ny + 1) + j) * nx + i;
    term(L.by[ry], j > 0, L.bc.lo[1]);
    term(L.by[ry + nx], j < ny - 1, L.bc.hi[1]);
    if (DIM == 3) {
        const size_t rz = ((size_t)k * ny + j) * nx + i, pl = (size_t)nx * ny;
        term(L.bz[rz], k > 0, L.bc.lo[2]);
        term(L.bz[rz + pl], k < nz - 1, L.bc.hi[2]);
    }
    return dg;
}

template <int DIM>
__global__ void k_invdiag(CellLevel<double> L, double* __restrict__ invd)
{
    const int total = L.nx * L.ny * L.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.nx, L.ny, i, j, k);
    invd[t] = recip(cell_dg<DIM>(L, i, j, k));
}

// ------------------------------------------------------------- smoothing

// One colour of red-black Gauss-Seidel: phi_c <- (off_c - b_c) / diag_c on
// cells with (i + j + k) % 2 == color.
template <int DIM, typename T>
__global__ void k_gsrb(CellLevel<T> L, T* __restrict__ x, const T* __restrict__ b, int color)
{
    const int total = L.nx * L.ny * L.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.nx, L.ny, i, j, k);
    if (((i + j + k) & 1) != color) return;
    x[t] = gs_value<DIM>(L, x, b, i, j, k);
}

// r = b - L x on the fine level, averaged over the 2^dim children of each coarse cell.
template <int DIM, typename T>
__global__ void k_resid_restrict(CellLevel<T> F, const T* __restrict__ x, const T* __restrict__ b,
                                 T* __restrict__ bc, int cnx, int cny, int cnz)
{
    const int total = cnx * cny * cnz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int ci, cj, ck;
    unflat(t, cnx, cny, ci, cj, ck);
    bc[t] = restrict_value<DIM>(F, x, b, ci, cj, ck);
}

// 3-D residual + restriction with one thread per fine cell: a (32, 2, 2) block
// covers the 2 x 2 x 2 children of 16 coarse cells; the residuals are summed
// over x by a shuffle and over y and z through shared memory, in the fixed order
// (x pair, then y, then z).  Used when nx % 32 == 0 and ny, nz are even.
template <typename T>
__global__ void __launch_bounds__(128) k_resid_restrict_t(CellLevel<T> F, const T* __restrict__ x,
                                                          const T* __restrict__ b, T* __restrict__ bc)
{
    __shared__ T sh[2][2][16];
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 2 + threadIdx.y, k = blockIdx.z * 2 + threadIdx.z;
    const size_t id = ((size_t)k * F.ny + j) * F.nx + i;
    T off, dg;
    cell_row<3>(F, i, j, k, GlobalPhi<T>{x, F.nx, F.ny}, off, dg);
    T r = b[id] - fmadd(-dg, x[id], off);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    if ((threadIdx.x & 1) == 0) sh[threadIdx.z][threadIdx.y][threadIdx.x >> 1] = r;
    __syncthreads();
    if (threadIdx.y == 0 && threadIdx.z == 0 && (threadIdx.x & 1) == 0) {
        const int q = threadIdx.x >> 1;
        const T s2 = (sh[0][0][q] + sh[0][1][q]) + (sh[1][0][q] + sh[1][1][q]);
        const int cnx = F.nx / 2, cny = F.ny / 2;
        bc[((size_t)blockIdx.z * cny + blockIdx.y) * cnx + (i >> 1)] = s2 * T(0.125);
    }
}

template <int DIM, typename T, int ORDER>
__global__ void k_prolong_add(CellLevel<T> F, CellLevel<T> C, T* __restrict__ xf, const T* __restrict__ xc)
{
    const int total = F.nx * F.ny * F.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, F.nx, F.ny, i, j, k);
    xf[t] += prolong_value<DIM>(F, C, xc, i, j, k, ORDER);
}

// -------------------------------------------------------- FP64 residuals

// r = f - L x in FP64, its FP32 copy r / fscale (fscale a power of two, folded
// into the conversion) and the partial sums of the copy's squares.  A thread
// takes quads of four consecutive cells (flat index), grid-stride; the sums
// follow that order, which the vectorised kernel below and the zero-guess
// initialisation share, so all three give the same norm.
template <int DIM, bool HAS_DIAG>
__global__ void k_resid64(CellLevel<double> L, const double* __restrict__ x, const double* __restrict__ b,
                          float* __restrict__ r32, const double* __restrict__ scale, double* __restrict__ partials)
{
    const int total = L.nx * L.ny * L.nz, nquad = (total + 3) / 4;
    const int sh = pow2_shift(*scale);
    float acc = 0.f;
    const GlobalPhi<double> ph{x, L.nx, L.ny};
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nquad; u += gridDim.x * blockDim.x)
        for (int t = 4 * u; t < 4 * u + 4 && t < total; ++t) {
            int i, j, k;
            unflat(t, L.nx, L.ny, i, j, k);
            double off, dg;
            cell_row<DIM>(L, i, j, k, ph, off, dg);
            const double d = HAS_DIAG ? L.diag[t] : dg;
            const float rs = f64_to_f32_pow2(b[t] - fmadd(-d, x[t], off), sh);
            acc = fmaf(rs, rs, acc);
            if (r32) r32[t] = rs;
        }
    double a[1] = {(double)acc};
    block_reduce_store<1>(a, partials);
}

// The same residual, four consecutive cells of an x-row per thread (3-D,
// nx % 4 == 0, stored diagonal): the row, its y- and z-neighbour rows, b, the
// diagonal and the y-/z-faces as 16-byte loads, the quad's x-neighbours from
// the neighbouring lanes, the integer index work once per quad.  Every cell's
// FP64 arithmetic is cell_row's (face terms x-lo, x-hi, y-lo, y-hi, z-lo, z-hi,
// fused multiply-adds from 0) followed by b - fma(-d, x, off): identical values.
// The body is shared with the batched residual (one block's share of one solve).
// vb, vgrid: the block's index and the grid size of that partition.
__device__ __forceinline__ void resid64_v4_block(const CellLevel<double>& L, const double* __restrict__ x,
                                                 const double* __restrict__ b, float* __restrict__ r32,
                                                 const double* __restrict__ scale, double* __restrict__ partials,
                                                 int vb, int vgrid)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz, nq = nx / 4;
    const int nquad = nq * ny * nz;
    const int sh = pow2_shift(*scale);
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const size_t plane = (size_t)nx * ny;
    float acc = 0.f;
    auto ld2 = [](const double* p) { return *reinterpret_cast<const double2*>(p); };
    const double2 z2 = make_double2(0.0, 0.0);
    const int stride = vgrid * blockDim.x;
    for (int u0 = vb * blockDim.x; u0 < nquad; u0 += stride) {
        // every lane of the warp runs the iteration (shuffles); lanes past the end compute the last quad
        const int ug = u0 + threadIdx.x;
        const bool live = ug < nquad;
        const int u = live ? ug : nquad - 1;
        const int q = u % nq, rowi = u / nq, j = rowi % ny, k = rowi / ny;
        const int i0 = 4 * q;
        const size_t row = (size_t)k * plane + (size_t)j * nx, c = row + i0;
        const double2 xa = ld2(x + c), xb = ld2(x + c + 2);
        const bool hym = j > 0 || py, hyp = j < ny - 1 || py, hzm = k > 0 || pz, hzp = k < nz - 1 || pz;
        const size_t rym = j > 0 ? row - nx : row + (size_t)(ny - 1) * nx;
        const size_t ryp = j < ny - 1 ? row + nx : row - (size_t)(ny - 1) * nx;
        const size_t rzm = k > 0 ? row - plane : row + (size_t)(nz - 1) * plane;
        const size_t rzp = k < nz - 1 ? row + plane : row - (size_t)(nz - 1) * plane;
        const double2 ym0 = hym ? ld2(x + rym + i0) : z2, ym1 = hym ? ld2(x + rym + i0 + 2) : z2;
        const double2 yp0 = hyp ? ld2(x + ryp + i0) : z2, yp1 = hyp ? ld2(x + ryp + i0 + 2) : z2;
        const double2 zm0 = hzm ? ld2(x + rzm + i0) : z2, zm1 = hzm ? ld2(x + rzm + i0 + 2) : z2;
        const double2 zp0 = hzp ? ld2(x + rzp + i0) : z2, zp1 = hzp ? ld2(x + rzp + i0 + 2) : z2;
        const double2 ba = ld2(b + c), bb = ld2(b + c + 2), da = ld2(L.diag + c), db = ld2(L.diag + c + 2);
        // x-neighbours: the previous / next quad's edge cells when that quad is in the same row and warp
        const int lane = threadIdx.x & 31;
        double xl = __shfl_up_sync(0xffffffffu, xb.y, 1), xr = __shfl_down_sync(0xffffffffu, xa.x, 1);
        if (lane == 0 || q == 0) xl = i0 > 0 ? x[c - 1] : (px ? x[row + nx - 1] : 0.0);
        if (lane == 31 || q == nq - 1) xr = i0 + 4 < nx ? x[c + 4] : (px ? x[row] : 0.0);
        const size_t fxb = ((size_t)k * ny + j) * (nx + 1) + i0;
        const double fx[5] = {L.bx[fxb], L.bx[fxb + 1], L.bx[fxb + 2], L.bx[fxb + 3], L.bx[fxb + 4]};
        const size_t fyb = ((size_t)k * (ny + 1) + j) * nx + i0;
        const double2 fyl0 = ld2(L.by + fyb), fyl1 = ld2(L.by + fyb + 2);
        const double2 fyh0 = ld2(L.by + fyb + nx), fyh1 = ld2(L.by + fyb + nx + 2);
        const double2 fzl0 = ld2(L.bz + c), fzl1 = ld2(L.bz + c + 2);
        const double2 fzh0 = ld2(L.bz + c + plane), fzh1 = ld2(L.bz + c + plane + 2);
        auto e2 = [](const double2& lo, const double2& hi, int p) { return p == 0 ? lo.x : p == 1 ? lo.y : p == 2 ? hi.x : hi.y; };
        const double xs[6] = {xl, xa.x, xa.y, xb.x, xb.y, xr};
        float rsv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = i0 + p;
            double off = 0.0;
            if (i > 0 || px) off = fmadd(fx[p], xs[p], off);
            if (i < nx - 1 || px) off = fmadd(fx[p + 1], xs[p + 2], off);
            if (hym) off = fmadd(e2(fyl0, fyl1, p), e2(ym0, ym1, p), off);
            if (hyp) off = fmadd(e2(fyh0, fyh1, p), e2(yp0, yp1, p), off);
            if (hzm) off = fmadd(e2(fzl0, fzl1, p), e2(zm0, zm1, p), off);
            if (hzp) off = fmadd(e2(fzh0, fzh1, p), e2(zp0, zp1, p), off);
            rsv[p] = f64_to_f32_pow2(e2(ba, bb, p) - fmadd(-e2(da, db, p), xs[p + 1], off), sh);
        }
        if (live) {
#pragma unroll
            for (int p = 0; p < 4; ++p) acc = fmaf(rsv[p], rsv[p], acc);
            if (r32) *reinterpret_cast<float4*>(r32 + c) = make_float4(rsv[0], rsv[1], rsv[2], rsv[3]);
        }
    }
    double a[1] = {(double)acc};
    block_reduce_store<1>(a, partials, vb);
}

__global__ void __launch_bounds__(256)
k_resid64_v4(CellLevel<double> L, const double* __restrict__ x, const double* __restrict__ b,
             float* __restrict__ r32, const double* __restrict__ scale, double* __restrict__ partials)
{
    resid64_v4_block(L, x, b, r32, scale, partials, blockIdx.x, gridDim.x);
}

// Batched FP64 residuals: one block per (solve, block of k_resid64_v4's
// kRedBlocks-block partition that has quads); each takes that block's quads
// and partial slot, so every solve's residual and norm partials are those of
// its solve alone.  The first block of a solve zeroes the slots of the
// partition's blocks without quads (their partials alone are 0).
__global__ void __launch_bounds__(256)
k_resid64_batch(const Resid64Item* __restrict__ items, const int* __restrict__ bmap, const int* __restrict__ run)
{
    const Resid64Item& it = items[__ldg(bmap + blockIdx.x)];
    if (!__ldg(run + it.solve)) return;
    const int vb = blockIdx.x - it.vb0;
    if (vb == 0)
        for (int t = it.nvb + threadIdx.x; t < kRedBlocks; t += blockDim.x) it.partials[t] = 0.0;
    resid64_v4_block(it.L, it.x, it.b, it.r32, it.scale, it.partials, vb, kRedBlocks);
}

bool cell_resid64_batch_ok(const CellLevel<double>& L, const double* x, const double* b, const float* r32)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return L.diag && L.nx % 4 == 0 && a16(x) && a16(b) && a16(L.diag) && a16(L.by) && a16(L.bz) &&
           (!r32 || a16(r32)) && (size_t)L.nx * L.ny * L.nz / 4 < (size_t)1 << 30;
}

void cell_resid64_batch(const Resid64Item* items, const int* bmap, int blocks, const int* run, cudaStream_t s)
{
    MGP_LAUNCH(k_resid64_batch<<<blocks, kThreads, 0, s>>>(items, bmap, run));
}

template <int DIM>
__global__ void k_diag(CellLevel<double> L, double* __restrict__ diag)
{
    const int total = L.nx * L.ny * L.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.nx, L.ny, i, j, k);
    diag[t] = cell_dg<DIM>(L, i, j, k);
}

template <int DIM>
__global__ void k_apply64(CellLevel<double> L, const double* __restrict__ x, double* __restrict__ out)
{
    const int total = L.nx * L.ny * L.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int i, j, k;
    unflat(t, L.nx, L.ny, i, j, k);
    double off, dg;
    cell_row<DIM>(L, i, j, k, GlobalPhi<double>{x, L.nx, L.ny}, off, dg);
    out[t] = off - dg * x[t];
}

// ------------------------------------------------------ RHS / projection

struct Ptr3 {
    const double* p[3];
};
struct MPtr3 {
    double* p[3];
};

// f = D(beta0 U) - beta0 S  (Eq. 6), partial sums {sum f, sum (beta0 S)^2, sum f^2}
template <int DIM>
__global__ void k_rhs(CellLevel<double> L, double ihx, double ihy, double ihz, Ptr3 U, Ptr3 B0, const double* b0c,
                      const double* S, double* __restrict__ f, double* __restrict__ partials)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int total = nx * ny * nz;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int i, j, k;
        unflat(t, nx, ny, i, j, k);
        const size_t rx = ((size_t)k * ny + j) * (nx + 1) + i;
        double v = (B0.p[0][rx + 1] * U.p[0][rx + 1] - B0.p[0][rx] * U.p[0][rx]) * ihx;
        const size_t ry = ((size_t)k * (ny + 1) + j) * nx + i;
        v += (B0.p[1][ry + nx] * U.p[1][ry + nx] - B0.p[1][ry] * U.p[1][ry]) * ihy;
        if (DIM == 3) {
            const size_t rz = (size_t)t, pl = (size_t)nx * ny;
            v += (B0.p[2][rz + pl] * U.p[2][rz + pl] - B0.p[2][rz] * U.p[2][rz]) * ihz;
        }
        const double src = b0c[t] * S[t];
        v -= src;
        if (f) f[t] = v;
        acc[0] += v;
        acc[1] += src * src;
        acc[2] += v * v;
    }
    block_reduce_store<3>(acc, partials);
}

// U_f -= (B_f / beta0_f) (G phi)_f along axis D; Bt h = B/h, Dirichlet faces
// use phi = 0 on the face at distance h/2, Neumann faces are left unchanged.
template <int D>
__global__ void k_project(CellLevel<double> L, double h, const double* __restrict__ phi, const double* __restrict__ b0f,
                          double* __restrict__ U, const double* __restrict__ Bt)
{
    const int mx = L.nx + (D == 0), my = L.ny + (D == 1), mz = L.nz + (D == 2);
    const int total = mx * my * mz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int f[3];
    unflat(t, mx, my, f[0], f[1], f[2]);
    const int n = (D == 0) ? L.nx : (D == 1) ? L.ny : L.nz;
    int lo[3] = {f[0], f[1], f[2]}, hi[3] = {f[0], f[1], f[2]};
    lo[D] -= 1;
    auto P = [&](const int* c) { return phi[((size_t)c[2] * L.ny + c[1]) * L.nx + c[0]]; };
    double flux;  // B (G phi) = Bt h^2 (G phi)
    if (f[D] == 0 || f[D] == n) {
        if (L.bc.lo[D] == BCP) {
            lo[D] = n - 1;
            hi[D] = 0;
            flux = Bt[t] * h * (P(hi) - P(lo));
        } else {
            const int bc = (f[D] == 0) ? L.bc.lo[D] : L.bc.hi[D];
            if (bc != BCD) return;
            flux = (f[D] == 0) ? 2.0 * Bt[t] * h * P(hi) : -2.0 * Bt[t] * h * P(lo);
        }
    } else {
        flux = Bt[t] * h * (P(hi) - P(lo));
    }
    U[t] -= flux * recip_nr(b0f[t]);
}

// ---------------------------------------------------------- dense coarsest

template <int DIM, typename T>
__global__ void k_dense_assemble(CellLevel<T> L, double* __restrict__ A, int lda)
{
    const int N = L.nx * L.ny * L.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * N) return;
    const int row = t / N, col = t % N;
    int i, j, k;
    unflat(row, L.nx, L.ny, i, j, k);
    T off, dg;
    const UnitPhi e{col, L.nx, L.ny};
    cell_row<DIM>(L, i, j, k, [&](int a, int b, int c) { return (T)e(a, b, c); }, off, dg);
    A[(size_t)row * lda + col] = (double)off - (row == col ? (double)dg : 0.0);
}

// ================================================================ launchers

static inline int nb(long long n) { return ceil_div(n, kThreads); }

void cell_faces_from_sigma(int dim, const CellLevel<double>& L, const double* sigma, const double* h, double* bx,
                           double* by, double* bz, cudaStream_t s)
{
    long long mx = (long long)(L.nx + 1) * L.ny * L.nz;
    MGP_LAUNCH(k_faces_from_sigma<0><<<nb(mx), kThreads, 0, s>>>(L, sigma, 1.0 / (h[0] * h[0]), bx));
    long long my = (long long)L.nx * (L.ny + 1) * L.nz;
    MGP_LAUNCH(k_faces_from_sigma<1><<<nb(my), kThreads, 0, s>>>(L, sigma, 1.0 / (h[1] * h[1]), by));
    if (dim == 3) {
        long long mz = (long long)L.nx * L.ny * (L.nz + 1);
        MGP_LAUNCH(k_faces_from_sigma<2><<<nb(mz), kThreads, 0, s>>>(L, sigma, 1.0 / (h[2] * h[2]), bz));
    }
}

void cell_scale_faces(int dim, const CellLevel<double>& L, const double* const face[3], const double* h, double* bx,
                      double* by, double* bz, cudaStream_t s)
{
    double* out[3] = {bx, by, bz};
    for (int d = 0; d < dim; ++d) {
        long long m = (long long)(L.nx + (d == 0)) * (L.ny + (d == 1)) * (L.nz + (d == 2));
        MGP_LAUNCH(k_scale<<<nb(m), kThreads, 0, s>>>(face[d], 1.0 / (h[d] * h[d]), out[d], (int)m));
    }
}

void cell_coarsen_faces(int dim, const CellLevel<double>& F, const CellLevel<double>& C, double* bx, double* by,
                        double* bz, cudaStream_t s)
{
    long long mx = (long long)(C.nx + 1) * C.ny * C.nz, my = (long long)C.nx * (C.ny + 1) * C.nz;
    if (dim == 2) {
        MGP_LAUNCH(k_coarsen_faces<2, 0><<<nb(mx), kThreads, 0, s>>>(F, C, F.bx, bx));
        MGP_LAUNCH(k_coarsen_faces<2, 1><<<nb(my), kThreads, 0, s>>>(F, C, F.by, by));
    } else {
        long long mz = (long long)C.nx * C.ny * (C.nz + 1);
        MGP_LAUNCH(k_coarsen_faces<3, 0><<<nb(mx), kThreads, 0, s>>>(F, C, F.bx, bx));
        MGP_LAUNCH(k_coarsen_faces<3, 1><<<nb(my), kThreads, 0, s>>>(F, C, F.by, by));
        MGP_LAUNCH(k_coarsen_faces<3, 2><<<nb(mz), kThreads, 0, s>>>(F, C, F.bz, bz));
    }
}

void cell_invdiag(int dim, const CellLevel<double>& L, double* invd, cudaStream_t s)
{
    long long n = (long long)L.nx * L.ny * L.nz;
    if (dim == 2) MGP_LAUNCH(k_invdiag<2><<<nb(n), kThreads, 0, s>>>(L, invd));
    else MGP_LAUNCH(k_invdiag<3><<<nb(n), kThreads, 0, s>>>(L, invd));
}

template <typename T>
void cell_gsrb(int dim, const CellLevel<T>& L, T* x, const T* b, int color, cudaStream_t s)
{
    long long n = (long long)L.nx * L.ny * L.nz;
    if (dim == 2) MGP_LAUNCH(k_gsrb<2, T><<<nb(n), kThreads, 0, s>>>(L, x, b, color));
    else MGP_LAUNCH(k_gsrb<3, T><<<nb(n), kThreads, 0, s>>>(L, x, b, color));
}

template <typename T>
void cell_resid_restrict(int dim, const CellLevel<T>& F, const T* x, const T* b, T* bc, cudaStream_t s)
{
    if (dim == 3 && F.nx % 32 == 0 && F.ny % 2 == 0 && F.nz % 2 == 0) {
        MGP_LAUNCH(k_resid_restrict_t<T><<<dim3(F.nx / 32, F.ny / 2, F.nz / 2), dim3(32, 2, 2), 0, s>>>(F, x, b, bc));
        return;
    }
    const int cnx = F.nx / 2, cny = F.ny / 2, cnz = dim == 3 ? F.nz / 2 : 1;
    long long n = (long long)cnx * cny * cnz;
    if (dim == 2) MGP_LAUNCH(k_resid_restrict<2, T><<<nb(n), kThreads, 0, s>>>(F, x, b, bc, cnx, cny, cnz));
    else MGP_LAUNCH(k_resid_restrict<3, T><<<nb(n), kThreads, 0, s>>>(F, x, b, bc, cnx, cny, cnz));
}

template <typename T>
void cell_prolong_add(int dim, const CellLevel<T>& F, const CellLevel<T>& C, T* xf, const T* xc, int order,
                      cudaStream_t s)
{
    long long n = (long long)F.nx * F.ny * F.nz;
    if constexpr (std::is_same<T, float>::value) {
        if (order == 1 && cell_prolong_v4_ok(dim, F, xf, xc)) {
            cell_prolong_v4(F, C, xf, xc, s);
            return;
        }
    }
    if (dim == 2) {
        if (order == 0) MGP_LAUNCH(k_prolong_add<2, T, 0><<<nb(n), kThreads, 0, s>>>(F, C, xf, xc));
        else MGP_LAUNCH(k_prolong_add<2, T, 1><<<nb(n), kThreads, 0, s>>>(F, C, xf, xc));
    } else {
        if (order == 0) MGP_LAUNCH(k_prolong_add<3, T, 0><<<nb(n), kThreads, 0, s>>>(F, C, xf, xc));
        else MGP_LAUNCH(k_prolong_add<3, T, 1><<<nb(n), kThreads, 0, s>>>(F, C, xf, xc));
    }
}

void cell_resid64(int dim, const CellLevel<double>& L, const double* x, const double* b, float* r32,
                  const double* scale, double* partials, cudaStream_t s, bool vec)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    if (vec && dim == 3 && L.diag && L.nx % 4 == 0 && a16(x) && a16(b) && a16(L.diag) && a16(L.by) && a16(L.bz) &&
        (!r32 || a16(r32)) && (size_t)L.nx * L.ny * L.nz / 4 < (size_t)1 << 30) {
        MGP_LAUNCH(k_resid64_v4<<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
        return;
    }
    if (dim == 2) {
        if (L.diag) MGP_LAUNCH(k_resid64<2, true><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
        else MGP_LAUNCH(k_resid64<2, false><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
    } else {
        if (L.diag) MGP_LAUNCH(k_resid64<3, true><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
        else MGP_LAUNCH(k_resid64<3, false><<<kRedBlocks, kThreads, 0, s>>>(L, x, b, r32, scale, partials));
    }
}

void cell_diag(int dim, const CellLevel<double>& L, double* diag, cudaStream_t s)
{
    long long n = (long long)L.nx * L.ny * L.nz;
    if (dim == 2) MGP_LAUNCH(k_diag<2><<<nb(n), kThreads, 0, s>>>(L, diag));
    else MGP_LAUNCH(k_diag<3><<<nb(n), kThreads, 0, s>>>(L, diag));
}

void cell_apply64(int dim, const CellLevel<double>& L, const double* x, double* out, cudaStream_t s)
{
    long long n = (long long)L.nx * L.ny * L.nz;
    if (dim == 2) MGP_LAUNCH(k_apply64<2><<<nb(n), kThreads, 0, s>>>(L, x, out));
    else MGP_LAUNCH(k_apply64<3><<<nb(n), kThreads, 0, s>>>(L, x, out));
}

void cell_rhs(int dim, const CellLevel<double>& L, const double* h, const double* const U[3],
              const double* const b0f[3], const double* b0c, const double* S, double* f, double* partials,
              cudaStream_t s)
{
    Ptr3 u{{U[0], U[1], dim == 3 ? U[2] : nullptr}}, b{{b0f[0], b0f[1], dim == 3 ? b0f[2] : nullptr}};
    const double ihz = dim == 3 ? 1.0 / h[2] : 0.0;
    if (dim == 2) MGP_LAUNCH(k_rhs<2><<<kRedBlocks, kThreads, 0, s>>>(L, 1.0 / h[0], 1.0 / h[1], ihz, u, b, b0c, S, f, partials));
    else MGP_LAUNCH(k_rhs<3><<<kRedBlocks, kThreads, 0, s>>>(L, 1.0 / h[0], 1.0 / h[1], ihz, u, b, b0c, S, f, partials));
}

void cell_project(int dim, const CellLevel<double>& L, const double* h, const double* phi, const double* const b0f[3],
                  double* const U[3], cudaStream_t s)
{
    long long mx = (long long)(L.nx + 1) * L.ny * L.nz, my = (long long)L.nx * (L.ny + 1) * L.nz;
    MGP_LAUNCH(k_project<0><<<nb(mx), kThreads, 0, s>>>(L, h[0], phi, b0f[0], U[0], L.bx));
    MGP_LAUNCH(k_project<1><<<nb(my), kThreads, 0, s>>>(L, h[1], phi, b0f[1], U[1], L.by));
    if (dim == 3) {
        long long mz = (long long)L.nx * L.ny * (L.nz + 1);
        MGP_LAUNCH(k_project<2><<<nb(mz), kThreads, 0, s>>>(L, h[2], phi, b0f[2], U[2], L.bz));
    }
}

template <typename T>
void cell_dense_assemble(int dim, const CellLevel<T>& L, double* A, int lda, cudaStream_t s)
{
    long long N = (long long)L.nx * L.ny * L.nz;
    if (dim == 2) MGP_LAUNCH(k_dense_assemble<2, T><<<nb(N * N), kThreads, 0, s>>>(L, A, lda));
    else MGP_LAUNCH(k_dense_assemble<3, T><<<nb(N * N), kThreads, 0, s>>>(L, A, lda));
}

template void cell_gsrb<float>(int, const CellLevel<float>&, float*, const float*, int, cudaStream_t);
template void cell_gsrb<double>(int, const CellLevel<double>&, double*, const double*, int, cudaStream_t);
template void cell_resid_restrict<float>(int, const CellLevel<float>&, const float*, const float*, float*, cudaStream_t);
template void cell_resid_restrict<double>(int, const CellLevel<double>&, const double*, const double*, double*,
                                          cudaStream_t);
template void cell_prolong_add<float>(int, const CellLevel<float>&, const CellLevel<float>&, float*, const float*, int,
                                      cudaStream_t);
template void cell_prolong_add<double>(int, const CellLevel<double>&, const CellLevel<double>&, double*,
                                       const double*, int, cudaStream_t);
template void cell_dense_assemble<float>(int, const CellLevel<float>&, double*, int, cudaStream_t);
template void cell_dense_assemble<double>(int, const CellLevel<double>&, double*, int, cudaStream_t);

}  // namespace mgp
