// mg_gsrb4.cu -- one colour pass of red-black Gauss-Seidel, four cells per thread.
//
// A thread owns four consecutive cells of an x-row and updates the two of them
// that have the pass's colour, in place.  Every operand comes in 16-byte loads
// where the layout allows: the four cells, the rows above and below, the
// planes in front and behind, b and the y- and z-face coefficients (x-faces
// have n+1 per row, so those are four scalar loads); the one x-neighbour
// outside the quad is a scalar load.  The quad is written back as one 16-byte
// store; its two cells of the other colour are rewritten with the values read,
// which nothing changes during the pass.  Warps cover 32 consecutive quads of
// a row, so every access is coalesced, and the instruction count per cell is a
// small fraction of a shared-memory tiled sweep's.  Levels whose x is the
// fastest axis of at most a few hundred kilobytes per plane keep the
// neighbouring planes in L2 between the rows that share them; b and the face
// arrays are read once per pass with the streaming cache hint.
//
// The row arithmetic -- the order of the six face terms, the boundary cases and
// the diagonal -- is that of k_gsrb (cell_row), so two passes of this kernel
// equal two passes of k_gsrb bit for bit.  Requirements (checked by the
// launcher): FP32, nx % 4 == 0.
#include "mg_cellquad.cuh"

namespace mgp {

namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4s(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float el(const float4& v, int p) { return p == 0 ? v.x : p == 1 ? v.y : p == 2 ? v.z : v.w; }

}  // namespace

template <int DIM>
__global__ void __launch_bounds__(256)
k_gsrb_v4(CellLevel<float> L, float* __restrict__ x, const float* __restrict__ b, int color)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (4 * q >= L.nx || j >= L.ny) return;
    gsrb4_quad<DIM, false>(L, x, b, color, q, j, k, false);
}

bool cell_gsrb_v4_ok(int dim, const CellLevel<float>& L, const float* x, const float* b)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return L.nx % 4 == 0 && L.nx >= 8 && L.invd == nullptr && a16(x) && a16(b) && a16(L.by) &&
           (dim == 2 || a16(L.bz));
}

void cell_gsrb_v4(int dim, const CellLevel<float>& L, float* x, const float* b, int color, cudaStream_t s, int bxw)
{
    const int nq = L.nx / 4;
    const int bx = bxw > 0 ? bxw : nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, 256 / bx);
    const dim3 grid((nq + bx - 1) / bx, (L.ny + block.y - 1) / block.y, dim == 3 ? L.nz : 1);
    if (dim == 2) MGP_LAUNCH(k_gsrb_v4<2><<<grid, block, 0, s>>>(L, x, b, color));
    else MGP_LAUNCH(k_gsrb_v4<3><<<grid, block, 0, s>>>(L, x, b, color));
}

}  // namespace mgp

namespace mgp {

// Residual r = b - L x of a 3-D FP32 level averaged over the 2 x 2 x 2 children
// of each coarse cell, vectorised like k_gsrb_v4.  A thread owns one quad of
// four x-cells in one fine row and plane; the lanes along x are consecutive
// quads of the same row, so every load is a contiguous run, and a block holds
// the four fine rows of two coarse rows in the two fine planes of a coarse
// plane (threadIdx.y, threadIdx.z).  The x-neighbours of a quad come from the
// neighbouring lanes by shuffles (a load only at the ends of a warp's run of
// quads); the five x-faces are scalar loads (one aligned 16-byte load plus
// shuffles and a data-dependent select measured slower).  Each thread sums its
// residuals over x-pairs; the row and plane pairs are added through shared
// memory by the threads of the lower fine row and plane.  The per-cell
// arithmetic and the order of the sums (x pair, then y, then z) are those of
// k_resid_restrict_t, so the coarse right-hand sides are identical.
// Requirements: nx % 4 == 0, ny and nz even; blocks of (32 or a divisor of 32)
// x 4 x 2 threads.
constexpr int kRRy = 4;
__global__ void __launch_bounds__(256, 4)
k_resid_restrict_v4(CellLevel<float> F, const float* __restrict__ x, const float* __restrict__ b,
                    float* __restrict__ bc)
{
    __shared__ float2 part[2][kRRy][32];
    const int nx = F.nx, ny = F.ny, nz = F.nz, nq = nx / 4;
    const int qg = blockIdx.x * blockDim.x + threadIdx.x;      // quad along x
    const int jg = blockIdx.y * kRRy + threadIdx.y;             // fine row
    const bool live = qg < nq && jg < ny;
    // lanes past the end work on the last quad / row (their results are
    // dropped), so that every lane of a warp takes part in the shuffles
    const int q = qg < nq ? qg : nq - 1, j = jg < ny ? jg : ny - 1;
    const int k = 2 * blockIdx.z + threadIdx.z;
    const bool first = threadIdx.x == 0 || q == 0, last = threadIdx.x == blockDim.x - 1 || q == nq - 1;
    const int i0 = 4 * q;
    const size_t plane = (size_t)nx * ny;
    const bool px = F.bc.lo[0] == BCP, py = F.bc.lo[1] == BCP, pz = F.bc.lo[2] == BCP;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t row = (size_t)k * plane + (size_t)j * nx;
    const bool hym = j > 0 || py, hyp = j < ny - 1 || py;
    const bool hzm = k > 0 || pz, hzp = k < nz - 1 || pz;
    const size_t rym = j > 0 ? row - nx : row + (size_t)(ny - 1) * nx;
    const size_t ryp = j < ny - 1 ? row + nx : row - (size_t)(ny - 1) * nx;
    const size_t rzm = k > 0 ? row - plane : row + (size_t)(nz - 1) * plane;
    const size_t rzp = k < nz - 1 ? row + plane : row - (size_t)(nz - 1) * plane;
    const float4 xc = ld4(x + row + i0);
    const float4 bb = ld4s(b + row + i0);
    const float4 xym = hym ? ld4(x + rym + i0) : zero4;
    const float4 xyp = hyp ? ld4(x + ryp + i0) : zero4;
    const float4 xzm = hzm ? ld4(x + rzm + i0) : zero4;
    const float4 xzp = hzp ? ld4(x + rzp + i0) : zero4;
    const size_t fxb = ((size_t)k * ny + j) * (nx + 1) + i0;
    const float fx[5] = {__ldcs(F.bx + fxb), __ldcs(F.bx + fxb + 1), __ldcs(F.bx + fxb + 2),
                         __ldcs(F.bx + fxb + 3), __ldcs(F.bx + fxb + 4)};
    const size_t fyb = ((size_t)k * (ny + 1) + j) * nx + i0;
    const float4 fyl = ld4s(F.by + fyb), fyh = ld4s(F.by + fyb + nx);
    const float4 fzl = ld4s(F.bz + row + i0), fzh = ld4s(F.bz + row + plane + i0);
    // x-neighbours of the quad: the neighbouring lanes' edge cells
    float xl = __shfl_up_sync(0xffffffffu, xc.w, 1), xr = __shfl_down_sync(0xffffffffu, xc.x, 1);
    if (first) xl = i0 > 0 ? x[row + i0 - 1] : (px ? x[row + nx - 1] : 0.f);
    if (last) xr = i0 + 4 < nx ? x[row + i0 + 4] : (px ? x[row] : 0.f);
    const float xs[6] = {xl, xc.x, xc.y, xc.z, xc.w, xr};
    float r[4];
    // quads away from every non-periodic boundary: the same operations in the
    // same order, without the per-face presence tests
    const bool inner = hym && hyp && hzm && hzp && (px || (i0 > 0 && i0 + 4 < nx));
    if (inner) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float off = 0.f, dg = 0.f;
            off = fmadd(fx[p], xs[p], off); dg += fx[p];
            off = fmadd(fx[p + 1], xs[p + 2], off); dg += fx[p + 1];
            const float byl = el(fyl, p), byh = el(fyh, p);
            off = fmadd(byl, el(xym, p), off); dg += byl;
            off = fmadd(byh, el(xyp, p), off); dg += byh;
            const float bzl = el(fzl, p), bzh = el(fzh, p);
            off = fmadd(bzl, el(xzm, p), off); dg += bzl;
            off = fmadd(bzh, el(xzp, p), off); dg += bzh;
            r[p] = el(bb, p) - fmadd(-dg, xs[p + 1], off);
        }
    } else
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + p;
        float off = 0.f, dg = 0.f;
        const float bxl = fx[p], bxh = fx[p + 1];
        if (i > 0 || px) { off = fmadd(bxl, xs[p], off); dg += bxl; }
        else if (F.bc.lo[0] == BCD) { dg += 2.f * bxl; }
        if (i < nx - 1 || px) { off = fmadd(bxh, xs[p + 2], off); dg += bxh; }
        else if (F.bc.hi[0] == BCD) { dg += 2.f * bxh; }
        const float byl = el(fyl, p), byh = el(fyh, p);
        if (hym) { off = fmadd(byl, el(xym, p), off); dg += byl; }
        else if (F.bc.lo[1] == BCD) { dg += 2.f * byl; }
        if (hyp) { off = fmadd(byh, el(xyp, p), off); dg += byh; }
        else if (F.bc.hi[1] == BCD) { dg += 2.f * byh; }
        const float bzl = el(fzl, p), bzh = el(fzh, p);
        if (hzm) { off = fmadd(bzl, el(xzm, p), off); dg += bzl; }
        else if (F.bc.lo[2] == BCD) { dg += 2.f * bzl; }
        if (hzp) { off = fmadd(bzh, el(xzp, p), off); dg += bzh; }
        else if (F.bc.hi[2] == BCD) { dg += 2.f * bzh; }
        r[p] = el(bb, p) - fmadd(-dg, xs[p + 1], off);
    }
    part[threadIdx.z][threadIdx.y][threadIdx.x] = make_float2(r[0] + r[1], r[2] + r[3]);
    __syncthreads();
    if (live && threadIdx.z == 0 && (threadIdx.y & 1) == 0) {
        const float2 a0 = part[0][threadIdx.y][threadIdx.x], a1 = part[0][threadIdx.y + 1][threadIdx.x];
        const float2 c0 = part[1][threadIdx.y][threadIdx.x], c1 = part[1][threadIdx.y + 1][threadIdx.x];
        const int cnx = nx / 2, cny = ny / 2;
        float2 v;
        v.x = ((a0.x + a1.x) + (c0.x + c1.x)) * 0.125f;
        v.y = ((a0.y + a1.y) + (c0.y + c1.y)) * 0.125f;
        *reinterpret_cast<float2*>(bc + ((size_t)blockIdx.z * cny + (jg >> 1)) * cnx + 2 * q) = v;
    }
}

bool cell_resid_restrict_v4_ok(int dim, const CellLevel<float>& F, const float* x, const float* b, const float* bc)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return dim == 3 && F.nx % 4 == 0 && F.nx >= 8 && F.ny % 2 == 0 && F.nz % 2 == 0 && a16(x) && a16(b) &&
           a16(F.bx) && a16(F.by) && a16(F.bz) && ((uintptr_t)bc & 7) == 0;
}

void cell_resid_restrict_v4(const CellLevel<float>& F, const float* x, const float* b, float* bc, cudaStream_t s)
{
    const int nq = F.nx / 4, cny = F.ny / 2, cnz = F.nz / 2;
    const int bx = nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, kRRy, 2);
    const dim3 grid((nq + bx - 1) / bx, (2 * cny + kRRy - 1) / kRRy, cnz);
    MGP_LAUNCH(k_resid_restrict_v4<<<grid, block, 0, s>>>(F, x, b, bc));
}

}  // namespace mgp

namespace mgp {

// Linear prolongation and correction, x_f += P x_c, four fine cells of a row per
// thread (one 16-byte read-modify-write).  The four cells share their coarse
// rows (parent and neighbour in y, times parent and neighbour in z) and, along
// x, the parents c0 = i0/2, c0+1 and the outer neighbours of cells i0 and i0+3:
// 4 x 4 coarse values (a pair load and two scalars per row, through L1), each
// x-interpolation formed once.  The arithmetic -- weights, fused multiply-adds
// and their order -- is prolong_value's, so the result equals k_prolong_add's.
__global__ void __launch_bounds__(256)
k_prolong_add_v4(CellLevel<float> F, CellLevel<float> C, float* __restrict__ xf, const float* __restrict__ xc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (4 * q >= F.nx || j >= F.ny) return;
    prolong4_quad<false>(F, C, xf, xc, q, j, k);
}

bool cell_prolong_v4_ok(int dim, const CellLevel<float>& F, const float* xf, const float* xc)
{
    return dim == 3 && F.nx % 4 == 0 && F.nx >= 8 && ((uintptr_t)xf & 15) == 0 && ((uintptr_t)xc & 7) == 0;
}

void cell_prolong_v4(const CellLevel<float>& F, const CellLevel<float>& C, float* xf, const float* xc, cudaStream_t s)
{
    const int nq = F.nx / 4;
    const int bx = nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, 256 / bx);
    const dim3 grid((nq + bx - 1) / bx, (F.ny + block.y - 1) / block.y, F.nz);
    MGP_LAUNCH(k_prolong_add_v4<<<grid, block, 0, s>>>(F, C, xf, xc));
}

}  // namespace mgp
