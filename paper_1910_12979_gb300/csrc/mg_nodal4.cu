// mg_nodal4.cu -- FP32 nodal Jacobi sweep and residual, four nodes per thread.
//
// The counterpart of k_gsrb_v4 for the Q1 nodal operator: a thread owns four
// consecutive nodes of an x-row and keeps in registers everything their rows
// need -- phi on the 3 x 3 rows/planes around them (16-byte loads plus the two
// x-neighbours), sigma of the 2 x 2 cell rows/planes (16-byte loads plus the
// cell left of the quad) and b -- instead of staging tiles in shared memory;
// warps cover 32 consecutive quads, so every access is coalesced.  Cells
// outside a non-periodic boundary read sigma 0 and add 0 * (...), which leaves
// the sums unchanged.  The row arithmetic -- cells in node_row's order, the four
// phi of a cell summed left to right, the fused multiply-adds -- is that of
// k_jacobi / k_node_resid, so the results are identical.  Requirements
// (checked by the launcher): FP32, 3-D, x periodic (nodes = cells along x),
// nx % 4 == 0.
#include "mg_nodal.cuh"

namespace mgp {

namespace {

__device__ __forceinline__ float4 nld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

}  // namespace

template <bool RESID>
__global__ void __launch_bounds__(256, 4)
k_node_jacobi_v4(NodeLevel<float> L, const float* __restrict__ x, float* __restrict__ out,
                 const float* __restrict__ b, float omega)
{
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (4 * q >= Nx || j >= Ny) return;
    const int i0 = 4 * q;
    const bool py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const size_t nplane = (size_t)Nx * Ny, cplane = (size_t)nx * ny;

    // one node plane k + dz of phi: rows j - 1 .. j + 1, columns i0 - 1 .. i0 + 4 (x periodic)
    auto load_phi = [&](int dz, float (&r)[3][6]) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            int jj = j + dy, kk = k + dz;
            bool ok = true;
            if (jj < 0 || jj >= Ny) { if (py) jj = jj < 0 ? jj + Ny : jj - Ny; else ok = false; }
            if (kk < 0 || kk >= Nz) { if (pz) kk = kk < 0 ? kk + Nz : kk - Nz; else ok = false; }
            if (ok) {
                const float* row = x + (size_t)kk * nplane + (size_t)jj * Nx;
                const float4 v = nld4(row + i0);
                r[dy + 1][0] = row[i0 > 0 ? i0 - 1 : Nx - 1];
                r[dy + 1][1] = v.x; r[dy + 1][2] = v.y; r[dy + 1][3] = v.z; r[dy + 1][4] = v.w;
                r[dy + 1][5] = row[i0 + 4 < Nx ? i0 + 4 : 0];
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) r[dy + 1][c] = 0.f;
            }
        }
    };
    // one cell plane k - 1 + cz of sigma: rows j - 1, j; columns i0 - 1 .. i0 + 3 (0 outside)
    auto load_sig = [&](int cz, float (&r)[2][5]) {
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            int cj, ck;
            if (cell_ok(j - 1 + cy, ny, L.bc.lo[1], cj) && cell_ok(k - 1 + cz, nz, L.bc.lo[2], ck)) {
                const float* row = L.sigma + (size_t)ck * cplane + (size_t)cj * nx;
                const float4 v = nld4(row + i0);
                r[cy][0] = row[i0 > 0 ? i0 - 1 : nx - 1];
                r[cy][1] = v.x; r[cy][2] = v.y; r[cy][3] = v.z; r[cy][4] = v.w;
            } else {
#pragma unroll
                for (int c = 0; c < 5; ++c) r[cy][c] = 0.f;
            }
        }
    };
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, ssum[4] = {0.f, 0.f, 0.f, 0.f};
    float xi[4];
    // the cells below the node plane (node_row's c = 0..3), then those above (c = 4..7);
    // pm: the node plane on the cells' far side, p0: node plane k
    float p0[3][6], pm[3][6], sg[2][5];
    load_phi(0, p0);
#pragma unroll
    for (int p = 0; p < 4; ++p) xi[p] = p0[1][p + 1];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        load_phi(half ? 1 : -1, pm);
        load_sig(half, sg);
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1;
                const float s = sg[sy > 0 ? 1 : 0][sx > 0 ? p + 1 : p];
                const int a = p + 1 + sx;  // phi column of node i + sx
                const float v = ((p0[1 + sy][a] + pm[1][a]) + pm[1 + sy][p + 1]) + pm[1 + sy][a];
                acc[p] = fmadd(s, v, acc[p]);
                ssum[p] += s;
            }
    }
    const float4 bb = nld4(b + (size_t)k * nplane + (size_t)j * Nx + i0);
    const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
    const float c12 = L.ih2 / 12.f, c3 = L.ih2 / 3.f;
    float res[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float off = acc[p] * c12;
        const float dg = -ssum[p] * c3;
        if (node_dirichlet(L, i0 + p, j, k, 3)) {
            res[p] = 0.f;
        } else if (RESID) {
            res[p] = bv[p] - fmadd(dg, xi[p], off);
        } else {
            res[p] = fmadd(omega * (bv[p] - fmadd(dg, xi[p], off)), recip(dg), xi[p]);
        }
    }
    *reinterpret_cast<float4*>(out + (size_t)k * nplane + (size_t)j * Nx + i0) =
        make_float4(res[0], res[1], res[2], res[3]);
}

bool node_v4_ok(int dim, const NodeLevel<float>& L, const float* x, const float* out, const float* b)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return dim == 3 && L.bc.lo[0] == BCP && L.nx % 4 == 0 && L.nx >= 8 && L.Nx == L.nx && L.invd == nullptr &&
           a16(x) && a16(out) && a16(b) && a16(L.sigma);
}

void node_v4(const NodeLevel<float>& L, const float* x, float* out, const float* b, float omega, bool resid,
             cudaStream_t s, int bxw)
{
    const int nq = L.Nx / 4;
    const int bx = bxw > 0 ? bxw : nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, 256 / bx);
    const dim3 grid((nq + bx - 1) / bx, (L.Ny + block.y - 1) / block.y, L.Nz);
    if (resid) MGP_LAUNCH(k_node_jacobi_v4<true><<<grid, block, 0, s>>>(L, x, out, b, omega));
    else MGP_LAUNCH(k_node_jacobi_v4<false><<<grid, block, 0, s>>>(L, x, out, b, omega));
}

}  // namespace mgp

namespace mgp {

// Trilinear prolongation and correction of nodal FP32 levels, four fine nodes
// of a row per thread (one 16-byte read-modify-write); coarse values through
// L1.  Same weights and order of operations as k_node_prolong.  Requirements:
// x periodic, Nx % 4 == 0.
__global__ void __launch_bounds__(256)
k_node_prolong_v4(NodeLevel<float> F, NodeLevel<float> C, float* __restrict__ xf, const float* __restrict__ xc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (4 * q >= F.Nx || j >= F.Ny) return;
    const int i0 = 4 * q;
    const size_t id = ((size_t)k * F.Ny + j) * F.Nx + i0;
    float4 v = *reinterpret_cast<const float4*>(xf + id);
    float o[4] = {v.x, v.y, v.z, v.w};
    const int cy0 = j >> 1, ny_ = 1 + (j & 1), cz0 = k >> 1, nz_ = 1 + (k & 1);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + p;
        if (node_dirichlet(F, i, j, k, 3)) continue;
        const int cx0 = i >> 1, nx_ = 1 + (i & 1);
        float s = 0.f;
        for (int c = 0; c < nz_; ++c)
            for (int b = 0; b < ny_; ++b)
                for (int a = 0; a < nx_; ++a) {
                    int qx = cx0 + a, qy = cy0 + b, qz = cz0 + c;
                    float w = 1.f;
                    if (nx_ == 2) w *= 0.5f;
                    if (qx >= C.Nx) qx -= C.Nx;   // x periodic
                    if (ny_ == 2) w *= 0.5f;
                    if (C.bc.lo[1] == BCP && qy >= C.Ny) qy -= C.Ny;
                    if (nz_ == 2) w *= 0.5f;
                    if (C.bc.lo[2] == BCP && qz >= C.Nz) qz -= C.Nz;
                    s += w * xc[((size_t)qz * C.Ny + qy) * C.Nx + qx];
                }
        o[p] += s;
    }
    *reinterpret_cast<float4*>(xf + id) = make_float4(o[0], o[1], o[2], o[3]);
}

bool node_prolong_v4_ok(int dim, const NodeLevel<float>& F, const float* xf)
{
    return dim == 3 && F.bc.lo[0] == BCP && F.Nx % 4 == 0 && F.Nx >= 8 && ((uintptr_t)xf & 15) == 0;
}

void node_prolong_v4(const NodeLevel<float>& F, const NodeLevel<float>& C, float* xf, const float* xc, cudaStream_t s)
{
    const int nq = F.Nx / 4;
    const int bx = nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, 256 / bx);
    const dim3 grid((nq + bx - 1) / bx, (F.Ny + block.y - 1) / block.y, F.Nz);
    MGP_LAUNCH(k_node_prolong_v4<<<grid, block, 0, s>>>(F, C, xf, xc));
}

}  // namespace mgp
