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
__global__ void __launch_bounds__(256)
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
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    // phi rows: index [dy + 1][dz + 1] for node rows j + dy, planes k + dz; six
    // columns i0 - 1 .. i0 + 4 (x periodic: wrapped)
    float ph[3][3][6];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            int jj = j + dy, kk = k + dz;
            bool ok = true;
            if (jj < 0 || jj >= Ny) { if (py) jj = jj < 0 ? jj + Ny : jj - Ny; else ok = false; }
            if (kk < 0 || kk >= Nz) { if (pz) kk = kk < 0 ? kk + Nz : kk - Nz; else ok = false; }
            float* r = ph[dy + 1][dz + 1];
            if (ok) {
                const float* row = x + (size_t)kk * nplane + (size_t)jj * Nx;
                const float4 v = nld4(row + i0);
                r[0] = row[i0 > 0 ? i0 - 1 : Nx - 1];
                r[1] = v.x; r[2] = v.y; r[3] = v.z; r[4] = v.w;
                r[5] = row[i0 + 4 < Nx ? i0 + 4 : 0];
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) r[c] = 0.f;
            }
        }
    // sigma: [cy][cz] for cell rows j - 1 + cy, planes k - 1 + cz; five columns i0 - 1 .. i0 + 3
    float sg[2][2][5];
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            int cj, ck;
            const bool ok = cell_ok(j - 1 + cy, ny, L.bc.lo[1], cj) && cell_ok(k - 1 + cz, nz, L.bc.lo[2], ck);
            float* r = sg[cy][cz];
            if (ok) {
                const float* row = L.sigma + (size_t)ck * cplane + (size_t)cj * nx;
                const float4 v = nld4(row + i0);
                r[0] = row[i0 > 0 ? i0 - 1 : nx - 1];
                r[1] = v.x; r[2] = v.y; r[3] = v.z; r[4] = v.w;
            } else {
#pragma unroll
                for (int c = 0; c < 5; ++c) r[c] = 0.f;
            }
        }
    const float4 bb = nld4(b + (size_t)k * nplane + (size_t)j * Nx + i0);
    const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
    const float c12 = L.ih2 / 12.f, c3 = L.ih2 / 3.f;
    float res[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float acc = 0.f, ssum = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1, sz = (c & 4) ? 1 : -1;
            const float s = sg[sy > 0 ? 1 : 0][sz > 0 ? 1 : 0][sx > 0 ? p + 1 : p];
            const int a = p + 1 + sx;            // phi column of node i + sx
            const float v = ((ph[1 + sy][1][a] + ph[1][1 + sz][a]) + ph[1 + sy][1 + sz][p + 1]) +
                            ph[1 + sy][1 + sz][a];
            acc = fmadd(s, v, acc);
            ssum += s;
        }
        const float off = acc * c12;
        const float dg = -ssum * c3;
        const float xi = ph[1][1][p + 1];
        if (node_dirichlet(L, i0 + p, j, k, 3)) {
            res[p] = 0.f;
        } else if (RESID) {
            res[p] = bv[p] - fmadd(dg, xi, off);
        } else {
            res[p] = fmadd(omega * (bv[p] - fmadd(dg, xi, off)), recip(dg), xi);
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
             cudaStream_t s)
{
    const int nq = L.Nx / 4;
    const int bx = nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, 256 / bx);
    const dim3 grid((nq + bx - 1) / bx, (L.Ny + block.y - 1) / block.y, L.Nz);
    if (resid) MGP_LAUNCH(k_node_jacobi_v4<true><<<grid, block, 0, s>>>(L, x, out, b, omega));
    else MGP_LAUNCH(k_node_jacobi_v4<false><<<grid, block, 0, s>>>(L, x, out, b, omega));
}

}  // namespace mgp
