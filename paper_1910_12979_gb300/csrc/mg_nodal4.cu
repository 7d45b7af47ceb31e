// mg_nodal4.cu -- FP32 nodal Jacobi sweep and residual, four nodes per thread.
//
// The counterpart of k_gsrb_v4 for the Q1 nodal operator: a thread owns four
// consecutive nodes of an x-row and keeps in registers everything their rows
// need -- phi on the 3 x 3 rows/planes around them (16-byte loads plus the two
// x-neighbours), sigma of the 2 x 2 cell rows/planes (16-byte loads plus the
// cell left of the quad) and b -- instead of staging tiles in shared memory;
// warps cover 32 consecutive quads, so every access is coalesced.  With KZ > 1
// a thread marches up KZ node planes and keeps a rolling window of three phi
// planes and two sigma planes, so each plane costs 3 phi rows, 2 sigma rows and
// b (14 loads) instead of 9 + 4 + 1 (36), with the row and boundary index work
// done once per thread (the one-plane kernel is bound by instruction issue,
// not bytes), and the loads of a step are issued a step ahead of their use.  Cells
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

template <bool RESID, int KZ>
__global__ void __launch_bounds__(256, KZ > 1 ? 2 : 4)
k_node_jacobi_v4(NodeLevel<float> L, const float* __restrict__ x, float* __restrict__ out,
                 const float* __restrict__ b, float omega)
{
    const int Nx = L.Nx, Ny = L.Ny, Nz = L.Nz, nx = L.nx, ny = L.ny, nz = L.nz;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z * KZ;
    if (4 * q >= Nx || j >= Ny) return;
    const int i0 = 4 * q;
    const bool pz = L.bc.lo[2] == BCP;
    const size_t nplane = (size_t)Nx * Ny, cplane = (size_t)nx * ny;
    const int il = i0 > 0 ? i0 - 1 : Nx - 1, ih = i0 + 4 < Nx ? i0 + 4 : 0;   // x periodic: Nx == nx
    // offsets within a plane of node rows j - 1 .. j + 1 and of cell rows j - 1, j (-1: absent)
    int prow[3], crow[2];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        int jj = j - 1 + dy;
        if (jj < 0 || jj >= Ny) jj = L.bc.lo[1] == BCP ? (jj < 0 ? jj + Ny : jj - Ny) : -1;
        prow[dy] = jj < 0 ? -1 : jj * Nx;
    }
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
        int cj;
        crow[cy] = cell_ok(j - 1 + cy, ny, L.bc.lo[1], cj) ? cj * nx : -1;
    }

    // one node plane kk of phi: rows j - 1 .. j + 1, columns i0 - 1 .. i0 + 4
    auto load_phi = [&](int kk, float (&r)[3][6]) {
        bool ok = true;
        if (kk < 0 || kk >= Nz) { if (pz) kk = kk < 0 ? kk + Nz : kk - Nz; else ok = false; }
        const float* pl = x + (size_t)(ok ? kk : 0) * nplane;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            if (ok && prow[dy] >= 0) {
                const float* row = pl + prow[dy];
                const float4 v = nld4(row + i0);
                r[dy][0] = row[il];
                r[dy][1] = v.x; r[dy][2] = v.y; r[dy][3] = v.z; r[dy][4] = v.w;
                r[dy][5] = row[ih];
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) r[dy][c] = 0.f;
            }
        }
    };
    // one cell plane ckr of sigma: rows j - 1, j; columns i0 - 1 .. i0 + 3 (0 outside)
    auto load_sig = [&](int ckr, float (&r)[2][5]) {
        int ck = 0;
        const bool okz = cell_ok(ckr, nz, L.bc.lo[2], ck);
        const float* pl = L.sigma + (size_t)(okz ? ck : 0) * cplane;
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            if (okz && crow[cy] >= 0) {
                const float* row = pl + crow[cy];
                const float4 v = nld4(row + i0);
                r[cy][0] = row[il];
                r[cy][1] = v.x; r[cy][2] = v.y; r[cy][3] = v.z; r[cy][4] = v.w;
            } else {
#pragma unroll
                for (int c = 0; c < 5; ++c) r[cy][c] = 0.f;
            }
        }
    };

    // rolling window of node planes k - 1 .. k + 1 and cell planes k - 1, k.  The
    // eight cells of a node are summed in node_row's order: the four below the
    // node plane (half 0), then the four above (half 1).  Half 0 of plane k + 1
    // needs nothing newer than plane k + 1, so it is computed in step k, after
    // half 1 of plane k, while the loads of planes k + 2 (phi) and k + 1
    // (sigma), issued at the top of step k, are in flight: a load has a whole
    // step of arithmetic to arrive.
    float P[3][3][6], S[2][2][5];
    float acc[4], ssum[4];
    const float c12 = L.ih2 / 12.f, c3 = L.ih2 / 3.f;
    // cells on one side of node plane k: pc = plane k, pm = the node plane on the cells' far side
    auto half_sum = [&](const float(&pc)[3][6], const float(&pm)[3][6], const float(&sg)[2][5]) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1;
                const float sv = sg[sy > 0 ? 1 : 0][sx > 0 ? p + 1 : p];
                const int a = p + 1 + sx;  // phi column of node i + sx
                const float v = ((pc[1 + sy][a] + pm[1][a]) + pm[1 + sy][p + 1]) + pm[1 + sy][a];
                acc[p] = fmadd(sv, v, acc[p]);
                ssum[p] += sv;
            }
    };
    load_phi(k0 - 1, P[0]);
    load_phi(k0, P[1]);
    load_sig(k0 - 1, S[0]);
    if (KZ > 1) {
        load_phi(k0 + 1, P[2]);
        load_sig(k0, S[1]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[p] = ssum[p] = 0.f;
    half_sum(P[1], P[0], S[0]);
#pragma unroll
    for (int t = 0; t < KZ; ++t) {
        const int k = k0 + t;
        if (k >= Nz) break;
        const bool more = t + 1 < KZ && k + 1 < Nz;   // node plane k + 1 belongs to this thread
        if (KZ == 1) {
            load_phi(k + 1, P[2]);
            load_sig(k, S[1]);
        } else if (more) {
            load_phi(k + 2, P[t % 3]);
            load_sig(k + 1, S[t % 2]);
        }
        const size_t id = (size_t)k * nplane + (size_t)j * Nx + i0;
        const float4 bb = nld4(b + id);
        const float(&pc)[3][6] = P[(t + 1) % 3];
        half_sum(pc, P[(t + 2) % 3], S[(t + 1) % 2]);
        const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
        float res[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float xi = pc[1][p + 1];
            const float off = acc[p] * c12;
            const float dg = -ssum[p] * c3;
            if (node_dirichlet(L, i0 + p, j, k, 3)) {
                res[p] = 0.f;
            } else if (RESID) {
                res[p] = bv[p] - fmadd(dg, xi, off);
            } else {
                res[p] = fmadd(omega * (bv[p] - fmadd(dg, xi, off)), recip(dg), xi);
            }
        }
        *reinterpret_cast<float4*>(out + id) = make_float4(res[0], res[1], res[2], res[3]);
        if (more) {
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[p] = ssum[p] = 0.f;
            half_sum(P[(t + 2) % 3], pc, S[(t + 1) % 2]);
        }
    }
}

bool node_v4_ok(int dim, const NodeLevel<float>& L, const float* x, const float* out, const float* b)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return dim == 3 && L.bc.lo[0] == BCP && L.nx % 4 == 0 && L.nx >= 8 && L.Nx == L.nx && L.invd == nullptr &&
           a16(x) && a16(out) && a16(b) && a16(L.sigma);
}

void node_v4(const NodeLevel<float>& L, const float* x, float* out, const float* b, float omega, bool resid,
             cudaStream_t s, int bxw, int kz)
{
    const int nq = L.Nx / 4;
    const int bx = bxw > 0 ? bxw : nq >= 32 ? 32 : nq >= 16 ? 16 : nq >= 8 ? 8 : nq >= 4 ? 4 : 2;
    const dim3 block(bx, 256 / bx);
    const long long cols = (long long)((nq + bx - 1) / bx) * ((L.Ny + block.y - 1) / block.y);
    // default: march eight (else four) planes per thread where that still
    // leaves at least two waves of two resident blocks per SM (256^3: the
    // eight-plane sweep takes 86 us, the four-plane one 96)
    if (kz <= 0)
        kz = cols * ((L.Nz + 7) / 8) >= 4LL * kNumSMs ? 8 : cols * ((L.Nz + 3) / 4) >= 4LL * kNumSMs ? 4 : 1;
    kz = kz == 8 ? 8 : kz == 4 ? 4 : 1;
    const dim3 grid((nq + bx - 1) / bx, (L.Ny + block.y - 1) / block.y, (L.Nz + kz - 1) / kz);
    if (kz == 8) {
        if (resid) MGP_LAUNCH(k_node_jacobi_v4<true, 8><<<grid, block, 0, s>>>(L, x, out, b, omega));
        else MGP_LAUNCH(k_node_jacobi_v4<false, 8><<<grid, block, 0, s>>>(L, x, out, b, omega));
    } else if (kz == 4) {
        if (resid) MGP_LAUNCH(k_node_jacobi_v4<true, 4><<<grid, block, 0, s>>>(L, x, out, b, omega));
        else MGP_LAUNCH(k_node_jacobi_v4<false, 4><<<grid, block, 0, s>>>(L, x, out, b, omega));
    } else {
        if (resid) MGP_LAUNCH(k_node_jacobi_v4<true, 1><<<grid, block, 0, s>>>(L, x, out, b, omega));
        else MGP_LAUNCH(k_node_jacobi_v4<false, 1><<<grid, block, 0, s>>>(L, x, out, b, omega));
    }
}

}  // namespace mgp

namespace mgp {

// Trilinear prolongation and correction of nodal FP32 levels, four fine nodes
// of a row per thread (one 16-byte read-modify-write).  Along x the four nodes
// i0 .. i0+3 (i0 = 4q, x periodic) use the coarse nodes c = i0/2, c+1 and c+2
// (node i0: c; i0+1: c, c+1; i0+2: c+1; i0+3: c+1, c+2), so each coarse row
// (one or two in y, times one or two in z) is read once: a pair load and a
// scalar through L1.  The weights and the order of the fused multiply-adds
// (z, then y, then x) are k_node_prolong's.  Requirements: x periodic,
// Nx % 4 == 0, xc 8-byte aligned.
__global__ void __launch_bounds__(256)
k_node_prolong_v4(NodeLevel<float> F, NodeLevel<float> C, float* __restrict__ xf, const float* __restrict__ xc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (4 * q >= F.Nx || j >= F.Ny) return;
    const int i0 = 4 * q, cx = 2 * q, cx2 = cx + 2 < C.Nx ? cx + 2 : cx + 2 - C.Nx;
    const size_t id = ((size_t)k * F.Ny + j) * F.Nx + i0;
    float4 v = *reinterpret_cast<const float4*>(xf + id);
    const int ny_ = 1 + (j & 1), nz_ = 1 + (k & 1);
    const float wyz = (ny_ == 2 ? 0.5f : 1.f) * (nz_ == 2 ? 0.5f : 1.f);
    const float we = wyz, wo = 0.5f * wyz;   // weights of even / odd nodes
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c = 0; c < nz_; ++c) {
        int qz = (k >> 1) + c;
        if (C.bc.lo[2] == BCP && qz >= C.Nz) qz -= C.Nz;
        for (int b = 0; b < ny_; ++b) {
            int qy = (j >> 1) + b;
            if (C.bc.lo[1] == BCP && qy >= C.Ny) qy -= C.Ny;
            const float* r = xc + ((size_t)qz * C.Ny + qy) * C.Nx;
            const float2 m = *reinterpret_cast<const float2*>(r + cx);
            const float x2 = r[cx2];
            s[0] = fmadd(we, m.x, s[0]);
            s[1] = fmadd(wo, m.y, fmadd(wo, m.x, s[1]));
            s[2] = fmadd(we, m.y, s[2]);
            s[3] = fmadd(wo, x2, fmadd(wo, m.y, s[3]));
        }
    }
    float o[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (!node_dirichlet(F, i0 + p, j, k, 3)) o[p] += s[p];
    *reinterpret_cast<float4*>(xf + id) = make_float4(o[0], o[1], o[2], o[3]);
}

bool node_prolong_v4_ok(int dim, const NodeLevel<float>& F, const float* xf, const float* xc)
{
    return dim == 3 && F.bc.lo[0] == BCP && F.Nx % 4 == 0 && F.Nx >= 8 && ((uintptr_t)xf & 15) == 0 &&
           ((uintptr_t)xc & 7) == 0;
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

namespace mgp {

// Full-weighting restriction b_c = 2^-3 sum w r_f of FP32 nodal levels, two
// coarse nodes (2q, 2q+1) of a row per thread.  With x periodic their fine
// x-positions 4q-1 .. 4q+3 are one 16-byte load and one scalar per fine row;
// the (up to) 3 x 3 fine rows are visited in k_node_restrict's order (z, then
// y, then x: -1, 0, +1) with the same weights and fused multiply-adds, so the
// coarse values are identical.  Requirements: 3-D, x periodic, nx % 4 == 0.
__global__ void __launch_bounds__(256)
k_node_restrict_v4(NodeLevel<float> F, NodeLevel<float> C, const float* __restrict__ rf, float* __restrict__ bc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;   // coarse nodes 2q, 2q + 1
    const int j = blockIdx.y * blockDim.y + threadIdx.y;   // coarse row
    const int k = blockIdx.z;                              // coarse plane
    if (2 * q >= C.Nx || j >= C.Ny) return;
    const int f0 = 4 * q, fl = f0 > 0 ? f0 - 1 : F.Nx - 1;
    float s0 = 0.f, s1 = 0.f;
    for (int oz = -1; oz <= 1; ++oz) {
        int c;
        if (!fine_pos(2 * k + oz, F.nz, F.bc.lo[2], c)) continue;
        const float wz = (oz == 0) ? 1.f : 0.5f;
        for (int oy = -1; oy <= 1; ++oy) {
            int b;
            if (!fine_pos(2 * j + oy, F.ny, F.bc.lo[1], b)) continue;
            const float wy = (oy == 0) ? 1.f : 0.5f;
            const float* r = rf + ((size_t)c * F.Ny + b) * F.Nx;
            const float4 v = nld4(r + f0);
            const float vl = r[fl];
            const float wh = wz * wy * 0.5f, w1 = wz * wy * 1.f;
            s0 = fmadd(wh, v.y, fmadd(w1, v.x, fmadd(wh, vl, s0)));
            s1 = fmadd(wh, v.w, fmadd(w1, v.z, fmadd(wh, v.y, s1)));
        }
    }
    float2 o;
    o.x = node_dirichlet(C, 2 * q, j, k, 3) ? 0.f : s0 * (1.f / 8.f);
    o.y = node_dirichlet(C, 2 * q + 1, j, k, 3) ? 0.f : s1 * (1.f / 8.f);
    *reinterpret_cast<float2*>(bc + ((size_t)k * C.Ny + j) * C.Nx + 2 * q) = o;
}

bool node_restrict_v4_ok(int dim, const NodeLevel<float>& F, const float* rf, const float* bc)
{
    return dim == 3 && F.bc.lo[0] == BCP && F.nx % 4 == 0 && F.Nx == F.nx && ((uintptr_t)rf & 15) == 0 &&
           ((uintptr_t)bc & 7) == 0;
}

void node_restrict_v4(const NodeLevel<float>& F, const NodeLevel<float>& C, const float* rf, float* bc, cudaStream_t s)
{
    const int np = C.Nx / 2;
    const int bx = np >= 32 ? 32 : np >= 16 ? 16 : np >= 8 ? 8 : np >= 4 ? 4 : np >= 2 ? 2 : 1;
    const dim3 block(bx, 256 / bx);
    const dim3 grid((np + bx - 1) / bx, (C.Ny + block.y - 1) / block.y, C.Nz);
    MGP_LAUNCH(k_node_restrict_v4<<<grid, block, 0, s>>>(F, C, rf, bc));
}

}  // namespace mgp
