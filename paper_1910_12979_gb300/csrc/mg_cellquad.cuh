// mg_cellquad.cuh -- per-quad arithmetic of the FP32 cell kernels.
//
// A "quad" is four consecutive cells of an x-row (i0 = 4q .. 4q + 3).  The
// colour pass, the residual of a quad and the linear prolongation onto a quad
// are written here once and called by the one-pass-per-launch kernels
// (k_gsrb_v4, k_prolong_add_v4) and by the pipelined fine-level kernel
// (k_cell_pipe), so that every path computes the same bits.  The only
// difference between the callers is how x is loaded: plain loads (L1-cached)
// where nothing else writes x during the launch, or ld.global.cg (served by L2,
// the point of coherence of the GPU) where other CTAs of the same launch write
// x.  The face terms are summed in cell_row's order (x, y, z; low face before
// high face), with explicit fused multiply-adds, so the results also equal the
// plain one-cell-per-thread kernels'.
#pragma once

#include "mg_cellops.cuh"

namespace mgp {

template <bool CG>
__device__ __forceinline__ float4 xld4(const float* p)
{
    if constexpr (CG) return __ldcg(reinterpret_cast<const float4*>(p));
    else return *reinterpret_cast<const float4*>(p);
}
template <bool CG>
__device__ __forceinline__ float xld1(const float* p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}
// b and the face coefficients are never written during these launches: the
// one-pass kernels stream them with the evict-first hint (each is read once
// per launch), the pipelined kernel reads them through the read-only path with
// normal L2 priority (every pass of the leg reads them again).
template <bool CG>
__device__ __forceinline__ float4 ro4(const float* p)
{
    if constexpr (CG) return __ldg(reinterpret_cast<const float4*>(p));
    else return __ldcs(reinterpret_cast<const float4*>(p));
}
template <bool CG>
__device__ __forceinline__ float ro1(const float* p)
{
    if constexpr (CG) return __ldg(p);
    else return __ldcs(p);
}
__device__ __forceinline__ float el4(const float4& v, int p) { return p == 0 ? v.x : p == 1 ? v.y : p == 2 ? v.z : v.w; }

// Operands of one colour-pass update of a quad: the quad, its rows and planes
// above and below, b, the x-neighbour outside the quad and the face
// coefficients of the two cells being updated.
struct Gs4 {
    float4 xc, bb, xym, xyp, xzm, xzp, fyl, fyh, fzl, fzh;
    float xout, fx0, fx1, fx2, fx3;
};

// Loads the operands of quad q of row j, plane k for the colour pass `color`.
// ZX: x is known to be zero everywhere (the first pass of a solve started from
// zero): no x is loaded and zeros take part in the same arithmetic.
template <int DIM, bool CG>
__device__ __forceinline__ void gs4_load(const CellLevel<float>& L, const float* __restrict__ x,
                                         const float* __restrict__ b, int color, int q, int j, int k, bool ZX, Gs4& g)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int i0 = 4 * q;
    const size_t plane = (size_t)nx * ny;
    const size_t row = (size_t)k * plane + (size_t)j * nx;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    g.xc = ZX ? zero4 : xld4<CG>(x + row + i0);
    g.bb = ro4<CG>(b + row + i0);
    // neighbour rows / planes (present: inside, or wrapped on a periodic axis)
    const bool hym = j > 0 || py, hyp = j < ny - 1 || py;
    const bool hzm = DIM == 3 && (k > 0 || pz), hzp = DIM == 3 && (k < nz - 1 || pz);
    const size_t rym = j > 0 ? row - nx : row + (size_t)(ny - 1) * nx;
    const size_t ryp = j < ny - 1 ? row + nx : row - (size_t)(ny - 1) * nx;
    const size_t rzm = k > 0 ? row - plane : row + (size_t)(nz - 1) * plane;
    const size_t rzp = k < nz - 1 ? row + plane : row - (size_t)(nz - 1) * plane;
    g.xym = hym && !ZX ? xld4<CG>(x + rym + i0) : zero4;
    g.xyp = hyp && !ZX ? xld4<CG>(x + ryp + i0) : zero4;
    g.xzm = hzm && !ZX ? xld4<CG>(x + rzm + i0) : zero4;
    g.xzp = hzp && !ZX ? xld4<CG>(x + rzp + i0) : zero4;
    // the cells of this colour are p0 and p0 + 2 (i0 is even)
    const int p0 = (color + j + k) & 1;
    // x-neighbour outside the quad: left of cell 0 (p0 == 0) or right of cell 3 (p0 == 1)
    g.xout = 0.f;
    if (!ZX) {
        if (p0 == 0) {
            if (i0 > 0) g.xout = xld1<CG>(x + row + i0 - 1);
            else if (px) g.xout = xld1<CG>(x + row + nx - 1);
        } else {
            if (i0 + 4 < nx) g.xout = xld1<CG>(x + row + i0 + 4);
            else if (px) g.xout = xld1<CG>(x + row);
        }
    }
    // face coefficients: x-faces i0+p0 .. i0+p0+3; y-faces of rows j, j+1; z-faces of planes k, k+1
    const size_t fxb = ((size_t)k * ny + j) * (nx + 1) + i0 + p0;
    g.fx0 = ro1<CG>(L.bx + fxb);
    g.fx1 = ro1<CG>(L.bx + fxb + 1);
    g.fx2 = ro1<CG>(L.bx + fxb + 2);
    g.fx3 = ro1<CG>(L.bx + fxb + 3);
    const size_t fyb = ((size_t)k * (ny + 1) + j) * nx + i0;
    g.fyl = ro4<CG>(L.by + fyb);
    g.fyh = ro4<CG>(L.by + fyb + nx);
    g.fzl = zero4;
    g.fzh = zero4;
    if (DIM == 3) {
        g.fzl = ro4<CG>(L.bz + row + i0);
        g.fzh = ro4<CG>(L.bz + row + plane + i0);
    }
}

// The quad after the colour pass: the two cells of colour `color`
// ((i + j + k) % 2 == color) get their Gauss-Seidel value, the other two keep
// the values read.
template <int DIM>
__device__ __forceinline__ float4 gs4_value(const CellLevel<float>& L, int color, int q, int j, int k, const Gs4& g)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int i0 = 4 * q;
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP, pz = L.bc.lo[2] == BCP;
    const bool hym = j > 0 || py, hyp = j < ny - 1 || py;
    const bool hzm = DIM == 3 && (k > 0 || pz), hzp = DIM == 3 && (k < nz - 1 || pz);
    const int p0 = (color + j + k) & 1;
    auto update = [&](int p, float bxl, float bxh, float xl, float xh) -> float {
        const int i = i0 + p;
        float off = 0.f, dg = 0.f;
        if (i > 0 || px) { off = fmadd(bxl, xl, off); dg += bxl; }
        else if (L.bc.lo[0] == BCD) { dg += 2.f * bxl; }
        if (i < nx - 1 || px) { off = fmadd(bxh, xh, off); dg += bxh; }
        else if (L.bc.hi[0] == BCD) { dg += 2.f * bxh; }
        const float byl = el4(g.fyl, p), byh = el4(g.fyh, p);
        if (hym) { off = fmadd(byl, el4(g.xym, p), off); dg += byl; }
        else if (L.bc.lo[1] == BCD) { dg += 2.f * byl; }
        if (hyp) { off = fmadd(byh, el4(g.xyp, p), off); dg += byh; }
        else if (L.bc.hi[1] == BCD) { dg += 2.f * byh; }
        if (DIM == 3) {
            const float bzl = el4(g.fzl, p), bzh = el4(g.fzh, p);
            if (hzm) { off = fmadd(bzl, el4(g.xzm, p), off); dg += bzl; }
            else if (L.bc.lo[2] == BCD) { dg += 2.f * bzl; }
            if (hzp) { off = fmadd(bzh, el4(g.xzp, p), off); dg += bzh; }
            else if (L.bc.hi[2] == BCD) { dg += 2.f * bzh; }
        }
        return (off - el4(g.bb, p)) * recip(dg);
    };
    // quads away from every non-periodic boundary: the same operations in the
    // same order, without the per-face presence tests
    const bool inner = hym && hyp && (DIM == 2 || (hzm && hzp)) && (px || (i0 > 0 && i0 + 4 < nx));
    auto update_in = [&](int p, float bxl, float bxh, float xl, float xh) -> float {
        float off = 0.f, dg = 0.f;
        off = fmadd(bxl, xl, off); dg += bxl;
        off = fmadd(bxh, xh, off); dg += bxh;
        const float byl = el4(g.fyl, p), byh = el4(g.fyh, p);
        off = fmadd(byl, el4(g.xym, p), off); dg += byl;
        off = fmadd(byh, el4(g.xyp, p), off); dg += byh;
        if (DIM == 3) {
            const float bzl = el4(g.fzl, p), bzh = el4(g.fzh, p);
            off = fmadd(bzl, el4(g.xzm, p), off); dg += bzl;
            off = fmadd(bzh, el4(g.xzp, p), off); dg += bzh;
        }
        return (off - el4(g.bb, p)) * recip(dg);
    };
    const float4 xc = g.xc;
    float4 out = xc;
    if (inner) {
        if (p0 == 0) {
            out.x = update_in(0, g.fx0, g.fx1, g.xout, xc.y);
            out.z = update_in(2, g.fx2, g.fx3, xc.y, xc.w);
        } else {
            out.y = update_in(1, g.fx0, g.fx1, xc.x, xc.z);
            out.w = update_in(3, g.fx2, g.fx3, xc.z, g.xout);
        }
    } else if (p0 == 0) {
        out.x = update(0, g.fx0, g.fx1, g.xout, xc.y);
        out.z = update(2, g.fx2, g.fx3, xc.y, xc.w);
    } else {
        out.y = update(1, g.fx0, g.fx1, xc.x, xc.z);
        out.w = update(3, g.fx2, g.fx3, xc.z, g.xout);
    }
    return out;
}

__device__ __forceinline__ float* quad_ptr(const CellLevel<float>& L, float* x, int q, int j, int k)
{
    return x + ((size_t)k * L.ny + j) * L.nx + 4 * q;
}

// One colour pass of red-black Gauss-Seidel on quad q of row j, plane k, in
// place (the quad is written back whole).
template <int DIM, bool CG>
__device__ __forceinline__ void gsrb4_quad(const CellLevel<float>& L, float* __restrict__ x,
                                           const float* __restrict__ b, int color, int q, int j, int k, bool ZX)
{
    Gs4 g;
    gs4_load<DIM, CG>(L, x, b, color, q, j, k, ZX, g);
    *reinterpret_cast<float4*>(quad_ptr(L, x, q, j, k)) = gs4_value<DIM>(L, color, q, j, k, g);
}

// Residuals r = b - L x of the four cells of quad q, row j, plane k of a 3-D
// level, in the arithmetic of k_resid_restrict_v4 (face terms in cell_row's
// order; r = b - fma(-diag, x, off)).
template <bool CG>
__device__ __forceinline__ void resid4_quad(const CellLevel<float>& F, const float* __restrict__ x,
                                            const float* __restrict__ b, int q, int j, int k, float (&r)[4])
{
    const int nx = F.nx, ny = F.ny, nz = F.nz;
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
    const float4 xc = xld4<CG>(x + row + i0);
    const float4 bb = ro4<CG>(b + row + i0);
    const float4 xym = hym ? xld4<CG>(x + rym + i0) : zero4;
    const float4 xyp = hyp ? xld4<CG>(x + ryp + i0) : zero4;
    const float4 xzm = hzm ? xld4<CG>(x + rzm + i0) : zero4;
    const float4 xzp = hzp ? xld4<CG>(x + rzp + i0) : zero4;
    const size_t fxb = ((size_t)k * ny + j) * (nx + 1) + i0;
    const float fx[5] = {ro1<CG>(F.bx + fxb), ro1<CG>(F.bx + fxb + 1), ro1<CG>(F.bx + fxb + 2),
                         ro1<CG>(F.bx + fxb + 3), ro1<CG>(F.bx + fxb + 4)};
    const size_t fyb = ((size_t)k * (ny + 1) + j) * nx + i0;
    const float4 fyl = ro4<CG>(F.by + fyb), fyh = ro4<CG>(F.by + fyb + nx);
    const float4 fzl = ro4<CG>(F.bz + row + i0), fzh = ro4<CG>(F.bz + row + plane + i0);
    const float xl = i0 > 0 ? xld1<CG>(x + row + i0 - 1) : (px ? xld1<CG>(x + row + nx - 1) : 0.f);
    const float xr = i0 + 4 < nx ? xld1<CG>(x + row + i0 + 4) : (px ? xld1<CG>(x + row) : 0.f);
    const float xs[6] = {xl, xc.x, xc.y, xc.z, xc.w, xr};
    const bool inner = hym && hyp && hzm && hzp && (px || (i0 > 0 && i0 + 4 < nx));
    if (inner) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float off = 0.f, dg = 0.f;
            off = fmadd(fx[p], xs[p], off); dg += fx[p];
            off = fmadd(fx[p + 1], xs[p + 2], off); dg += fx[p + 1];
            const float byl = el4(fyl, p), byh = el4(fyh, p);
            off = fmadd(byl, el4(xym, p), off); dg += byl;
            off = fmadd(byh, el4(xyp, p), off); dg += byh;
            const float bzl = el4(fzl, p), bzh = el4(fzh, p);
            off = fmadd(bzl, el4(xzm, p), off); dg += bzl;
            off = fmadd(bzh, el4(xzp, p), off); dg += bzh;
            r[p] = el4(bb, p) - fmadd(-dg, xs[p + 1], off);
        }
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = i0 + p;
            float off = 0.f, dg = 0.f;
            const float bxl = fx[p], bxh = fx[p + 1];
            if (i > 0 || px) { off = fmadd(bxl, xs[p], off); dg += bxl; }
            else if (F.bc.lo[0] == BCD) { dg += 2.f * bxl; }
            if (i < nx - 1 || px) { off = fmadd(bxh, xs[p + 2], off); dg += bxh; }
            else if (F.bc.hi[0] == BCD) { dg += 2.f * bxh; }
            const float byl = el4(fyl, p), byh = el4(fyh, p);
            if (hym) { off = fmadd(byl, el4(xym, p), off); dg += byl; }
            else if (F.bc.lo[1] == BCD) { dg += 2.f * byl; }
            if (hyp) { off = fmadd(byh, el4(xyp, p), off); dg += byh; }
            else if (F.bc.hi[1] == BCD) { dg += 2.f * byh; }
            const float bzl = el4(fzl, p), bzh = el4(fzh, p);
            if (hzm) { off = fmadd(bzl, el4(xzm, p), off); dg += bzl; }
            else if (F.bc.lo[2] == BCD) { dg += 2.f * bzl; }
            if (hzp) { off = fmadd(bzh, el4(xzp, p), off); dg += bzh; }
            else if (F.bc.hi[2] == BCD) { dg += 2.f * bzh; }
            r[p] = el4(bb, p) - fmadd(-dg, xs[p + 1], off);
        }
    }
}

// Linear prolongation and correction of quad q, row j, plane k of a 3-D level:
// x_f += P x_c, the arithmetic of prolong_value (weights, fused multiply-adds
// and their order) with each coarse row's x-interpolation formed once for the
// four cells.  The coarse x is not written during the launches that call this.
template <bool CG>
__device__ __forceinline__ void prolong4_quad(const CellLevel<float>& F, const CellLevel<float>& C,
                                              float* __restrict__ xf, const float* __restrict__ xc, int q, int j,
                                              int k)
{
    const int i0 = 4 * q, c0 = 2 * q;
    const Lin1D l0 = lin1d(i0, C.nx, F.bc.lo[0], F.bc.hi[0]);       // p = c0, q: left neighbour
    const Lin1D l3 = lin1d(i0 + 3, C.nx, F.bc.lo[0], F.bc.hi[0]);   // p = c0 + 1, q: right neighbour
    const Lin1D ly = lin1d(j, C.ny, F.bc.lo[1], F.bc.hi[1]);
    const Lin1D lz = lin1d(k, C.nz, F.bc.lo[2], F.bc.hi[2]);
    const float w1 = 0.75f, w2 = 0.25f;
    const float a0 = w2 * l0.sq, a3 = w2 * l3.sq, ay = w2 * ly.sq, az = w2 * lz.sq;
    // prolong_value's lo / hi of one coarse row for the four cells
    auto xint = [&](int cb, int cc, float (&o)[4]) {
        const float* r = xc + ((size_t)cc * C.ny + cb) * C.nx;
        const float2 m = *reinterpret_cast<const float2*>(r + c0);
        const float vl = r[l0.q], vr = r[l3.q];
        o[0] = fmadd(a0, vl, w1 * m.x);   // cell i0:     P = c0,     Q = l0.q
        o[1] = fmadd(w2, m.y, w1 * m.x);  // cell i0 + 1: P = c0,     Q = c0 + 1
        o[2] = fmadd(w2, m.x, w1 * m.y);  // cell i0 + 2: P = c0 + 1, Q = c0
        o[3] = fmadd(a3, vr, w1 * m.y);   // cell i0 + 3: P = c0 + 1, Q = l3.q
    };
    float pl[2][4];   // prolong_value's plane(lz.p), plane(lz.q)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int cc = e ? lz.q : lz.p;
        float lo[4], hi[4];
        xint(ly.p, cc, lo);
        xint(ly.q, cc, hi);
#pragma unroll
        for (int p = 0; p < 4; ++p) pl[e][p] = fmadd(ay, hi[p], w1 * lo[p]);
    }
    float* px = xf + ((size_t)k * F.ny + j) * F.nx + i0;
    float4 v = xld4<CG>(px);
    v.x += fmadd(az, pl[1][0], w1 * pl[0][0]);
    v.y += fmadd(az, pl[1][1], w1 * pl[0][1]);
    v.z += fmadd(az, pl[1][2], w1 * pl[0][2]);
    v.w += fmadd(az, pl[1][3], w1 * pl[0][3]);
    *reinterpret_cast<float4*>(px) = v;
}

}  // namespace mgp
