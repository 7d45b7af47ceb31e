// mg_gsrb_tma.cu -- one red-black Gauss-Seidel sweep in one pass over memory
// (FP32 cell levels), with the operands staged by the Tensor Memory
// Accelerator.
//
// A CTA owns R whole x-rows (y0 .. y0+R-1) of a column and marches up a range
// of z-planes, reading xin and writing xout (ping-pong: every old value stays
// readable).  Plane m's operands -- x rows y0-2 .. y0+R+1, b, the x- and
// z-face rows of cell rows y0-1 .. y0+R and the y-face rows y0-1 .. y0+R+1 --
// arrive as one *stage* of row copies (cp.async.bulk completing on one
// mbarrier per stage) in a ring of NS stages, issued NS-3 planes ahead of
// their first use.  Step k of the march
//   1. updates the red cells of plane k+1 from old values only (stages k, k+1,
//      k+2), for the CTA's rows and for the rows y0-1 and y0+R just outside
//      them, and publishes them in a ring of the red values of 3 planes;
//   2. (one barrier) refills the slot of plane k-1 with plane k+NS-1;
//   3. updates the black cells of plane k from the new reds (the ring for
//      plane k, registers for planes k-1 and k+1 of a thread's own quad) and
//      the coefficients of stage k, and writes the quad of plane k (red and
//      black) once.
// Four consecutive cells per thread; the row arithmetic is cell_row's (same
// order of the face terms, same boundary cases, the same fused multiply-adds),
// so the result equals two plain colour passes bit for bit, while x, b and the
// three face arrays cross HBM once per sweep instead of once per colour pass.
//
// Every wait on a stage is bounded: a copy that has not landed after about two
// seconds makes the CTA set the caller's error word (read back with the solve's
// scalars), wait, again bounded, for the copies it issued, and return.
//
// Requirements (checked by cell_gsrb_tma_ok): 3-D, nx % 4 == 0, 32 <= nx <=
// 256, R | ny, nz >= 2, z not periodic, 16-byte aligned vectors and face
// arrays, and the x-face array readable up to 3 floats past its end.
#include <atomic>

#include "mg_cellops.cuh"

namespace mgp {

namespace {

constexpr int kTR = 4;                             // rows per CTA
constexpr int kTMaxStages = 5;
constexpr long long kWaitCycles = 4000000000LL;    // about two seconds at 2 GHz

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ float tel(const float4& v, int p) { return p == 0 ? v.x : p == 1 ? v.y : p == 2 ? v.z : v.w; }
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// one cell update in cell_row's order: neighbour values nb[6] (x-lo, x-hi,
// y-lo, y-hi, z-lo, z-hi), presence, face values f[6], b
__device__ __forceinline__ float row_update(const CellLevel<float>& L, const bool (&has)[6], const float (&nb)[6],
                                            const float (&f)[6], float bv)
{
    float off = 0.f, dg = 0.f;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int d = e >> 1;
        const int bc = (e & 1) ? L.bc.hi[d] : L.bc.lo[d];
        if (has[e]) { off = fmadd(f[e], nb[e], off); dg += f[e]; }
        else if (bc == BCD) { dg += 2.f * f[e]; }
    }
    return (off - bv) * recip(dg);
}

// Stage layout (floats): X rows y0-2 .. y0+R+1; B rows y0-1 .. y0+R; BX rows
// y0-1 .. y0+R at stride W + 8, each starting at its own 16-byte misalignment
// a; BY face rows y0-1 .. y0+R+1; BZ rows y0-1 .. y0+R of the z-faces below
// the plane's cells.  Every row starts on a 16-byte boundary (W % 4 == 0).
struct Stage {
    int W;
    __device__ __forceinline__ int x(int r) const { return r * W; }
    __device__ __forceinline__ int b(int r) const { return (kTR + 4 + r) * W; }
    __device__ __forceinline__ int bx(int r) const { return (2 * kTR + 6) * W + r * (W + 8); }
    __device__ __forceinline__ int by(int r) const { return (2 * kTR + 6) * W + (kTR + 2) * (W + 8) + r * W; }
    __device__ __forceinline__ int bz(int r) const { return (3 * kTR + 9) * W + (kTR + 2) * (W + 8) + r * W; }
};
constexpr int kCopies = 5 * kTR + 13;   // row copies per stage

__host__ __device__ inline int stage_floats(int W) { return (4 * kTR + 11) * W + (kTR + 2) * (W + 8); }
__host__ __device__ inline int red_floats(int W) { return 3 * (kTR + 2) * (W / 4) * 2; }

}  // namespace

__global__ void __launch_bounds__(256)
k_gsrb_tma(CellLevel<float> L, const float* __restrict__ xin, float* __restrict__ xout, const float* __restrict__ b,
           int ns, int* __restrict__ err)
{
    extern __shared__ __align__(128) float sm[];
    const int W = L.nx, ny = L.ny, nz = L.nz, nq = W / 4;
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * nq + lane;
    const int sf = stage_floats(W);
    float* red = sm + (size_t)ns * sf;   // [plane % 3][ring row 0 .. R+1][quad][2]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(red + red_floats(W));
    const Stage S{W};
    const bool px = L.bc.lo[0] == BCP, py = L.bc.lo[1] == BCP;
    const size_t plane = (size_t)W * ny;

    if (tid == 0)
        for (int s = 0; s < ns; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();

    // wrapped row index (-1: absent)
    auto rowy = [&](int v) { return v >= 0 && v < ny ? v : (py ? (v < 0 ? v + ny : v - ny) : -1); };

    // stage of plane m into slot s, by the threads of warp 0 (tid < 32): the
    // row copies are spread over its lanes; lane 0 arms the barrier with the
    // byte total before any copy is issued
    auto issue = [&](int m, int y0, int s) {
        float* st = sm + (size_t)s * sf;
        const bool pin = m >= 0 && m < nz, fin = m >= 0 && m <= nz;
        unsigned bytes = 0;
        const float* src[2] = {nullptr, nullptr};
        float* dst[2] = {nullptr, nullptr};
        unsigned nb[2] = {0u, 0u};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = tid + 32 * e;
            if (c >= kCopies) continue;
            if (c < kTR + 4) {                                   // x rows
                const int jr = rowy(y0 - 2 + c);
                if (pin && jr >= 0) { src[e] = xin + m * plane + (size_t)jr * W; dst[e] = st + S.x(c); nb[e] = 4 * W; }
            } else if (c < 2 * kTR + 6) {                        // b rows
                const int r = c - (kTR + 4), jr = rowy(y0 - 1 + r);
                if (pin && jr >= 0) { src[e] = b + m * plane + (size_t)jr * W; dst[e] = st + S.b(r); nb[e] = 4 * W; }
            } else if (c < 3 * kTR + 8) {                        // x-face rows, rounded out to 16 bytes
                const int r = c - (2 * kTR + 6), jr = rowy(y0 - 1 + r);
                if (pin && jr >= 0) {
                    const size_t gx = ((size_t)m * ny + jr) * (W + 1);
                    const int a = jr & 3;   // gx mod 4: W and ny are multiples of 4
                    src[e] = L.bx + (gx - a);
                    dst[e] = st + S.bx(r);
                    nb[e] = 4 * ((W + 1 + a + 3) & ~3);
                }
            } else if (c < 4 * kTR + 11) {                       // y-face rows y0-1 .. y0+R+1
                const int r = c - (3 * kTR + 8), v = y0 - 1 + r;
                int fr = v >= 0 && v <= ny ? v : -1;
                if (py && v < 0) fr = ny - 1;                   // low face of cell row ny-1
                if (py && v > ny) fr = 1;                       // high face of cell row 0
                if (pin && fr >= 0) {
                    src[e] = L.by + ((size_t)m * (ny + 1) + fr) * W;
                    dst[e] = st + S.by(r);
                    nb[e] = 4 * W;
                }
            } else {                                            // z-face rows of face plane m
                const int r = c - (4 * kTR + 11), jr = rowy(y0 - 1 + r);
                if (fin && jr >= 0) { src[e] = L.bz + m * plane + (size_t)jr * W; dst[e] = st + S.bz(r); nb[e] = 4 * W; }
            }
            bytes += nb[e];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
        if (tid == 0) mbar_arrive_expect(&bars[s], bytes);
        // the slot was last read through the generic proxy: order those reads
        // (completed before the barrier that freed it) before the bulk writes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (nb[e]) bulk_copy(dst[e], src[e], nb[e], &bars[s]);
    };

    // the two red values of quad q in tile row t (-1 .. R) of plane m
    // (positions p0 and p0 + 2, p0 = (jr + m) & 1), from stages s0 (m-1), s1 (m), s2 (m+1)
    auto red_quad = [&](const float* s0, const float* s1, const float* s2, int jr, int t, int m, int q, float& r0,
                        float& r1) {
        const int i0 = 4 * q;
        const bool hym = jr > 0 || py, hyp = jr < ny - 1 || py, hzm = m > 0, hzp = m < nz - 1;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float* xr = s1 + S.x(t + 2);
        const float4 xc = lds4(xr + i0);
        const float4 xym = hym ? lds4(s1 + S.x(t + 1) + i0) : z4, xyp = hyp ? lds4(s1 + S.x(t + 3) + i0) : z4;
        const float4 xzm = hzm ? lds4(s0 + S.x(t + 2) + i0) : z4, xzp = hzp ? lds4(s2 + S.x(t + 2) + i0) : z4;
        const float4 bb = lds4(s1 + S.b(t + 1) + i0);
        const int p0 = (jr + m) & 1;
        float xo = 0.f;   // the x-neighbour outside the quad: left of cell 0 (p0 == 0) or right of cell 3
        if (p0 == 0) {
            if (i0 > 0) xo = xr[i0 - 1];
            else if (px) xo = xr[W - 1];
        } else {
            if (i0 + 4 < W) xo = xr[i0 + 4];
            else if (px) xo = xr[0];
        }
        const float* fxr = s1 + S.bx(t + 1) + (jr & 3) + i0 + p0;
        const float fx0 = fxr[0], fx1 = fxr[1], fx2 = fxr[2], fx3 = fxr[3];
        const float4 fyl = lds4(s1 + S.by(t + 1) + i0), fyh = lds4(s1 + S.by(t + 2) + i0);
        const float4 fzl = lds4(s1 + S.bz(t + 1) + i0), fzh = lds4(s2 + S.bz(t + 1) + i0);
        auto upd = [&](int p, float bxl, float bxh, float xl, float xh) {
            const int i = i0 + p;
            const bool has[6] = {i > 0 || px, i < W - 1 || px, hym, hyp, hzm, hzp};
            const float nbv[6] = {xl, xh, tel(xym, p), tel(xyp, p), tel(xzm, p), tel(xzp, p)};
            const float f[6] = {bxl, bxh, tel(fyl, p), tel(fyh, p), tel(fzl, p), tel(fzh, p)};
            return row_update(L, has, nbv, f, tel(bb, p));
        };
        if (p0 == 0) {
            r0 = upd(0, fx0, fx1, xo, xc.y);
            r1 = upd(2, fx2, fx3, xc.y, xc.w);
        } else {
            r0 = upd(1, fx0, fx1, xc.x, xc.z);
            r1 = upd(3, fx2, fx3, xc.z, xo);
        }
    };
    auto ring = [&](int m, int rr) { return red + ((size_t)(m % 3) * (kTR + 2) + rr) * nq * 2; };

    // reds of plane m for the tile (own quad) and the two ring rows (the first
    // 2 nq threads: row y0-1 for tid < nq, row y0+R for nq <= tid < 2 nq)
    auto reds_of_plane = [&](const float* s0, const float* s1, const float* s2, int y0, int m, float& r0,
                             float& r1) {
        red_quad(s0, s1, s2, y0 + w, w, m, lane, r0, r1);
        float* o = ring(m, w + 1) + 2 * lane;
        o[0] = r0;
        o[1] = r1;
        if (tid < 2 * nq) {
            const int t = tid < nq ? -1 : kTR, q = tid < nq ? tid : tid - nq;
            const int jr = rowy(y0 + t);
            if (jr >= 0) {
                float q0, q1;
                red_quad(s0, s1, s2, jr, t, m, q, q0, q1);
                float* oq = ring(m, t + 1) + 2 * q;
                oq[0] = q0;
                oq[1] = q1;
            }
        }
    };

    const int cols = ny / kTR;
    const long long U = (long long)cols * nz;
    const long long u_begin = U * blockIdx.x / gridDim.x, u_end = U * (blockIdx.x + 1) / gridDim.x;
    // stages are issued in plane order into slots 0, 1, .., ns-1, 0, ..; the
    // n-th use of a slot completes its barrier's phase n, so a consumer waits
    // with the parity of the number of earlier waits on that slot (bit s of wpar)
    auto inc = [&](int sl) { return sl + 1 == ns ? 0 : sl + 1; };
    int s_issue = 0;          // slot of the next stage to issue
    unsigned wpar = 0;        // per-slot parity of the next wait
    int pending = 0;          // stages issued and not yet waited for
    bool failed = false;

    for (long long u = u_begin; u < u_end && !failed;) {
        const int col = (int)(u / nz), z0 = (int)(u % nz);
        const int z1 = (int)min((long long)nz, (long long)z0 + (u_end - u));
        u += z1 - z0;
        const int y0 = col * kTR, j = y0 + w;
        const int mlo = z0 - 2, mhi = z1 + 1;   // planes staged for this segment
        const int s_lo = s_issue;                // slot of plane mlo
        auto wait = [&](int sl) {
            const bool ok = mbar_wait(&bars[sl], (wpar >> sl) & 1u);
            if (ok) { wpar ^= 1u << sl; --pending; }
            return ok;
        };
        int next = mlo;   // next plane to issue
        for (; next <= mhi && next < mlo + ns; ++next) {
            if (tid < 32) issue(next, y0, s_issue);
            s_issue = inc(s_issue);
            ++pending;
        }
        // slots of planes k-1 .. k+2 during step k, advanced incrementally
        int sm1 = s_lo, s0 = inc(sm1), s1 = inc(s0), s2 = inc(s1);   // planes z0-2 .. z0+1
        bool ok = wait(sm1) && wait(s0) && wait(s1) && wait(s2);
        float rp0 = 0.f, rp1 = 0.f, rc0 = 0.f, rc1 = 0.f, rn0 = 0.f, rn1 = 0.f;
        if (ok) {
            if (z0 > 0)
                red_quad(sm + (size_t)sm1 * sf, sm + (size_t)s0 * sf, sm + (size_t)s1 * sf, j, w, z0 - 1, lane, rp0,
                         rp1);
            reds_of_plane(sm + (size_t)s0 * sf, sm + (size_t)s1 * sf, sm + (size_t)s2 * sf, y0, z0, rc0, rc1);
        }
        if (__syncthreads_or(!ok)) { failed = true; break; }
        // the slot of plane z0-2 is free
        if (next <= mhi) {
            if (tid < 32) issue(next, y0, s_issue);
            s_issue = inc(s_issue);
            ++pending;
            ++next;
        }
        // step k: stage slots of planes k (p0), k+1 (p1), k+2 (p2)
        int p0 = s1, p1 = s2, p2 = inc(s2);
        for (int k = z0; k < z1; ++k) {
            ok = wait(p2);
            if (ok && k + 1 < nz)
                reds_of_plane(sm + (size_t)p0 * sf, sm + (size_t)p1 * sf, sm + (size_t)p2 * sf, y0, k + 1, rn0, rn1);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            // the slot of plane k-1 is free
            if (next <= mhi) {
                if (tid < 32) issue(next, y0, s_issue);
                s_issue = inc(s_issue);
                ++pending;
                ++next;
            }
            // black cells of plane k: positions p1b and p1b + 2
            const float* st1 = sm + (size_t)p0 * sf;
            const float* st2 = sm + (size_t)p1 * sf;
            const int i0 = 4 * lane;
            const int p1b = ((j + k) & 1) ^ 1;
            const bool hym = j > 0 || py, hyp = j < ny - 1 || py, hzm = k > 0, hzp = k < nz - 1;
            const float* rk = ring(k, w + 1);
            const int ql = lane > 0 ? lane - 1 : nq - 1, qr = lane < nq - 1 ? lane + 1 : 0;
            const float xl = rk[2 * ql + 1];   // the left quad's red at position 3
            const float xh = rk[2 * qr];       // the right quad's red at position 0
            float ym0 = 0.f, ym1 = 0.f, yp0 = 0.f, yp1 = 0.f;
            if (hym) { const float* q = ring(k, w) + 2 * lane; ym0 = q[0]; ym1 = q[1]; }
            if (hyp) { const float* q = ring(k, w + 2) + 2 * lane; yp0 = q[0]; yp1 = q[1]; }
            const float4 bb = lds4(st1 + S.b(w + 1) + i0);
            const float* fxr = st1 + S.bx(w + 1) + (j & 3) + i0 + p1b;
            const float fx0 = fxr[0], fx1 = fxr[1], fx2 = fxr[2], fx3 = fxr[3];
            const float4 fyl = lds4(st1 + S.by(w + 1) + i0), fyh = lds4(st1 + S.by(w + 2) + i0);
            const float4 fzl = lds4(st1 + S.bz(w + 1) + i0), fzh = lds4(st2 + S.bz(w + 1) + i0);
            auto upd = [&](int p, int e, float bxl, float bxh, float xlo, float xhi) {
                const int i = i0 + p;
                const bool has[6] = {i > 0 || px, i < W - 1 || px, hym, hyp, hzm, hzp};
                const float nbv[6] = {xlo, xhi, e ? ym1 : ym0, e ? yp1 : yp0, e ? rp1 : rp0, e ? rn1 : rn0};
                const float f[6] = {bxl, bxh, tel(fyl, p), tel(fyh, p), tel(fzl, p), tel(fzh, p)};
                return row_update(L, has, nbv, f, tel(bb, p));
            };
            float4 out;
            if (p1b == 0) {   // black at 0, 2; red at 1, 3
                out.x = upd(0, 0, fx0, fx1, xl, rc0);
                out.y = rc0;
                out.z = upd(2, 1, fx2, fx3, rc0, rc1);
                out.w = rc1;
            } else {          // black at 1, 3; red at 0, 2
                out.x = rc0;
                out.y = upd(1, 0, fx0, fx1, rc0, rc1);
                out.z = rc1;
                out.w = upd(3, 1, fx2, fx3, rc1, xh);
            }
            *reinterpret_cast<float4*>(xout + k * plane + (size_t)j * W + i0) = out;
            rp0 = rc0; rp1 = rc1;
            rc0 = rn0; rc1 = rn1;
            p0 = p1; p1 = p2; p2 = inc(p2);
        }
        if (failed) break;
        __syncthreads();   // every stage of the segment consumed; slots and the red ring are free
    }
    if (failed) {
        // let the copies already issued land (bounded) before the shared memory is released:
        // the unwaited stages occupy the `pending` slots before s_issue
        int sl = s_issue;
        for (int n = 0; n < pending; ++n) sl = sl == 0 ? ns - 1 : sl - 1;
        for (int n = 0; n < pending; ++n, sl = inc(sl)) (void)mbar_wait(&bars[sl], (wpar >> sl) & 1u);
        if (tid == 0) atomicOr(err, 1);
    }
}

bool cell_gsrb_tma_ok(int dim, const CellLevel<float>& L, const float* xin, const float* xout, const float* b)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return dim == 3 && L.nx % 4 == 0 && L.nx >= 32 && L.nx <= 256 && L.ny % kTR == 0 && L.nz >= 2 &&
           L.bc.lo[2] != BCP && L.invd == nullptr && a16(xin) && a16(xout) && a16(b) && a16(L.bx) && a16(L.by) &&
           a16(L.bz);
}

static size_t tma_smem(int W, int ns)
{
    return ((size_t)ns * stage_floats(W) + red_floats(W)) * sizeof(float) + (size_t)ns * 8;
}

// device limits, and the kernel's dynamic shared-memory allowance (set once,
// outside any stream capture: mg_setup calls cell_gsrb_tma_fits)
static std::atomic<int> g_tma_smem{0}, g_tma_sms{0};
static void tma_init()
{
    if (g_tma_smem.load(std::memory_order_acquire)) return;
    int dev = 0, v = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(k_gsrb_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, v) != cudaSuccess) v = 48 * 1024;
    g_tma_sms.store(n > 0 ? n : kNumSMs, std::memory_order_relaxed);
    g_tma_smem.store(v > 0 ? v : 1, std::memory_order_release);
}

bool cell_gsrb_tma_fits(int nx)
{
    tma_init();
    return tma_smem(nx, 4) <= (size_t)g_tma_smem.load(std::memory_order_acquire);
}

void cell_gsrb_tma(const CellLevel<float>& L, const float* xin, float* xout, const float* b, int* err, cudaStream_t s)
{
    tma_init();
    const int W = L.nx, nq = W / 4;
    // as many stages as the shared memory of one CTA holds (at most 5, at least 4)
    int ns = kTMaxStages;
    while (ns > 4 && tma_smem(W, ns) > (size_t)g_tma_smem.load(std::memory_order_acquire)) --ns;
    const size_t smem = tma_smem(W, ns);
    const long long units = (long long)(L.ny / kTR) * L.nz;
    // one CTA per SM (the stages fill its shared memory); a CTA takes a
    // contiguous run of (column, plane) units, at least 8 planes long on average
    long long grid = g_tma_sms.load(std::memory_order_relaxed);
    if (grid > units / 8) grid = units / 8 > 0 ? units / 8 : 1;
    MGP_LAUNCH(k_gsrb_tma<<<(unsigned)grid, dim3(nq, kTR), smem, s>>>(L, xin, xout, b, ns, err));
}

}  // namespace mgp
