// mg_cellpipe.cu -- one leg of a cell V-cycle on the finest FP32 level as ONE
// launch, its colour passes pipelined through L2.
//
// The down leg of a V(nu1, nu2) cycle on the finest level is nu1 red-black
// sweeps (2 nu1 colour passes) and the residual restricted to the next level;
// the up leg is the prolongation of the coarse correction and nu2 sweeps.
// Launched pass by pass, every pass streams x, b and the three face arrays
// through HBM again (about 24 bytes per cell and pass at 256^3), although a
// pass only needs what the previous pass wrote one plane away.  Here the
// passes of a leg run concurrently in one persistent launch, each lagging the
// one before it by a few planes, so that the planes a pass reads were written
// by its predecessor moments earlier and are still in L2.
//
// Work items.  The level is cut into steps of Z planes and bands of kPipeBand
// rows.  Item (t, p, j) applies pass p to rows [8j, 8j + 8) of the planes
// [tZ - lag_p, tZ + Z - lag_p) (clipped to the level), where lag_0 = 0 and
// lag_p = lag_{p-1} + Z + 1.  Pass p reads what pass p - 1 wrote on its own
// planes and one plane either side, and (red-black passes) overwrites cells
// whose old values pass p - 1 read on those planes; with this lag both sets of
// planes belong to items (t - 1 .. t - dep_p, p - 1, j - 1 .. j + 1), and to no
// item of the same step, so the passes of one step are independent of each
// other.  Items are handed out in the order (t, p, j) by an atomic ticket: an
// item waits only for items with lower tickets, which CTAs that are already
// running hold, so the wait always ends (whatever the grid size); each wait is
// still bounded by a clock limit, after which the item is skipped, an error
// word is set and every later wait gives up at once.  A finished item
// publishes its flag (release, after a fence); a waiter reads flags with
// acquire loads and the CTA then reads x only through ld.global.cg (L2, the
// point of coherence), never through an L1 line that another SM's write could
// have made stale.  Flags hold a per-launch epoch read from device memory at
// the start of the launch and advanced by the last CTA to leave, so neither
// the flags nor the counters need clearing between launches, and the launch
// can be replayed from a CUDA graph.
//
// Arithmetic.  Each item calls the per-quad functions of k_gsrb_v4,
// k_resid_restrict_v4 and k_prolong_add_v4 (mg_cellquad.cuh), and every value
// it reads is the value the pass-by-pass launches would have read, so the
// results are identical bit for bit.  A down leg started from x = 0 takes the
// first red pass with x known to be zero (no zero fill, no x loads).
//
// Requirements (cell_pipe_ok): 3-D FP32 level, nx % 4 == 0, ny and nz even,
// z not periodic (the lagged planes must not wrap), 16-byte aligned x, b and
// face arrays, 8-byte aligned coarse b.
#include <algorithm>
#include <atomic>

#include "mg_cellquad.cuh"

namespace mgp {

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr long long kPipeWaitCycles = 2000000000LL;   // about one second at 2 GHz
constexpr int kPipeRQ = 128;                           // quads per restriction chunk

static_assert(kPipeBand == 8, "the item loops below take a band of 8 rows");

__global__ void __launch_bounds__(256, 3)
k_cell_pipe(CellLevel<float> F, float* __restrict__ x, const float* __restrict__ b, CellLevel<float> C,
            float* __restrict__ bc, const float* __restrict__ xc, CellPipe P, PipeSync S)
{
    __shared__ unsigned s_next[2], s_ep;
    __shared__ int s_go;
    __shared__ float2 s_part[2][kPipeBand][kPipeRQ];
    const int nband = P.nband, npass = P.npass;
    const unsigned per_slot = (unsigned)nband * (unsigned)npass;
    const unsigned nitems = per_slot * (unsigned)P.nslot;
    const int nx = F.nx, ny = F.ny, nz = F.nz, nq = nx >> 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        s_ep = *(volatile unsigned*)(S.ctr + 2) + 1u;
        s_next[0] = atomicAdd(S.ctr, 1u);
    }
    __syncthreads();
    const unsigned ep = s_ep;
    unsigned tk = s_next[0];
    for (int it = 1; tk < nitems; ++it) {
        const int jb = (int)(tk % (unsigned)nband);
        const int ph = (int)((tk / (unsigned)nband) % (unsigned)npass);
        const int t = (int)(tk / per_slot) - P.K * ph;   // slot t + K ph holds step t of pass ph
        const bool live = t >= 0 && t < P.nstep;          // else: outside the pass's steps, no item
        if (threadIdx.x == 0) {
            // the next ticket is drawn now, so that its round trip overlaps this item
            s_next[it & 1] = atomicAdd(S.ctr, 1u);
            int go = 1;
            if (live && ph > 0) {
                const long long t0 = clock64();
                for (int dt = 1; dt <= P.dep[ph] && go; ++dt) {
                    const int ts = t - dt;
                    if (ts < 0) break;
                    for (int dj = -1; dj <= 1 && go; ++dj) {
                        int jj = jb + dj;
                        if (jj < 0 || jj >= nband) {
                            if (!P.yper) continue;
                            jj = jj < 0 ? jj + nband : jj - nband;
                        }
                        const unsigned* f = S.flags + ((size_t)ts * npass + (ph - 1)) * nband + jj;
                        while (ld_acquire_u32(f) != ep) {
                            if (*(volatile int*)S.err != 0 || clock64() - t0 > kPipeWaitCycles) {
                                go = 0;
                                break;
                            }
                            __nanosleep(32);
                        }
                    }
                }
                if (!go) atomicCAS(S.err, 0, 2);
            }
            s_go = go;
        }
        __syncthreads();
        if (live && s_go) {
            const int op = P.op[ph];
            const int w0 = t * P.Z - P.lag[ph];
            const int k0 = w0 > 0 ? w0 : 0, k1 = w0 + P.Z < nz ? w0 + P.Z : nz;
            const int j0 = jb * kPipeBand, j1 = j0 + kPipeBand < ny ? j0 + kPipeBand : ny;
            if (k0 < k1) {
                if (op == PIPE_RESTRICT) {
                    // one coarse plane (two fine planes) and up to kPipeRQ quads
                    // along x at a time: each thread forms the x-pair sums of one
                    // quad's residuals, the CTA adds rows and planes in shared
                    // memory in k_resid_restrict_v4's order (x pairs, then rows,
                    // then planes); warps take (plane, row) pairs, lanes quads
                    const int cnx = nx >> 1, cny = ny >> 1, rows = j1 - j0;
                    for (int kc = k0 >> 1; kc < (k1 >> 1); ++kc)
                        for (int qb = 0; qb < nq; qb += kPipeRQ) {
                            const int nqq = nq - qb < kPipeRQ ? nq - qb : kPipeRQ;
                            for (int rp = warp; rp < 2 * kPipeBand; rp += nwarp) {
                                const int pz = rp >> 3, jr = rp & 7;
                                if (jr >= rows) continue;
                                for (int qq = lane; qq < nqq; qq += 32) {
                                    float r[4];
                                    resid4_quad<true>(F, x, b, qb + qq, j0 + jr, 2 * kc + pz, r);
                                    s_part[pz][jr][qq] = make_float2(r[0] + r[1], r[2] + r[3]);
                                }
                            }
                            __syncthreads();
                            for (int jr = 2 * warp; jr < rows; jr += 2 * nwarp)
                                for (int qq = lane; qq < nqq; qq += 32) {
                                    const float2 a0 = s_part[0][jr][qq], a1 = s_part[0][jr + 1][qq];
                                    const float2 c0 = s_part[1][jr][qq], c1 = s_part[1][jr + 1][qq];
                                    float2 v;
                                    v.x = ((a0.x + a1.x) + (c0.x + c1.x)) * 0.125f;
                                    v.y = ((a0.y + a1.y) + (c0.y + c1.y)) * 0.125f;
                                    *reinterpret_cast<float2*>(bc + ((size_t)kc * cny + ((j0 + jr) >> 1)) * cnx +
                                                               2 * (qb + qq)) = v;
                                }
                            __syncthreads();
                        }
                } else {
                    // warps take (plane, row) pairs of the window, lanes consecutive quads
                    const bool zx = ph == 0 && P.zero_first;
                    for (int rp = warp; rp < (k1 - k0) * kPipeBand; rp += nwarp) {
                        const int kk = k0 + (rp >> 3), j = j0 + (rp & 7);
                        if (j >= j1) continue;
                        if (op == PIPE_PROLONG) {
                            for (int q = lane; q < nq; q += 32) prolong4_quad<true>(F, C, x, xc, q, j, kk);
                            continue;
                        }
                        for (int q = lane; q < nq; q += 32) gsrb4_quad<3, true>(F, x, b, op, q, j, kk, zx);
                    }
                }
            }
        }
        __syncthreads();   // the item's stores are issued; s_next[it & 1] is visible
        if (live && threadIdx.x == 0) st_release_u32(S.flags + ((size_t)t * npass + ph) * nband + jb, ep);
        tk = s_next[it & 1];
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned e = atomicAdd(S.ctr + 1, 1u);
        if (e == gridDim.x - 1) {   // the last CTA: every ticket of this launch is drawn
            S.ctr[0] = 0u;
            S.ctr[1] = 0u;
            __threadfence();
            atomicExch(S.ctr + 2, ep);
        }
    }
}

// resident CTAs of k_cell_pipe on the whole GPU (looked up once, outside any
// stream capture: mg_setup calls cell_pipe_grid)
std::atomic<int> g_pipe_grid{0};
int pipe_grid()
{
    int g = g_pipe_grid.load(std::memory_order_acquire);
    if (g == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cell_pipe, 256, 0) != cudaSuccess || per < 1)
            per = 1;
        g = (sms > 0 ? sms : kNumSMs) * per;
        g_pipe_grid.store(g, std::memory_order_release);
    }
    return g;
}

CellPipe make_pipe(const CellLevel<float>& F, const int* ops, int n, bool zero_first)
{
    CellPipe P{};
    P.npass = n;
    P.Z = kPipeZ;
    P.zero_first = zero_first ? 1 : 0;
    P.yper = F.bc.lo[1] == BCP ? 1 : 0;
    P.nband = (F.ny + kPipeBand - 1) / kPipeBand;
    for (int p = 0; p < n; ++p) {
        P.op[p] = ops[p];
        P.lag[p] = p == 0 ? 0 : P.lag[p - 1] + P.Z + 1;
        // steps of pass p - 1 whose planes pass p reads: a gap of g planes
        // reaches 1 + g / Z steps back
        P.dep[p] = p == 0 ? 0 : 1 + (P.lag[p] - P.lag[p - 1]) / P.Z;
    }
    P.nstep = (F.nz + P.lag[n - 1] + P.Z - 1) / P.Z;
    P.K = kPipeK;
    P.nslot = P.nstep + P.K * (n - 1);
    return P;
}

void launch(const CellLevel<float>& F, float* x, const float* b, const CellLevel<float>& C, float* bc, const float* xc,
            const CellPipe& P, const PipeSync& S, cudaStream_t s)
{
    const long long items = (long long)P.nstep * P.npass * P.nband;
    const int grid = (int)std::min<long long>(pipe_grid(), items);
    MGP_LAUNCH(k_cell_pipe<<<grid, 256, 0, s>>>(F, x, b, C, bc, xc, P, S));
}

}  // namespace

int cell_pipe_grid() { return pipe_grid(); }

size_t cell_pipe_flag_words(int ny, int nz, int nu_max)
{
    const int n = 2 * nu_max + 1;
    const int lag = (n - 1) * (kPipeZ + 1);
    const size_t nstep = (size_t)(nz + lag + kPipeZ - 1) / kPipeZ;
    return nstep * n * ((ny + kPipeBand - 1) / kPipeBand);
}

bool cell_pipe_ok(const CellLevel<float>& F, const float* x, const float* b)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return F.nx % 4 == 0 && F.nx >= 8 && F.ny % 2 == 0 && F.ny >= 2 && F.nz % 2 == 0 && F.nz >= 2 &&
           F.bc.lo[2] != BCP && F.invd == nullptr && a16(x) && a16(b) && a16(F.by) && a16(F.bz);
}

void cell_pipe_down(const CellLevel<float>& F, float* x, const float* b, float* bc, int nu1, bool zero_first,
                    const PipeSync& S, cudaStream_t s)
{
    int ops[kPipeMaxPass];
    int n = 0;
    for (int k = 0; k < nu1; ++k) {
        ops[n++] = PIPE_RED;
        ops[n++] = PIPE_BLACK;
    }
    ops[n++] = PIPE_RESTRICT;
    const CellPipe P = make_pipe(F, ops, n, zero_first);
    launch(F, x, b, F, bc, nullptr, P, S, s);
}

void cell_pipe_up(const CellLevel<float>& F, const CellLevel<float>& C, float* x, const float* b, const float* xc,
                  int nu2, const PipeSync& S, cudaStream_t s)
{
    int ops[kPipeMaxPass];
    int n = 0;
    ops[n++] = PIPE_PROLONG;
    for (int k = 0; k < nu2; ++k) {
        ops[n++] = PIPE_RED;
        ops[n++] = PIPE_BLACK;
    }
    const CellPipe P = make_pipe(F, ops, n, false);
    launch(F, x, b, C, nullptr, xc, P, S, s);
}

}  // namespace mgp
