// mg_batch.cu -- the FP32 level passes of many solves, one launch per step for all of them.
//
// A batch of independent cell solves of uneven sizes runs its V-cycles in
// lockstep: one launch per step (a colour pass, the residual + restriction or
// the prolongation of "level l" of every solve that has such a level) instead
// of one launch per step and solve.  The launch takes, as its parameter, a
// table of work items -- one per solve with work in the step, each covering
// its level's work units in warp tiles of 32 units -- so the table sits in the
// constant bank: a warp finds the item of its tile by a binary search over the
// items' first tiles (uniform across the warp, so each probe is one
// constant-cache broadcast) and reads the item's fields the same way.  The
// only global loads before the units' own are the solve's run flag.  Each warp
// takes one tile, with no barrier and no shared memory, so as many tiles are
// in flight as the SMs hold warps.  (A first version that read the items from
// global memory through a tile-to-item map needed four dependent round trips
// per warp and ran a quarter slower; a grid-stride walk over the tiles by
// resident warps, slower still, queued each warp's tiles behind their load
// latency.)  The unit index is split into quad, row and plane with
// multiply-shift divisions whose constants the item carries.  Tiles of a
// solve whose run flag is clear are skipped.  The small levels of dozens of
// solves, each far too small to fill the GPU, so share one launch and one
// dependency gap.
//
// Arithmetic: a colour-pass unit is one quad (gsrb4_quad, k_gsrb_v4's
// function), a prolongation unit one quad (prolong4_quad, k_prolong_add_v4's),
// and a restriction unit one column of four quads -- rows 2cj, 2cj + 1 of
// planes 2ck, 2ck + 1 at the same x -- whose residuals (resid4_quad) are summed
// in k_resid_restrict_v4's order (x pairs, then rows, then planes) into the two
// coarse cells above them.  So every value equals the single-solve kernels'.
#include "mg_cellquad.cuh"

namespace mgp {

namespace {

// floor(n / d) for 0 <= n < 2^31 with the item's (m, s) pair for d
__device__ __forceinline__ int mdiv(int n, unsigned m, int s)
{
    return (int)(((unsigned long long)(unsigned)n * m) >> s);
}

template <int OP>
__global__ void __launch_bounds__(256, OP == BATCH_RESTRICT ? 2 : 4)
k_batch_level(const __grid_constant__ BatchLaunch B, const int* __restrict__ run, int color, int zx)
{
    const int wt = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wt >= B.tiles) return;
    int lo = 0, hi = B.nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.items[mid].tile0 <= wt) lo = mid;
        else hi = mid - 1;
    }
    const BatchItem& it = B.items[lo];
    if (!__ldg(run + it.solve)) return;
    const int u = (wt - it.tile0) * kBatchTile + lane;
    if (u >= it.units) return;
    const int r = mdiv(u, it.mq, it.sq), q = u - r * (it.F.nx >> 2);
    if (OP == BATCH_GSRB || OP == BATCH_PROLONG) {
        const int k = mdiv(r, it.my, it.sy), j = r - k * it.F.ny;
        if (OP == BATCH_GSRB) gsrb4_quad<3, false>(it.F, it.x, it.b, color, q, j, k, zx != 0);
        else prolong4_quad<false>(it.F, it.C, it.x, it.xc, q, j, k);
    } else {
        const int cny = it.F.ny >> 1, ck = mdiv(r, it.my, it.sy), cj = r - ck * cny;
        float2 p[2][2];   // [plane][row]: x-pair sums of the quad's residuals
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                float rr[4];
                resid4_quad<false>(it.F, it.x, it.b, q, 2 * cj + dy, 2 * ck + dz, rr);
                p[dz][dy] = make_float2(rr[0] + rr[1], rr[2] + rr[3]);
            }
        float2 v;
        v.x = ((p[0][0].x + p[0][1].x) + (p[1][0].x + p[1][1].x)) * 0.125f;
        v.y = ((p[0][0].y + p[0][1].y) + (p[1][0].y + p[1][1].y)) * 0.125f;
        const int cnx = it.F.nx >> 1;
        *reinterpret_cast<float2*>(it.bc + ((size_t)ck * cny + cj) * cnx + 2 * q) = v;
    }
}

}  // namespace

void batch_magic(int d, unsigned* m, int* s)
{
    // Granlund-Montgomery with N = 31: l = ceil(log2 d), m = ceil(2^(31 + l) / d)
    // < 2^32, and then floor(n m / 2^(31 + l)) = floor(n / d) for 0 <= n < 2^31
    int l = 0;
    while ((1LL << l) < d) ++l;
    *m = (unsigned)(((1ULL << (31 + l)) + (unsigned long long)d - 1) / (unsigned long long)d);
    *s = 31 + l;
}

void batch_level(int op, const BatchLaunch& B, const int* run, int color, int zx, cudaStream_t s)
{
    const int grid = (B.tiles + 7) / 8;   // one warp tile per warp, eight per CTA of 256 threads
    if (op == BATCH_GSRB) MGP_LAUNCH(k_batch_level<BATCH_GSRB><<<grid, 256, 0, s>>>(B, run, color, zx));
    else if (op == BATCH_RESTRICT) MGP_LAUNCH(k_batch_level<BATCH_RESTRICT><<<grid, 256, 0, s>>>(B, run, color, zx));
    else MGP_LAUNCH(k_batch_level<BATCH_PROLONG><<<grid, 256, 0, s>>>(B, run, color, zx));
}

}  // namespace mgp
