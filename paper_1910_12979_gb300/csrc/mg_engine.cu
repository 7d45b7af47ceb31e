// mg_engine.cu -- multigrid hierarchy, V-cycle and refinement drivers, C ABI.
//
// Host side of the library.  A handle owns one resident hierarchy in one
// device workspace (caller-provided or cudaMalloc'd once at setup); solves
// allocate nothing.  Convergence decisions read one small scalar block back
// per iteration; everything else stays on the device.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <type_traits>
#include <new>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_device.cuh"

using namespace mgp;

namespace {

thread_local std::string g_last_error;

mg_status fail(mg_status s, const char* what)
{
    g_last_error = what;
    return s;
}

mg_status cuda_fail(cudaError_t e, const char* where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return MG_ERR_CUDA;
}

#define MG_CK(call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

// Bump allocator over the workspace; with base == nullptr it only counts.
struct Bump {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// ---- live per-kernel event timing (mg_prof_*)
struct ProfRec {
    int id, count;   // kernel class; launches inside the bracket
    double bytes, flops;
    cudaEvent_t a, b;
};
struct Prof {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRec> recs;
    size_t used = 0;
};
Prof& prof()
{
    static Prof p;
    return p;
}
constexpr size_t kProfMax = 65536;

// Returns a record index (or -1) after recording the start event on s.  The
// bracket holds count consecutive launches of the class; bytes and flops are
// their totals.
int prof_begin(int id, double bytes, cudaStream_t s, double flops = 0.0, int count = 1)
{
    Prof& P = prof();
    if (!P.on) return -1;
    std::lock_guard<std::mutex> lk(P.mu);
    if (P.used >= kProfMax) return -1;
    if (P.used == P.recs.size()) {
        ProfRec r{};
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
        P.recs.push_back(r);
    }
    ProfRec& r = P.recs[P.used];
    r.id = id;
    r.count = count;
    r.bytes = bytes;
    r.flops = flops;
    cudaEventRecord(r.a, s);
    return (int)P.used++;
}
void prof_end(int idx, cudaStream_t s)
{
    if (idx < 0) return;
    Prof& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    cudaEventRecord(P.recs[idx].b, s);
}

struct Level {
    int n[3];
    double h[3];
    int N[3];          // stored nodes (nodal)
    size_t ncell, nvec;  // cells; unknown-vector length (cells or stored nodes)
    double* B64[3];
    double* invd64;
    double* diag64;    // level 0: diagonal for the FP64 residual
    double* ew64[3];   // level 0, 3-D nodal: edge sigma sums of the sum-factorised residual
    double* dq64;      //   and its scaled diagonal part
    int kind;          // smoother kernel chosen by the autotuner (0: the default rule)
    float* B32[3];
    double* sig64;
    float* sig32;
    double *x64, *b64, *r64, *t64;
    float *x32, *b32, *r32, *t32;
};

}  // namespace

void mgp::set_last_error(const char* msg) { g_last_error = msg; }

struct mg_handle {
    mg_geometry geo;
    mg_bc bcin;
    mg_options opt;
    BC3 bc;
    int dim, loc, prec, singular;
    int nlev;
    Level lev[kMaxLevels];
    double* f64;
    double* phi_int;
    double* A;
    double* Minv;
    int Nd;
    double* partials;
    DevScalars* d;
    DevScalars* hs;  // pinned host copy
    DevScalars* hs_dev;  // the same pinned block as the device addresses it (written by k_put_words)
    cudaStream_t stream;
    void* ws;
    size_t ws_bytes;
    bool own_ws;
    std::atomic<int> busy;
    // graph-resident solve loops: [0] rhs taken from the caller, [1] rhs already in f64
    cudaGraphExec_t gx[2];
    long long g_fixed[2], g_body[2], g_if[2];  // kernel launches outside the loop / per iteration / per IF
    // host-driven loop: the V-cycle below the finest level, captured once per
    // arithmetic type ([0] FP32, [1] FP64) and replayed as one graph launch
    cudaGraphExec_t cg[2];
    long long cg_launches[2];
    bool cg_failed[2];
    // pipelined legs of the finest FP32 cell level (mg_cellpipe.cu): ticket,
    // exit and epoch counters and the work-item flags; null when not used
    unsigned* pipe_ctr;
    unsigned* pipe_flags;
    cudaEvent_t ev;   // batch projections: the handle's right-hand side is ready
};

void mgp::handle_info(const mg_handle* h, mg_geometry* g, mg_bc* bc, cudaStream_t* s)
{
    if (g) *g = h->geo;
    if (bc) *bc = h->bcin;
    if (s) *s = h->stream;
}

namespace {

bool valid_bc(int v) { return v == MG_BC_PERIODIC || v == MG_BC_NEUMANN || v == MG_BC_DIRICHLET; }

mg_status check_problem(const mg_geometry* g, const mg_bc* bc, const mg_options* o)
{
    if (!g || !bc || !o) return fail(MG_ERR_INVALID_ARG, "null geometry, bc or options");
    if (g->dim != 2 && g->dim != 3) return fail(MG_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (g->loc != MG_LOC_CELL && g->loc != MG_LOC_NODAL) return fail(MG_ERR_INVALID_ARG, "bad location");
    for (int d = 0; d < g->dim; ++d) {
        if (g->n[d] < 1 || !(g->h[d] > 0.0)) return fail(MG_ERR_INVALID_ARG, "n and h must be positive");
        if (!valid_bc(bc->lo[d]) || !valid_bc(bc->hi[d])) return fail(MG_ERR_INVALID_ARG, "bad boundary kind");
        if ((bc->lo[d] == MG_BC_PERIODIC) != (bc->hi[d] == MG_BC_PERIODIC))
            return fail(MG_ERR_INVALID_ARG, "periodic boundaries must be paired");
        if (g->loc == MG_LOC_NODAL && bc->lo[d] == MG_BC_PERIODIC && g->n[d] < 2)
            return fail(MG_ERR_INVALID_ARG, "a periodic nodal axis needs at least 2 cells");
    }
    if (g->dim == 2 && g->n[2] != 1) return fail(MG_ERR_INVALID_ARG, "2-D grids need n[2] == 1");
    double cells = 1.0;
    for (int d = 0; d < g->dim; ++d) cells *= (double)(g->n[d] + 1);
    if (cells > 2.0e9) return fail(MG_ERR_INVALID_ARG, "grid too large for 32-bit indexing");
    if (g->loc == MG_LOC_NODAL) {
        for (int d = 1; d < g->dim; ++d)
            if (fabs(g->h[d] - g->h[0]) > 1e-12 * g->h[0])
                return fail(MG_ERR_INVALID_ARG, "the nodal discretisation needs equal spacing on every axis");
    }
    if (o->prec != MG_PREC_FP64 && o->prec != MG_PREC_MIXED) return fail(MG_ERR_INVALID_ARG, "bad precision");
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 < 1 || o->nu1 > 16 || o->nu2 > 16)
        return fail(MG_ERR_INVALID_ARG, "smoothing sweeps out of range");
    if (o->max_iters < 1) return fail(MG_ERR_INVALID_ARG, "max_iters must be >= 1");
    if (o->interp_order != 0 && o->interp_order != 1) return fail(MG_ERR_INVALID_ARG, "interp_order must be 0 or 1");
    if (!(o->omega > 0.0 && o->omega <= 1.5)) return fail(MG_ERR_INVALID_ARG, "omega out of range");
    if (o->inner_cycles < 0 || o->inner_cycles > 16) return fail(MG_ERR_INVALID_ARG, "inner_cycles out of range");
    return MG_OK;
}

int node_extent(const mg_bc* bc, int n, int d, int dim) { return d >= dim ? 1 : (bc->lo[d] == MG_BC_PERIODIC ? n : n + 1); }

// Lay out the hierarchy (levels, arrays) in the bump allocator.
mg_status plan(mg_handle* h, Bump& B)
{
    const int dim = h->dim;
    const bool mixed = h->prec == MG_PREC_MIXED;
    const bool nodal = h->loc == MG_LOC_NODAL;
    int n[3] = {h->geo.n[0], h->geo.n[1], dim == 3 ? h->geo.n[2] : 1};
    double hh[3] = {h->geo.h[0], h->geo.h[1], dim == 3 ? h->geo.h[2] : 1.0};
    int L = 0;
    const long long cmax = h->opt.coarsest_max > 0 ? h->opt.coarsest_max : 8;
    for (;;) {
        if (L >= kMaxLevels) return fail(MG_ERR_UNSUPPORTED, "too many levels");
        Level& v = h->lev[L];
        memset(&v, 0, sizeof(v));
        for (int d = 0; d < 3; ++d) {
            v.n[d] = n[d];
            v.h[d] = hh[d];
            v.N[d] = node_extent(&h->bcin, n[d], d, dim);
        }
        v.ncell = (size_t)n[0] * n[1] * n[2];
        v.nvec = nodal ? (size_t)v.N[0] * v.N[1] * v.N[2] : v.ncell;
        const size_t nc = v.ncell, nv = v.nvec;
        if (L == 0) {
            if (nodal && dim == 3 && v.N[0] >= 32 && v.N[1] >= 8) {
                for (int d = 0; d < 3; ++d) v.ew64[d] = B.take<double>(nv);
                v.dq64 = B.take<double>(nv);
            } else {
                v.diag64 = B.take<double>(nv);
            }
        }
        if (!nodal) {
            for (int d = 0; d < dim; ++d) {
                size_t m = (size_t)(n[0] + (d == 0)) * (n[1] + (d == 1)) * (n[2] + (d == 2));
                v.B64[d] = B.take<double>(m);
                // + 4: the one-pass sweep copies x-face rows rounded out to 16-byte bounds
                if (mixed) v.B32[d] = B.take<float>(m + 4);
            }
            if (!mixed) v.invd64 = B.take<double>(nc);
        } else {
            v.sig64 = B.take<double>(nc);
            if (mixed) v.sig32 = B.take<float>(nc);
            else v.invd64 = B.take<double>(nv);
        }
        if (mixed) {
            v.x32 = B.take<float>(nv);
            v.b32 = B.take<float>(nv);
            v.t32 = B.take<float>(nv);
            if (nodal) v.r32 = B.take<float>(nv);
        } else {
            if (L > 0) { v.x64 = B.take<double>(nv); v.b64 = B.take<double>(nv); }
            v.t64 = B.take<double>(nv);
            if (nodal) v.r64 = B.take<double>(nv);
        }
        ++L;
        bool can = (long long)nc > cmax;
        for (int d = 0; d < dim; ++d) can = can && (n[d] % 2 == 0) && (n[d] >= 4);
        if (!can) break;
        for (int d = 0; d < dim; ++d) { n[d] /= 2; hh[d] *= 2.0; }
    }
    h->nlev = L;
    h->Nd = (int)h->lev[L - 1].nvec;
    if (h->Nd > kMaxDense) return fail(MG_ERR_UNSUPPORTED, "the grid does not coarsen to a dense-solvable size (<= 512 unknowns)");
    const int nd = h->Nd + (h->singular ? 1 : 0);
    h->f64 = B.take<double>(h->lev[0].nvec);
    h->phi_int = B.take<double>(h->lev[0].nvec);
    h->A = B.take<double>((size_t)nd * 2 * nd);
    h->Minv = B.take<double>((size_t)h->Nd * h->Nd);
    h->partials = B.take<double>((size_t)kRedSlots * kRedBlocks);
    h->d = B.take<DevScalars>(1);
    h->pipe_ctr = nullptr;
    h->pipe_flags = nullptr;
    {
        const Level& v0 = h->lev[0];
        if ((h->opt.flags & MG_FLAG_CELL_PIPE) && mixed && !nodal && dim == 3 && h->nlev >= 2 &&
            v0.ncell >= kPipeMinCells && v0.n[0] % 4 == 0 &&
            v0.n[1] % 2 == 0 && v0.n[2] % 2 == 0 && h->bc.lo[2] != BCP) {
            h->pipe_ctr = B.take<unsigned>(4);
            h->pipe_flags = B.take<unsigned>(cell_pipe_flag_words(v0.n[1], v0.n[2], kPipeMaxNu));
        }
    }
    return MG_OK;
}

template <typename T>
CellLevel<T> cview(const mg_handle* h, int l);
template <>
CellLevel<double> cview<double>(const mg_handle* h, int l)
{
    const Level& v = h->lev[l];
    return CellLevel<double>{v.n[0], v.n[1], v.n[2], h->bc, v.B64[0], v.B64[1], v.B64[2], v.invd64, v.diag64};
}
template <>
CellLevel<float> cview<float>(const mg_handle* h, int l)
{
    const Level& v = h->lev[l];
    return CellLevel<float>{v.n[0], v.n[1], v.n[2], h->bc, v.B32[0], v.B32[1], v.B32[2], nullptr, nullptr};
}

template <typename T>
NodeLevel<T> nview(const mg_handle* h, int l);
template <>
NodeLevel<double> nview<double>(const mg_handle* h, int l)
{
    const Level& v = h->lev[l];
    return NodeLevel<double>{v.n[0], v.n[1], v.n[2], v.N[0], v.N[1], v.N[2], h->bc, v.sig64,
                             1.0 / (v.h[0] * v.h[0]), v.invd64, v.diag64};
}
template <>
NodeLevel<float> nview<float>(const mg_handle* h, int l)
{
    const Level& v = h->lev[l];
    return NodeLevel<float>{v.n[0], v.n[1], v.n[2], v.N[0], v.N[1], v.N[2], h->bc, v.sig32,
                            (float)(1.0 / (v.h[0] * v.h[0])), nullptr, nullptr};
}

// Step a1: coefficients on every level and the dense inverse of the coarsest operator.
mg_status build_coefficients(mg_handle* h, const mg_coeff* c)
{
    if (!c || !c->sigma) return fail(MG_ERR_INVALID_ARG, "sigma is required");
    cudaStream_t s = h->stream;
    const int dim = h->dim;
    const bool mixed = h->prec == MG_PREC_MIXED;
    if (h->loc == MG_LOC_CELL) {
        Level& v0 = h->lev[0];
        CellLevel<double> L0 = cview<double>(h, 0);
        const bool explicit_faces = c->face[0] || c->face[1] || (dim == 3 && c->face[2]);
        if (explicit_faces) {
            for (int d = 0; d < dim; ++d)
                if (!c->face[d]) return fail(MG_ERR_INVALID_ARG, "explicit faces must be given for every axis");
            cell_scale_faces(dim, L0, c->face, v0.h, v0.B64[0], v0.B64[1], v0.B64[2], s);
        } else {
            cell_faces_from_sigma(dim, L0, c->sigma, v0.h, v0.B64[0], v0.B64[1], v0.B64[2], s);
        }
        for (int l = 1; l < h->nlev; ++l) {
            Level& v = h->lev[l];
            cell_coarsen_faces(dim, cview<double>(h, l - 1), cview<double>(h, l), v.B64[0], v.B64[1], v.B64[2], s);
        }
        for (int l = 0; l < h->nlev; ++l) {
            Level& v = h->lev[l];
            if (mixed) {
                for (int d = 0; d < dim; ++d) {
                    size_t m = (size_t)(v.n[0] + (d == 0)) * (v.n[1] + (d == 1)) * (v.n[2] + (d == 2));
                    vec_to_f32(v.B32[d], v.B64[d], m, s);
                }
            } else {
                CellLevel<double> V = cview<double>(h, l);
                V.invd = nullptr;
                cell_invdiag(dim, V, v.invd64, s);
            }
        }
        {
            CellLevel<double> V = cview<double>(h, 0);
            V.invd = nullptr;
            V.diag = nullptr;
            cell_diag(dim, V, h->lev[0].diag64, s);
        }
        const int n = h->Nd + h->singular;
        cell_dense_assemble(dim, cview<double>(h, h->nlev - 1), h->A, 2 * n, s);
    } else {
        vec_copy_f64(h->lev[0].sig64, c->sigma, h->lev[0].ncell, s);
        for (int l = 1; l < h->nlev; ++l)
            node_coarsen_sigma(dim, nview<double>(h, l - 1), nview<double>(h, l), h->lev[l].sig64, s);
        for (int l = 0; l < h->nlev; ++l) {
            Level& v = h->lev[l];
            if (mixed) {
                vec_to_f32(v.sig32, v.sig64, v.ncell, s);
            } else {
                NodeLevel<double> V = nview<double>(h, l);
                V.invd = nullptr;
                node_invdiag(dim, V, v.invd64, s);
            }
        }
        {
            NodeLevel<double> V = nview<double>(h, 0);
            V.invd = nullptr;
            V.diag = nullptr;
            const Level& v0 = h->lev[0];
            if (v0.dq64) node_edges(V, NodeEdges{{v0.ew64[0], v0.ew64[1], v0.ew64[2]}, v0.dq64}, s);
            else node_diag(dim, V, v0.diag64, s);
        }
        const int n = h->Nd + h->singular;
        NodeLevel<double> C = nview<double>(h, h->nlev - 1);
        C.invd = nullptr;
        node_dense_assemble(dim, C, h->A, 2 * n, s);
    }
    dense_invert(h->A, h->Nd, h->singular, h->Minv, &h->d->info, s);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

// Small device-to-host results (the scalar block, batch counters) are written
// into mapped pinned memory by a one-block kernel instead of a copy: a copy
// would queue on a copy engine behind whatever large transfer the caller has in
// flight on another stream (a step's uploads or read-backs), a kernel does not.
__global__ void k_put_words(int* __restrict__ dst, const int* __restrict__ src, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
void put_host(void* dst_dev, const void* src, size_t bytes, cudaStream_t s)
{
    MGP_LAUNCH(k_put_words<<<1, 64, 0, s>>>((int*)dst_dev, (const int*)src, (int)(bytes / sizeof(int))));
}
static_assert(sizeof(DevScalars) % sizeof(int) == 0, "scalar block copied as words");

mg_status readback(mg_handle* h)
{
    put_host(h->hs_dev, h->d, sizeof(DevScalars), h->stream);
    MG_CK(cudaStreamSynchronize(h->stream));
    if (h->hs->async_err) return fail(MG_ERR_CUDA, "a bounded wait inside a kernel (an asynchronous copy or a pipelined pass) gave up");
    return MG_OK;
}

__global__ void k_keep(DevScalars* d, int fslot, int srcslot)
{
    if (fslot >= 0) {
        d->fnorm2 = d->red[fslot];
        set_fscale(d);
    }
    if (srcslot >= 0) d->src2 = d->red[srcslot];
}

// f64 holds the system rhs, red[] holds {sum f, src2, sum f^2} from the rhs pass
// (or {sum f, sum f^2} when from vec_sum_sq with fslot = 1).  Removes the mean
// when singular and stores ||f||^2.
void finish_rhs(mg_handle* h, int fslot, int srcslot)
{
    cudaStream_t s = h->stream;
    if (srcslot >= 0) MGP_LAUNCH(k_keep<<<1, 1, 0, s>>>(h->d, -1, srcslot));
    if (h->singular) {
        const size_t n = h->lev[0].nvec;
        vec_sub_mean(h->f64, n, &h->d->red[0], (double)n, s);
        vec_sum_sq(h->f64, n, h->partials, s);
        reduce_finalize(h->partials, 2, h->d->red, s);
        fslot = 1;
    }
    MGP_LAUNCH(k_keep<<<1, 1, 0, s>>>(h->d, fslot, -1));
}

// FP64 operations per node of the sum-factorised nodal residual, an FMA
// counted as two: per cell position 3 adds (2x2 phi sum) + 1 add + 1 mul (Q),
// times 297/256 cell positions per node; per node 3 + 1 adds (2x2 Q sums),
// 6 FMAs (edge terms), 1 mul + 1 FMA (scaling and diagonal), 1 sub.  The
// residual's power-of-two scale folds into the FP32 conversion (no operation).
constexpr double kNodeResidSFFlops = 5.0 * 297.0 / 256.0 + 20.0;
// FP64 operations per cell of the cell residual: 6 FMAs (face terms), 1 FMA
// (stored diagonal), 1 sub; per node of the nodal row assembled from 8 sigma: 44
constexpr double kCellResidFlops = 15.0, kNodeResidRowFlops = 44.0;

// ||f - L phi||^2 / ||f||^2 -> d->rnorm2; optional FP32 copy of the residual
// divided by fscale (the power of two <= ||f||).
void residual64(mg_handle* h, const double* phi, float* r32)
{
    cudaStream_t s = h->stream;
    const bool nodal = h->loc == MG_LOC_NODAL;
    const double nv = (double)h->lev[0].nvec;
    const Level& v0 = h->lev[0];
    const bool sf = nodal && v0.dq64;
    const int pr = prof_begin(nodal ? MG_PROF_NODE_RESID64 : MG_PROF_RESID64, (24.0 + (r32 ? 4.0 : 0.0)) * nv, s,
                              (sf ? kNodeResidSFFlops : nodal ? kNodeResidRowFlops : kCellResidFlops) * nv);
    if (h->loc == MG_LOC_CELL)
        cell_resid64(h->dim, cview<double>(h, 0), phi, h->f64, r32, &h->d->fscale, h->partials, s,
                     !(h->opt.flags & MG_FLAG_NO_FUSED));
    else if (sf)
        node_resid64_sf(nview<double>(h, 0), NodeEdges{{v0.ew64[0], v0.ew64[1], v0.ew64[2]}, v0.dq64}, phi, h->f64,
                        r32, &h->d->fscale, h->partials, s);
    else
        node_resid64(h->dim, nview<double>(h, 0), phi, h->f64, r32, &h->d->fscale, h->partials, s);
    prof_end(pr, s);
    reduce_finalize(h->partials, 1, &h->d->rnorm2, s, &h->d->rscale2);
}

// The first residual when the solve starts from phi = 0 (MG_FLAG_ZERO_GUESS):
// phi is cleared and r = f needs no operator application.
void init_zero_guess(mg_handle* h, double* phi, float* r32)
{
    cudaStream_t s = h->stream;
    const size_t n = h->lev[0].nvec;
    cudaMemsetAsync(phi, 0, n * sizeof(double), s);
    vec_init_zero_guess(h->f64, r32, &h->d->fscale, h->partials, n, s);
    reduce_finalize(h->partials, 1, &h->d->rnorm2, s, &h->d->rscale2);
}

bool zero_guess(const mg_handle* h) { return (h->opt.flags & MG_FLAG_ZERO_GUESS) != 0; }

template <typename T>
T* lx(mg_handle* h, int l);
template <>
double* lx<double>(mg_handle* h, int l) { return h->lev[l].x64; }
template <>
float* lx<float>(mg_handle* h, int l) { return h->lev[l].x32; }
template <typename T>
T* lb(mg_handle* h, int l);
template <>
double* lb<double>(mg_handle* h, int l) { return h->lev[l].b64; }
template <>
float* lb<float>(mg_handle* h, int l) { return h->lev[l].b32; }
template <typename T>
T* lr(mg_handle* h, int l);
template <>
double* lr<double>(mg_handle* h, int l) { return h->lev[l].r64; }
template <>
float* lr<float>(mg_handle* h, int l) { return h->lev[l].r32; }
template <typename T>
T* lt(mg_handle* h, int l);
template <>
double* lt<double>(mg_handle* h, int l) { return h->lev[l].t64; }
template <>
float* lt<float>(mg_handle* h, int l) { return h->lev[l].t32; }

template <typename T>
void zero(T* p, size_t n, cudaStream_t s)
{
    cudaMemsetAsync(p, 0, n * sizeof(T), s);
}

// nu red-black sweeps (red, then black) on level l.  FP32 levels run two
// vectorised colour passes in place; with MG_FLAG_SWEEP_PIPE (or FP64 levels)
// levels that tile run one pipelined launch per sweep, ping-ponging between x
// and the level's temp vector; the rest run the plain colour passes.  All are
// the same arithmetic.  The finest level's launches are timed when profiling.
template <typename T>
void cell_smooth(mg_handle* h, int l, const CellLevel<T>& V, T* x, const T* b, int nu)
{
    cudaStream_t s = h->stream;
    const double cells = (double)h->lev[l].ncell;
    T* t = lt<T>(h, l);
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    const int kind = h->lev[l].kind;   // 1..3: four-cell passes, 8/16/32 quads per block row; 4: pipelined;
                                       // 8: one pass, TMA-staged
    if constexpr (std::is_same<T, float>::value) {
        const bool tma = kind == 8 || (kind == 0 && (h->opt.flags & MG_FLAG_SWEEP_TMA));
        if (tma && !(h->opt.flags & MG_FLAG_NO_FUSED) && cell_gsrb_tma_ok(h->dim, V, x, t, b) &&
            cell_gsrb_tma_fits(V.nx)) {
            T* src = x;
            T* dst = t;
            const int pr =
                l == 0 && nu > 0 ? prof_begin(MG_PROF_CELL_SMOOTH_FINE, 4.0 * sizeof(T) * cells * nu, s, 0.0, nu) : -1;
            for (int k = 0; k < nu; ++k) {
                cell_gsrb_tma(V, src, dst, b, &h->d->async_err, s);
                T* tmp = src;
                src = dst;
                dst = tmp;
            }
            prof_end(pr, s);
            if (src != x) cudaMemcpyAsync(x, src, h->lev[l].nvec * sizeof(T), cudaMemcpyDeviceToDevice, s);
            return;
        }
        const bool pipe = kind == 4 || (kind == 0 && (h->opt.flags & MG_FLAG_SWEEP_PIPE));
        if (!(h->opt.flags & MG_FLAG_NO_FUSED) && !pipe && cell_gsrb_v4_ok(h->dim, V, x, b)) {
            const int pr =
                l == 0 && nu > 0
                    ? prof_begin(MG_PROF_CELL_SMOOTH_FINE, 2.0 * sizeof(T) * cells * 2 * nu, s, 0.0, 2 * nu)
                    : -1;
            for (int k = 0; k < nu; ++k)
                for (int color = 0; color < 2; ++color)
                    cell_gsrb_v4(h->dim, V, x, b, color, s, kind >= 1 && kind <= 3 ? 4 << kind : 0);
            prof_end(pr, s);
            return;
        }
    }
    if (!(h->opt.flags & MG_FLAG_NO_FUSED) && cell_gsrb_fused_ok<T>(h->dim, V) && a16(x) && a16(t) && a16(b)) {
        T* src = x;
        T* dst = t;
        const int pr =
            l == 0 && nu > 0 ? prof_begin(MG_PROF_CELL_SMOOTH_FINE, 4.0 * sizeof(T) * cells * nu, s, 0.0, nu) : -1;
        for (int k = 0; k < nu; ++k) {
            cell_gsrb_sweep<T>(h->dim, V, src, dst, b, s);
            T* tmp = src;
            src = dst;
            dst = tmp;
        }
        prof_end(pr, s);
        if (src != x) cudaMemcpyAsync(x, src, h->lev[l].nvec * sizeof(T), cudaMemcpyDeviceToDevice, s);
        return;
    }
    const int pr =
        l == 0 && nu > 0 ? prof_begin(MG_PROF_CELL_SMOOTH_FINE, 2.0 * sizeof(T) * cells * 2 * nu, s, 0.0, 2 * nu)
                         : -1;
    for (int k = 0; k < nu; ++k)
        for (int color = 0; color < 2; ++color) cell_gsrb<T>(h->dim, V, x, b, color, s);
    prof_end(pr, s);
}

// The pipelined legs (mg_cellpipe.cu) apply, when MG_FLAG_CELL_PIPE asks for
// them, to the finest FP32 level of a handle that laid out their counters.
bool pipe_on(const mg_handle* h)
{
    return h->pipe_ctr && (h->opt.flags & MG_FLAG_CELL_PIPE) &&
           !(h->opt.flags & (MG_FLAG_NO_FUSED | MG_FLAG_SWEEP_PIPE | MG_FLAG_SWEEP_TMA));
}

PipeSync pipe_sync(mg_handle* h) { return PipeSync{h->pipe_ctr, h->pipe_flags, &h->d->async_err}; }

// Down leg of the finest cell level: (x0 = 0 if zero_init,) nu1 sweeps, and the
// residual restricted into level 1's b.  One pipelined launch where it
// applies; else the smoother passes and the residual + restriction kernel.
template <typename T>
void cell_down0(mg_handle* h, T* x0, const T* b0, bool zero_init)
{
    cudaStream_t s = h->stream;
    const int dim = h->dim;
    const CellLevel<T> V = cview<T>(h, 0);
    if constexpr (std::is_same<T, float>::value) {
        const int nu = h->opt.nu1;
        if (pipe_on(h) && nu >= 1 && nu <= kPipeMaxNu && cell_pipe_ok(V, x0, b0)) {
            // algorithmic words per cell: 4 per sweep, 3 + 1/8 for the residual + restriction
            const int pr = prof_begin(MG_PROF_CELL_PIPE_DOWN,
                                      (4.0 * nu + 3.0 + 0.125) * sizeof(T) * (double)h->lev[0].ncell, s);
            cell_pipe_down(V, x0, b0, lb<T>(h, 1), nu, zero_init, pipe_sync(h), s);
            prof_end(pr, s);
            return;
        }
    }
    if (zero_init) zero(x0, h->lev[0].nvec, s);
    cell_smooth<T>(h, 0, V, x0, b0, h->opt.nu1);
    const int pr = prof_begin(MG_PROF_CELL_RESTRICT_FINE, (3.0 + 1.0 / (1 << dim)) * sizeof(T) * h->lev[0].ncell, s);
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (!(h->opt.flags & (MG_FLAG_NO_FUSED | MG_FLAG_SWEEP_PIPE)) &&
            cell_resid_restrict_v4_ok(dim, V, x0, b0, lb<T>(h, 1))) {
            cell_resid_restrict_v4(V, x0, b0, lb<T>(h, 1), s);
            done = true;
        }
    }
    if (!done) cell_resid_restrict<T>(dim, V, x0, b0, lb<T>(h, 1), s);
    prof_end(pr, s);
}

// Up leg of the finest cell level: x0 += P x1, then nu2 sweeps; one pipelined
// launch where it applies (linear prolongation).
template <typename T>
void cell_up0(mg_handle* h, T* x0, const T* b0)
{
    cudaStream_t s = h->stream;
    const int dim = h->dim;
    const CellLevel<T> V = cview<T>(h, 0);
    if constexpr (std::is_same<T, float>::value) {
        const int nu = h->opt.nu2;
        if (pipe_on(h) && nu >= 1 && nu <= kPipeMaxNu && h->opt.interp_order == 1 && cell_pipe_ok(V, x0, b0) &&
            cell_prolong_v4_ok(dim, V, x0, lx<T>(h, 1))) {
            // algorithmic words per cell: the prolongation fused into the first
            // sweep 4 + 1/8, then 4 per further sweep
            const int pr =
                prof_begin(MG_PROF_CELL_PIPE_UP, (4.0 * nu + 0.125) * sizeof(T) * (double)h->lev[0].ncell, s);
            cell_pipe_up(V, cview<T>(h, 1), x0, b0, lx<T>(h, 1), nu, pipe_sync(h), s);
            prof_end(pr, s);
            return;
        }
    }
    cell_prolong_add<T>(dim, V, cview<T>(h, 1), x0, lx<T>(h, 1), h->opt.interp_order, s);
    cell_smooth<T>(h, 0, V, x0, b0, h->opt.nu2);
}

// First level of the one-launch coarse end of a cell V-cycle: levels lc .. L-1
// (at most kCoarseCells cells each) run as one launch; L when nothing is fused.
int cell_coarse_start(const mg_handle* h)
{
    const int L = h->nlev;
    if (h->opt.flags & MG_FLAG_NO_FUSED) return L;
    int lc = L - 1;
    while (lc > 0 && h->lev[lc - 1].ncell <= (size_t)kCoarseCells && L - (lc - 1) <= kCoarseMaxLevels) --lc;
    return lc == L - 1 ? L : lc;   // a single level: nothing to fuse
}

// Levels first .. L-1 of a cell V-cycle on L x = b: the down legs of levels
// first .. lc-1, the coarse end, and the up legs back to level first.  Level 0
// uses x0 and b0; the other levels their stored arrays.
template <typename T>
void vcycle_cell_range(mg_handle* h, int first, T* x0, const T* b0, bool zero_init)
{
    cudaStream_t s = h->stream;
    const int dim = h->dim, L = h->nlev, lc = cell_coarse_start(h);
    auto X = [&](int l) { return l == 0 ? x0 : lx<T>(h, l); };
    auto Bv = [&](int l) { return l == 0 ? b0 : (const T*)lb<T>(h, l); };
    for (int l = first; l < lc && l < L - 1; ++l) {
        if (l == 0) {
            cell_down0<T>(h, x0, b0, zero_init);
            continue;
        }
        zero(X(l), h->lev[l].nvec, s);
        const CellLevel<T> V = cview<T>(h, l);
        cell_smooth<T>(h, l, V, X(l), Bv(l), h->opt.nu1);
        const int pr = l == 0 ? prof_begin(MG_PROF_CELL_RESTRICT_FINE,
                                           (3.0 + 1.0 / (1 << dim)) * sizeof(T) * h->lev[0].ncell, s) : -1;
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
            if (!(h->opt.flags & (MG_FLAG_NO_FUSED | MG_FLAG_SWEEP_PIPE)) &&
                cell_resid_restrict_v4_ok(dim, V, X(l), Bv(l), lb<T>(h, l + 1))) {
                cell_resid_restrict_v4(V, X(l), Bv(l), lb<T>(h, l + 1), s);
                done = true;
            }
        }
        if (!done) cell_resid_restrict<T>(dim, V, X(l), Bv(l), lb<T>(h, l + 1), s);
        prof_end(pr, s);
    }
    if (lc < L) {
        CellLevel<T> Ls[kCoarseMaxLevels];
        T* xs[kCoarseMaxLevels];
        T* bs[kCoarseMaxLevels];
        for (int l = lc; l < L; ++l) {
            Ls[l - lc] = cview<T>(h, l);
            xs[l - lc] = X(l);
            bs[l - lc] = const_cast<T*>(Bv(l));
        }
        coarse_cycle<T>(dim, L - lc, Ls, xs, bs, h->Minv, h->Nd, h->opt.nu1, h->opt.nu2, h->opt.interp_order,
                        lc > 0 || zero_init, s);
    } else {
        dense_apply<T>(h->Minv, h->Nd, Bv(L - 1), X(L - 1), s);
    }
    for (int l = (lc < L ? lc : L - 1) - 1; l >= first; --l) {
        if (l == 0) {
            cell_up0<T>(h, x0, b0);
            continue;
        }
        const CellLevel<T> V = cview<T>(h, l);
        cell_prolong_add<T>(dim, V, cview<T>(h, l + 1), X(l), X(l + 1), h->opt.interp_order, s);
        cell_smooth<T>(h, l, V, X(l), Bv(l), h->opt.nu2);
    }
}

template <typename T>
void vcycle_node_range(mg_handle* h, int first, T* x0, const T* b0, bool zero_init);
int node_coarse_start(const mg_handle* h);

// The levels below the finest of a V-cycle (levels 1 .. L-1, which read the
// restricted residual in level 1's b and leave level 1's x for the
// prolongation) touch only arrays of the hierarchy, so in the host-driven loop
// they are captured once into a graph and replayed as one launch per V-cycle
// instead of some 30-40 stream launches of mostly small kernels.  Null when
// the hierarchy is too shallow for this to pay, while h->stream is itself
// being captured (a graph-resident solve records the levels inline), or if the
// capture failed (the caller then launches the levels one by one).
template <typename T>
cudaGraphExec_t coarse_graph(mg_handle* h)
{
    const bool nodal = h->loc == MG_LOC_NODAL;
    if ((nodal ? node_coarse_start(h) : cell_coarse_start(h)) < 2 || h->nlev < 3) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    const int i = std::is_same<T, float>::value ? 0 : 1;
    if (h->cg[i] || h->cg_failed[i]) return h->cg[i];
    h->cg_failed[i] = true;
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    const cudaStream_t saved = h->stream;
    const long long c0 = launch_count();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        h->stream = cap;
        if (nodal) vcycle_node_range<T>(h, 1, nullptr, nullptr, false);
        else vcycle_cell_range<T>(h, 1, nullptr, nullptr, false);
        h->stream = saved;
        ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && g;
    }
    const long long n = launch_count() - c0;
    add_launches(-n);   // capture enqueues nothing; replays are counted
    cudaGraphExec_t ex = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (!ok) {
        cudaGetLastError();   // clear a capture error: the levels run as plain launches
        return nullptr;
    }
    h->cg[i] = ex;
    h->cg_launches[i] = n;
    h->cg_failed[i] = false;
    return ex;
}

// One V-cycle on L x0 = b0 (level 0 arrays given), cell-centred.
template <typename T>
void vcycle_cell(mg_handle* h, T* x0, const T* b0, bool zero_init)
{
    cudaGraphExec_t cg = coarse_graph<T>(h);
    if (!cg) {
        vcycle_cell_range<T>(h, 0, x0, b0, zero_init);
        return;
    }
    cudaStream_t s = h->stream;
    cell_down0<T>(h, x0, b0, zero_init);
    cudaGraphLaunch(cg, s);
    add_launches(h->cg_launches[std::is_same<T, float>::value ? 0 : 1]);
    cell_up0<T>(h, x0, b0);
}

template <typename T>
void node_smooth(mg_handle* h, int l, T* x, const T* b, int sweeps)
{
    cudaStream_t s = h->stream;
    const NodeLevel<T> V = nview<T>(h, l);
    T* t = lt<T>(h, l);
    const T om = (T)h->opt.omega;
    const int pr = l == 0 && sweeps > 0
                       ? prof_begin(MG_PROF_NODE_SMOOTH_FINE, 4.0 * sizeof(T) * h->lev[0].nvec * sweeps, s, 0.0, sweeps)
                       : -1;
    for (int k = 0; k < sweeps; ++k) {
        const bool tiled = !(h->opt.flags & MG_FLAG_NO_FUSED);
        if (k % 2 == 0) node_jacobi<T>(h->dim, V, x, t, b, om, tiled, s, h->lev[l].kind);
        else node_jacobi<T>(h->dim, V, t, x, b, om, tiled, s, h->lev[l].kind);
    }
    prof_end(pr, s);
    if (sweeps % 2 == 1) cudaMemcpyAsync(x, t, h->lev[l].nvec * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

// First level of the one-launch coarse end of a nodal V-cycle (levels of at
// most kCoarseNodes stored nodes); L when nothing is fused.
int node_coarse_start(const mg_handle* h)
{
    const int L = h->nlev;
    if (h->opt.flags & MG_FLAG_NO_FUSED) return L;
    int lc = L - 1;
    while (lc > 0 && h->lev[lc - 1].nvec <= (size_t)kCoarseNodes && L - (lc - 1) <= kCoarseMaxLevels) --lc;
    return lc == L - 1 ? L : lc;   // a single level: nothing to fuse
}

// Levels first .. L-1 of a nodal V-cycle (as vcycle_cell_range).
template <typename T>
void vcycle_node_range(mg_handle* h, int first, T* x0, const T* b0, bool zero_init)
{
    cudaStream_t s = h->stream;
    const int dim = h->dim, L = h->nlev, lc = node_coarse_start(h);
    auto X = [&](int l) { return l == 0 ? x0 : lx<T>(h, l); };
    auto Bv = [&](int l) { return l == 0 ? b0 : (const T*)lb<T>(h, l); };
    for (int l = first; l < lc && l < L - 1; ++l) {
        if (l > 0 || zero_init) zero(X(l), h->lev[l].nvec, s);
        node_smooth<T>(h, l, X(l), Bv(l), h->opt.nu1);
        node_resid<T>(dim, nview<T>(h, l), X(l), Bv(l), lr<T>(h, l), !(h->opt.flags & MG_FLAG_NO_FUSED), s,
                      h->lev[l].kind);
        node_restrict<T>(dim, nview<T>(h, l), nview<T>(h, l + 1), lr<T>(h, l), lb<T>(h, l + 1), s);
    }
    if (lc < L) {
        NodeLevel<T> Ls[kCoarseMaxLevels];
        T *xs[kCoarseMaxLevels], *bs[kCoarseMaxLevels], *ts[kCoarseMaxLevels], *rs[kCoarseMaxLevels];
        for (int l = lc; l < L; ++l) {
            Ls[l - lc] = nview<T>(h, l);
            xs[l - lc] = X(l);
            bs[l - lc] = const_cast<T*>(Bv(l));
            ts[l - lc] = lt<T>(h, l);
            rs[l - lc] = lr<T>(h, l);
        }
        node_coarse_cycle<T>(dim, L - lc, Ls, xs, bs, ts, rs, h->Minv, h->Nd, h->opt.nu1, h->opt.nu2,
                             (T)h->opt.omega, lc > 0 || zero_init, s);
    } else {
        dense_apply<T>(h->Minv, h->Nd, Bv(L - 1), X(L - 1), s);
    }
    for (int l = (lc < L ? lc : L - 1) - 1; l >= first; --l) {
        node_prolong_add<T>(dim, nview<T>(h, l), nview<T>(h, l + 1), X(l), X(l + 1), s);
        node_smooth<T>(h, l, X(l), Bv(l), h->opt.nu2);
    }
}

template <typename T>
void vcycle_node(mg_handle* h, T* x0, const T* b0, bool zero_init)
{
    cudaGraphExec_t cg = coarse_graph<T>(h);
    if (!cg) {
        vcycle_node_range<T>(h, 0, x0, b0, zero_init);
        return;
    }
    cudaStream_t s = h->stream;
    const int dim = h->dim;
    if (zero_init) zero(x0, h->lev[0].nvec, s);
    node_smooth<T>(h, 0, x0, b0, h->opt.nu1);
    node_resid<T>(dim, nview<T>(h, 0), x0, b0, lr<T>(h, 0), !(h->opt.flags & MG_FLAG_NO_FUSED), s, h->lev[0].kind);
    node_restrict<T>(dim, nview<T>(h, 0), nview<T>(h, 1), lr<T>(h, 0), lb<T>(h, 1), s);
    cudaGraphLaunch(cg, s);
    add_launches(h->cg_launches[std::is_same<T, float>::value ? 0 : 1]);
    node_prolong_add<T>(dim, nview<T>(h, 0), nview<T>(h, 1), x0, lx<T>(h, 1), s);
    node_smooth<T>(h, 0, x0, b0, h->opt.nu2);
}

// Remove the mean of phi (singular problems).
void gauge(mg_handle* h, double* phi)
{
    cudaStream_t s = h->stream;
    const size_t n = h->lev[0].nvec;
    vec_sum_sq(phi, n, h->partials, s);
    reduce_finalize(h->partials, 2, h->d->red, s);
    vec_sub_mean(phi, n, &h->d->red[0], (double)n, s);
}

int inner_cycles(const mg_handle* h)
{
    if (h->opt.inner_cycles > 0) return h->opt.inner_cycles;
    return 2;
}

// Mixed refinement step: a few FP32 V-cycles on A e = r / fscale from e = 0,
// then phi += fscale e in FP64.
void mixed_correction(mg_handle* h, double* phi, int cycles)
{
    float* e = h->lev[0].x32;
    for (int j = 0; j < cycles; ++j) {
        if (h->loc == MG_LOC_NODAL) vcycle_node<float>(h, e, h->lev[0].b32, j == 0);
        else vcycle_cell<float>(h, e, h->lev[0].b32, j == 0);
    }
    vec_axpy_f32(phi, e, &h->d->fscale, h->lev[0].nvec, h->stream);
}

bool adaptive_cycles(const mg_handle* h) { return h->prec == MG_PREC_MIXED && h->opt.inner_cycles == 0; }

// Automatic inner cycles of mixed refinement.  The first step runs
// kMaxInner V-cycles.  After a step of m V-cycles that took the relative
// residual from prev_rel to rel, the rate per V-cycle is q^(1/m) with
// q = rel / prev_rel, and the next step runs the fewest V-cycles k <= kMaxInner
// that this rate predicts to reach half the tolerance:
//   rel q^(k/m) <= tol / 2   <=>   rel^m q^k <= (tol / 2)^m,
// tested in that second form, with products only, so that the host loop and
// the graph (k_check) take the same decision bit for bit.  Each outer step
// costs an FP64 residual about as long as an FP32 V-cycle, and an FP32 inner
// solve that runs on loses rate late in a step, so more than three V-cycles
// per step do not pay (at 256^3 a fixed four per step took 16 MAC and 12 nodal
// V-cycles, a fixed three 15 and 9, this rule 13 and 8).
constexpr int kMaxInner = 3;

__host__ __device__ inline int next_cycles(bool first, int last_m, double prev_rel, double rel, double tol)
{
    if (first || last_m < 1 || !(prev_rel > 0.0) || !(rel > 0.0) || !(rel < prev_rel)) return kMaxInner;
    const double q = rel / prev_rel, t = 0.5 * tol;
    double lhs = 1.0, rhs = 1.0;
    for (int i = 0; i < last_m; ++i) {
        lhs *= rel;
        rhs *= t;
    }
    for (int k = 1; k < kMaxInner; ++k) {
        lhs *= q;
        if (lhs <= rhs) return k;
    }
    return kMaxInner;
}


// Iterate on L phi = f64 (rhs and ||f|| already prepared on the device).
mg_status solve_core(mg_handle* h, double* phi, double tol, mg_stats* st, bool constraint_tol = false)
{
    cudaStream_t s = h->stream;
    const bool mixed = h->prec == MG_PREC_MIXED;
    const bool nodal = h->loc == MG_LOC_NODAL;
    float* r32 = mixed ? h->lev[0].b32 : nullptr;
    if (zero_guess(h)) {
        init_zero_guess(h, phi, r32);
    } else {
        if (nodal) node_zero_dirichlet<double>(h->dim, nview<double>(h, 0), phi, s);
        residual64(h, phi, r32);
    }
    mg_status rc = readback(h);
    if (rc != MG_OK) return rc;
    if (h->hs->info != 0)
        return fail(MG_ERR_UNSUPPORTED, "the coarsest-level operator is singular");
    const double fn2 = h->hs->fnorm2;
    if (constraint_tol && fn2 > 0.0 && h->hs->src2 > 0.0) {   // as k_constraint_tol
        const double c = tol * sqrt(h->hs->src2 / fn2);
        if (c < tol) tol = c;
    }
    if (st) { st->rhs_norm = sqrt(fn2); st->iters = 0; st->rel_resid = 0.0; }
    if (fn2 == 0.0) {
        zero(phi, h->lev[0].nvec, s);
        return MG_OK;
    }
    double rel = sqrt(h->hs->rnorm2);
    const double rel0 = rel;
    double best = rel;
    int stall = 0, it = 0;
    mg_status status = MG_OK;
    const bool adaptive = adaptive_cycles(h);
    int m = adaptive ? next_cycles(true, 0, 0.0, rel, tol) : inner_cycles(h), vcyc = 0;
    double prev = rel;
    while (rel > tol) {
        if (it >= h->opt.max_iters) { status = MG_ERR_NOT_CONVERGED; break; }
        if (mixed) {
            mixed_correction(h, phi, m);
            vcyc += m;
        } else {
            vcyc += 1;
            if (nodal) vcycle_node<double>(h, phi, h->f64, false);
            else vcycle_cell<double>(h, phi, h->f64, false);
        }
        ++it;
        residual64(h, phi, r32);
        rc = readback(h);
        if (rc != MG_OK) return rc;
        rel = sqrt(h->hs->rnorm2);
        if (!isfinite(rel) || rel > 1e6 * (rel0 > 1.0 ? rel0 : 1.0)) { status = MG_ERR_DIVERGED; break; }
        if (rel < 0.9 * best) { best = rel; stall = 0; }
        else if (++stall >= 4) { status = rel <= tol ? MG_OK : MG_ERR_NOT_CONVERGED; break; }
        if (rel < best) best = rel;
        if (adaptive) m = next_cycles(false, m, prev, rel, tol);   // as k_check
        prev = rel;
    }
    if (h->singular) gauge(h, phi);
    if (st) { st->iters = it; st->rel_resid = rel; st->vcycles = vcyc; }
    if (status != MG_OK) {
        char buf[160];
        snprintf(buf, sizeof buf, "stopped after %d iterations at relative residual %.3e (tol %.3e)", it, rel, tol);
        g_last_error = buf;
    }
    return status;
}


// ======================================================= graph-resident solves
//
// A whole solve is captured once into a CUDA graph: rhs staging, the initial
// residual, a conditional WHILE node whose body is one V-cycle (+ refinement
// update) followed by the FP64 residual and a one-thread check kernel that
// decides on the device whether to iterate again (cudaGraphSetConditional),
// then the gauge, the copy-out of phi and a copy of the scalar block to pinned
// host memory.  A solve is then one graph launch and one synchronisation; the
// per-call pointers and tolerance reach the graph through the scalar block
// (k_set_io), so the captured graph stays valid for every call.  The decisions
// are the host loop's, made with the same formulas, so both paths iterate the
// same number of times and produce the same phi.

__global__ void k_set_io(DevScalars* d, const double* rhs, double* phi, double tol, int maxit)
{
    d->rhs_in = rhs;
    d->phi_io = phi;
    d->tol = tol;
    d->maxit = maxit;
    d->ncyc = kMaxInner;
    d->n_extra = 0;
}

// MAC projection: the constraint after the update equals the solver residual
// (L = D B G), so ||D(beta0 U) - beta0 S|| <= tol ||beta0 S|| needs
// ||f - L phi|| <= tol ||beta0 S||.  The stopping tolerance on ||r||/||f|| becomes
// tol * min(1, ||beta0 S|| / ||f||); solve_core computes the same value on the host.
__global__ void k_constraint_tol(DevScalars* d)
{
    if (d->fnorm2 > 0.0 && d->src2 > 0.0) {
        const double c = d->tol * sqrt(d->src2 / d->fnorm2);
        if (c < d->tol) d->tol = c;
    }
}

// dir 0: dst <- rhs_in; 1: dst <- phi_io; 2: phi_io <- dst.  No-op when aliased.
__global__ void k_copy_io(double* __restrict__ dst, const DevScalars* __restrict__ d, size_t n, int dir)
{
    const double* src = dir == 0 ? d->rhs_in : (dir == 1 ? d->phi_io : dst);
    double* out = dir == 2 ? d->phi_io : dst;
    if (src == out) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        out[t] = src[t];
}

__global__ void k_zero_if_f0(double* __restrict__ phi, size_t n, const DevScalars* __restrict__ d)
{
    if (d->fnorm2 != 0.0) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        phi[t] = 0.0;
}

// Convergence decision after a residual (first: the initial one).  Mirrors the
// host loop of solve_core.
__device__ unsigned check_state(DevScalars* d, int first)
{
    const double fn2 = d->fnorm2;
    unsigned cont = 0;
    if (fn2 == 0.0) {
        d->rel = 0.0;
        if (first) d->iters = 0;
        d->status = MG_OK;
    } else {
        const double rel = sqrt(d->rnorm2);
        d->rel = rel;
        int st = MG_OK, stop = 0;
        if (first) {
            d->iters = 0;
            d->rel0 = rel;
            d->best = rel;
            d->stall = 0;
        } else {
            d->iters += 1;
            const double r0 = d->rel0 > 1.0 ? d->rel0 : 1.0;
            if (!isfinite(rel) || rel > 1e6 * r0) { st = MG_ERR_DIVERGED; stop = 1; }
            else if (rel < 0.9 * d->best) { d->best = rel; d->stall = 0; }
            else if (++d->stall >= 4) { st = rel <= d->tol ? MG_OK : MG_ERR_NOT_CONVERGED; stop = 1; }
            if (!stop && rel < d->best) d->best = rel;
        }
        if (!stop && rel > d->tol && d->iters >= d->maxit) { st = MG_ERR_NOT_CONVERGED; stop = 1; }
        d->status = st;
        cont = (!stop && rel > d->tol) ? 1u : 0u;
        const int m = next_cycles(first != 0, d->ncyc, d->prev_rel, rel, d->tol);
        if (first) d->n_extra = 0;
        d->ncyc = m;
        d->prev_rel = rel;
    }
    return cont;
}

__global__ void k_check(DevScalars* d, cudaGraphConditionalHandle c, int first)
{
    if (threadIdx.x != 0) return;
    cudaGraphSetConditional(c, check_state(d, first));
}

// the IF node of V-cycle k + 1 (k >= 1) of a refinement step
__global__ void k_set_cycle(DevScalars* d, cudaGraphConditionalHandle c, int k)
{
    if (threadIdx.x != 0) return;
    const bool run = d->ncyc > k;
    if (run) d->n_extra += 1;
    cudaGraphSetConditional(c, run ? 1u : 0u);
}

// Launches of a batched graph that run a data-dependent number of times.
struct BatchCounters {
    int loops;                 // iterations of the WHILE body
    int ifruns[kMaxInner];     // runs of the IF node of V-cycle v + 1 of a step (v >= 1)
    int any;                   // the last check's decision (host-driven loop)
};

// The convergence decisions of a batched solve loop: each solve's check as
// k_check, for the solves still iterating (all of them after the initial
// residual); run[s] keeps whether solve s iterates again, and the WHILE
// condition is set while any does.
__global__ void k_batch_check(DevScalars* const* ds, int* run, int count, cudaGraphConditionalHandle c, int first,
                              BatchCounters* ctr, int use_cond)
{
    int any = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x)
        if (first || run[i]) {
            const unsigned cont = check_state(ds[i], first);
            run[i] = cont ? 1 : 0;
            any |= run[i];
        }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        if (first) {
            ctr->loops = 0;
            for (int v = 0; v < kMaxInner; ++v) ctr->ifruns[v] = 0;
        } else {
            ctr->loops += 1;
        }
        ctr->any = any;
        if (use_cond) cudaGraphSetConditional(c, any ? 1u : 0u);
    }
}

// The run flags of V-cycle v + 1 (v >= 1) of a refinement step: the solves
// still iterating whose step takes more than v V-cycles (k_set_cycle's test);
// the IF condition is set when any does.
__global__ void k_batch_gate(DevScalars* const* ds, const int* run0, int* runv, int count,
                             cudaGraphConditionalHandle c, int v, BatchCounters* ctr, int use_cond)
{
    int any = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        DevScalars* d = ds[i];
        const int r = run0[i] && d->ncyc > v;
        if (r) d->n_extra += 1;
        runv[i] = r;
        any |= r;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        if (any) ctr->ifruns[v] += 1;
        if (use_cond) cudaGraphSetConditional(c, any ? 1u : 0u);
    }
}

// One refinement iteration (mixed) or V-cycle (FP64) on phi, then the residual.
mg_status capture_deps(cudaStream_t s, cudaGraph_t* g, std::vector<cudaGraphNode_t>& deps);

// One refinement step inside the graph's WHILE body (h->stream is capturing).
// With automatic inner cycles, V-cycles 2 .. kMaxInner of the step sit in IF
// nodes whose conditions k_set_cycle takes from the scalar block (set by
// k_check); the launches of one such V-cycle are counted into if_launches,
// those of all of them into if_total.
mg_status iterate_once(mg_handle* h, double* phi, float* r32, cudaStream_t if_stream, long long& if_launches,
                       long long& if_total)
{
    const bool nodal = h->loc == MG_LOC_NODAL;
    if_launches = if_total = 0;
    if (h->prec == MG_PREC_MIXED && adaptive_cycles(h)) {
        cudaStream_t s = h->stream;
        float* e = h->lev[0].x32;
        if (nodal) vcycle_node<float>(h, e, h->lev[0].b32, true);
        else vcycle_cell<float>(h, e, h->lev[0].b32, true);
        for (int k = 1; k < kMaxInner; ++k) {
            cudaGraph_t g;
            std::vector<cudaGraphNode_t> deps;
            mg_status rc = capture_deps(s, &g, deps);
            if (rc != MG_OK) return rc;
            cudaGraphConditionalHandle ifh;
            MG_CK(cudaGraphConditionalHandleCreate(&ifh, g, 0, 0));
            MGP_LAUNCH(k_set_cycle<<<1, 32, 0, s>>>(h->d, ifh, k));
            rc = capture_deps(s, &g, deps);
            if (rc != MG_OK) return rc;
            cudaGraphNodeParams prm = {};
            prm.type = cudaGraphNodeTypeConditional;
            prm.conditional.handle = ifh;
            prm.conditional.type = cudaGraphCondTypeIf;
            prm.conditional.size = 1;
            cudaGraphNode_t ifnode;
            MG_CK(cudaGraphAddNode(&ifnode, g, deps.data(), nullptr, deps.size(), &prm));
            MG_CK(cudaStreamUpdateCaptureDependencies(s, &ifnode, nullptr, 1, cudaStreamSetCaptureDependencies));
            cudaGraph_t ifg = prm.conditional.phGraph_out[0];
            MG_CK(cudaStreamBeginCaptureToGraph(if_stream, ifg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            const long long c0 = launch_count();
            h->stream = if_stream;
            if (nodal) vcycle_node<float>(h, e, h->lev[0].b32, false);
            else vcycle_cell<float>(h, e, h->lev[0].b32, false);
            h->stream = s;
            if_launches = launch_count() - c0;   // the same V-cycle in every IF node
            if_total += if_launches;
            MG_CK(cudaStreamEndCapture(if_stream, &ifg));
        }
        vec_axpy_f32(phi, e, &h->d->fscale, h->lev[0].nvec, s);
        residual64(h, phi, r32);
        return MG_OK;
    }
    if (h->prec == MG_PREC_MIXED) {
        mixed_correction(h, phi, inner_cycles(h));
    } else {
        if (nodal) vcycle_node<double>(h, phi, h->f64, false);
        else vcycle_cell<double>(h, phi, h->f64, false);
    }
    residual64(h, phi, r32);
    return MG_OK;
}

mg_status capture_deps(cudaStream_t s, cudaGraph_t* g, std::vector<cudaGraphNode_t>& deps)
{
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    MG_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, g, &d, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(MG_ERR_CUDA, "stream is not capturing");
    deps.assign(d, d + nd);
    return MG_OK;
}

// The part of a captured solve before its iteration loop: rhs staging (from
// the caller's rhs when rhs_from_io) and the initial residual.
void capture_prologue(mg_handle* h, bool rhs_from_io)
{
    cudaStream_t s = h->stream;
    const size_t n = h->lev[0].nvec;
    const bool nodal = h->loc == MG_LOC_NODAL;
    double* phi = h->phi_int;
    float* r32 = h->prec == MG_PREC_MIXED ? h->lev[0].b32 : nullptr;
    if (rhs_from_io) {
        MGP_LAUNCH(k_copy_io<<<kRedBlocks, kThreads, 0, s>>>(h->f64, h->d, n, 0));
        if (nodal) node_zero_dirichlet<double>(h->dim, nview<double>(h, 0), h->f64, s);
        vec_sum_sq(h->f64, n, h->partials, s);
        reduce_finalize(h->partials, 2, h->d->red, s);
        finish_rhs(h, 1, -1);
    }
    if (zero_guess(h)) {
        init_zero_guess(h, phi, r32);
    } else {
        MGP_LAUNCH(k_copy_io<<<kRedBlocks, kThreads, 0, s>>>(phi, h->d, n, 1));
        if (nodal) node_zero_dirichlet<double>(h->dim, nview<double>(h, 0), phi, s);
        residual64(h, phi, r32);
    }
}

// The part after the loop: gauge, copy-out of phi, scalar block to the host.
mg_status capture_epilogue(mg_handle* h)
{
    cudaStream_t s = h->stream;
    const size_t n = h->lev[0].nvec;
    double* phi = h->phi_int;
    if (h->singular) gauge(h, phi);
    MGP_LAUNCH(k_zero_if_f0<<<kRedBlocks, kThreads, 0, s>>>(phi, n, h->d));
    MGP_LAUNCH(k_copy_io<<<kRedBlocks, kThreads, 0, s>>>(phi, h->d, n, 2));
    put_host(h->hs_dev, h->d, sizeof(DevScalars), s);
    return MG_OK;
}

// Enqueue one whole solve of L phi_int = f64 on h->stream, which is capturing.
mg_status capture_solve(mg_handle* h, bool rhs_from_io, cudaStream_t body_stream, cudaStream_t if_stream,
                        long long& fixed, long long& body, long long& if_body)
{
    cudaStream_t s = h->stream;
    double* phi = h->phi_int;
    float* r32 = h->prec == MG_PREC_MIXED ? h->lev[0].b32 : nullptr;
    const long long c0 = launch_count();
    capture_prologue(h, rhs_from_io);
    cudaGraph_t g;
    std::vector<cudaGraphNode_t> deps;
    mg_status rc = capture_deps(s, &g, deps);
    if (rc != MG_OK) return rc;
    cudaGraphConditionalHandle cond;
    MG_CK(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    MGP_LAUNCH(k_check<<<1, 32, 0, s>>>(h->d, cond, 1));
    rc = capture_deps(s, &g, deps);
    if (rc != MG_OK) return rc;
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = cond;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t wnode;
    MG_CK(cudaGraphAddNode(&wnode, g, deps.data(), nullptr, deps.size(), &prm));
    MG_CK(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    const long long c1 = launch_count();
    cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
    MG_CK(cudaStreamBeginCaptureToGraph(body_stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    h->stream = body_stream;
    long long if_total = 0;
    rc = iterate_once(h, phi, r32, if_stream, if_body, if_total);
    if (rc != MG_OK) { h->stream = s; cudaStreamEndCapture(body_stream, &bodyg); return rc; }
    MGP_LAUNCH(k_check<<<1, 32, 0, body_stream>>>(h->d, cond, 0));
    h->stream = s;
    MG_CK(cudaStreamEndCapture(body_stream, &bodyg));
    const long long c2 = launch_count();
    rc = capture_epilogue(h);
    if (rc != MG_OK) return rc;
    const long long c3 = launch_count();
    fixed = (c1 - c0) + (c3 - c2);
    body = (c2 - c1) - if_total;
    MG_CK(cudaGetLastError());
    return MG_OK;
}

struct CaptureStreams {
    cudaStream_t main = nullptr, body = nullptr, inner = nullptr;
    ~CaptureStreams()
    {
        if (main) cudaStreamDestroy(main);
        if (body) cudaStreamDestroy(body);
        if (inner) cudaStreamDestroy(inner);
    }
    mg_status make()
    {
        MG_CK(cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking));
        MG_CK(cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking));
        MG_CK(cudaStreamCreateWithFlags(&inner, cudaStreamNonBlocking));
        return MG_OK;
    }
};

// Capture the handles' solves as independent branches of one graph.
mg_status build_graph(mg_handle* const* hs, int count, bool rhs_from_io, cudaGraphExec_t* exec,
                      std::vector<long long>& fixed, std::vector<long long>& body, std::vector<long long>& ifb)
{
    CaptureStreams cs;
    mg_status rc = cs.make();
    if (rc != MG_OK) return rc;
    fixed.assign(count, 0);
    body.assign(count, 0);
    ifb.assign(count, 0);
    const long long cap0 = launch_count();
    MG_CK(cudaStreamBeginCapture(cs.main, cudaStreamCaptureModeRelaxed));
    std::vector<cudaGraphNode_t> join;
    for (int i = 0; i < count && rc == MG_OK; ++i) {
        // every branch starts from the (empty) root of the graph
        cudaStreamUpdateCaptureDependencies(cs.main, nullptr, nullptr, 0, cudaStreamSetCaptureDependencies);
        cudaStream_t saved = hs[i]->stream;
        hs[i]->stream = cs.main;
        rc = capture_solve(hs[i], rhs_from_io, cs.body, cs.inner, fixed[i], body[i], ifb[i]);
        hs[i]->stream = saved;
        cudaGraph_t g;
        std::vector<cudaGraphNode_t> sinks;
        if (rc == MG_OK) rc = capture_deps(cs.main, &g, sinks);
        join.insert(join.end(), sinks.begin(), sinks.end());
    }
    if (rc == MG_OK)
        cudaStreamUpdateCaptureDependencies(cs.main, join.data(), nullptr, join.size(), cudaStreamSetCaptureDependencies);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs.main, &graph);
    add_launches(-(launch_count() - cap0));  // capture enqueues nothing; replays are counted after each run
    if (rc != MG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return MG_OK;
}

bool use_graph(const mg_handle* h) { return !(h->opt.flags & MG_FLAG_NO_GRAPH) && !prof().on; }

mg_status ensure_graph(mg_handle* h, int which)
{
    if (h->gx[which]) return MG_OK;
    std::vector<long long> f, b, fi;
    mg_status rc = build_graph(&h, 1, which == 0, &h->gx[which], f, b, fi);
    if (rc != MG_OK) return rc;
    h->g_fixed[which] = f[0];
    h->g_body[which] = b[0];
    h->g_if[which] = fi[0];
    return MG_OK;
}

// Result of a finished graph solve (the scalar block is in h->hs).
mg_status graph_result(mg_handle* h, long long fixed, long long body, long long ifb, mg_stats* st)
{
    const DevScalars& r = *h->hs;
    add_launches(fixed + body * r.iters + ifb * r.n_extra);
    if (r.async_err) return fail(MG_ERR_CUDA, "a bounded wait inside a kernel (an asynchronous copy or a pipelined pass) gave up");
    if (r.info != 0) return fail(MG_ERR_UNSUPPORTED, "the coarsest-level operator is singular");
    if (st) {
        st->iters = r.iters;
        st->rel_resid = r.rel;
        st->rhs_norm = sqrt(r.fnorm2);
        st->vcycles = h->prec == MG_PREC_MIXED
                          ? (adaptive_cycles(h) ? r.iters + r.n_extra : r.iters * inner_cycles(h))
                          : r.iters;
    }
    if (r.status != MG_OK) {
        char buf[160];
        snprintf(buf, sizeof buf, "stopped after %d iterations at relative residual %.3e (tol %.3e)", r.iters, r.rel,
                 r.tol);
        g_last_error = buf;
    }
    return (mg_status)r.status;
}

// ------------------------------------------------ batched (lockstep) solve loops
//
// When every solve of a batch is a 3-D mixed-precision cell solve whose
// levels the batched kernels take, the batch graph shares one iteration loop:
// each solve's rhs staging and initial residual (its own branch), then one
// WHILE node whose body runs V-cycle 1 of a refinement step for every solve
// still iterating, V-cycles 2 .. kMaxInner in IF nodes, the FP64 updates,
// residuals and norms, and the checks -- one launch per step for all solves
// (mg_batch.cu and the batched launchers) -- then each solve's copy-out.  The
// V-cycles run the solves' levels in lockstep from the finest: step l holds
// level l of every solve with more launched levels than l; the levels of at
// most kBatchCoarseCells cells run in the solves' coarse ends, one CTA per
// solve in one launch.  Each solve's decisions are k_check's on its own
// scalar block, so it iterates exactly as alone, and its arithmetic is that
// of the single-solve kernels: the results equal the solves run alone.

// first level of a handle's batched coarse end
int batch_coarse_start(const mg_handle* h)
{
    const int L = h->nlev;
    int l = 1;
    while (l < L - 1 && (h->lev[l].ncell > kBatchCoarseCells || L - l > kCoarseMaxLevels)) ++l;
    return l;
}

bool batch_kernels_ok(const mg_handle* h)
{
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    auto a8 = [](const void* p) { return ((uintptr_t)p & 7) == 0; };
    if (h->loc != MG_LOC_CELL || h->dim != 3 || h->prec != MG_PREC_MIXED || !adaptive_cycles(h)) return false;
    if (h->opt.interp_order != 1 || h->opt.nu1 < 1 || h->opt.nu2 < 0 || h->nlev < 2) return false;
    if (h->opt.flags & (MG_FLAG_NO_FUSED | MG_FLAG_BATCH_BRANCHES)) return false;
    if (h->Nd > kMaxDense || h->lev[0].nvec % 4 != 0 || !a16(h->phi_int)) return false;
    if (!cell_resid64_batch_ok(cview<double>(h, 0), h->phi_int, h->f64, h->lev[0].b32)) return false;
    const int lc = batch_coarse_start(h);
    if (h->nlev - lc > kCoarseMaxLevels) return false;
    for (int l = 0; l < lc; ++l) {
        const CellLevel<float> V = cview<float>(h, l);
        float* x = h->lev[l].x32;
        const float* b = h->lev[l].b32;
        if (V.nx % 4 != 0 || V.nx < 8 || V.ny % 2 != 0 || V.nz % 2 != 0 || V.invd) return false;
        if (!a16(x) || !a16(b) || !a16(V.by) || !a16(V.bz)) return false;
        if (!a8(h->lev[l + 1].b32) || !a8(h->lev[l + 1].x32)) return false;
    }
    return true;
}

// Whether the solves of hs share one batched loop (graph or host-driven).
bool batch_eligible(mg_handle* const* hs, int count)
{
    if (count < 2) return false;
    for (int i = 0; i < count; ++i)
        if (!batch_kernels_ok(hs[i]) || hs[i]->opt.nu1 != hs[0]->opt.nu1 || hs[i]->opt.nu2 != hs[0]->opt.nu2)
            return false;
    return true;
}

// The device tables of a batched loop (one allocation) and its launch shapes.
struct BatchPlan {
    struct Step {
        std::vector<BatchLaunch> launches;   // the step's items, at most kBatchLaunchItems per launch
        double cells = 0.0;                  // fine cells of the step's items (profiling bytes)
        void add(const BatchItem& it)
        {
            if (launches.empty() || launches.back().nitems == kBatchLaunchItems) {
                launches.emplace_back();
                launches.back().nitems = 0;
                launches.back().tiles = 0;
            }
            BatchLaunch& B = launches.back();
            B.items[B.nitems] = it;
            B.items[B.nitems].tile0 = B.tiles;
            B.tiles += (it.units + kBatchTile - 1) / kBatchTile;
            B.nitems += 1;
        }
    };
    int count = 0, nsteps = 0, nu1 = 0, nu2 = 0;
    std::vector<mg_handle*> hs;       // the group's handles (its solves 0 .. count - 1)
    long long body = 0, ifb = 0;      // launches per loop iteration (outside the IF nodes) and per IF run
    double cells0 = 0.0;              // cells of the solves' finest levels
    char* dmem = nullptr;
    int* run = nullptr;               // [kMaxInner][count]
    DevScalars** ds = nullptr;        // [count]
    BatchCounters* ctr = nullptr;     // device counters
    BatchCounters* hctr = nullptr;    // pinned host copy, written at the end of each run
    BatchCounters* hctr_dev = nullptr;   // its device address
    Step smooth[kMaxLevels], restr[kMaxLevels], prolong[kMaxLevels];
    CoarseArgs<float>* coarse = nullptr;
    Resid64Item* resid = nullptr;
    int* resid_bmap = nullptr;        // item of every block of the batched residual
    int resid_blocks = 0;
    FinalItem* fin = nullptr;
    AxpyItem* axpy = nullptr;
    int axpy_tiles = 0, axpy_grid = 0;
    ~BatchPlan()
    {
        if (dmem) cudaFree(dmem);
        if (hctr) cudaFreeHost(hctr);
    }
};

// Lay out and upload the tables of a batched loop over hs[0..count).
mg_status make_batch_plan(mg_handle* const* hs, int count, BatchPlan& P)
{
    P.count = count;
    P.hs.assign(hs, hs + count);
    P.nu1 = hs[0]->opt.nu1;
    P.nu2 = hs[0]->opt.nu2;
    std::vector<int> lc(count);
    for (int i = 0; i < count; ++i) {
        lc[i] = batch_coarse_start(hs[i]);
        P.nsteps = std::max(P.nsteps, lc[i]);
    }
    for (int l = 0; l < P.nsteps; ++l) {
        for (int i = 0; i < count; ++i) {
            if (l >= lc[i]) continue;
            mg_handle* h = hs[i];
            BatchItem it{};
            it.F = cview<float>(h, l);
            it.C = cview<float>(h, l + 1);
            it.x = h->lev[l].x32;
            it.b = h->lev[l].b32;
            it.bc = h->lev[l + 1].b32;
            it.xc = h->lev[l + 1].x32;
            it.solve = i;
            const int nq = it.F.nx / 4;
            batch_magic(nq, &it.mq, &it.sq);
            batch_magic(it.F.ny, &it.my, &it.sy);
            it.units = nq * it.F.ny * it.F.nz;
            P.smooth[l].cells += 4.0 * it.units;
            P.smooth[l].add(it);
            P.prolong[l].add(it);
            it.units = nq * (it.F.ny / 2) * (it.F.nz / 2);
            batch_magic(it.F.ny / 2, &it.my, &it.sy);
            P.restr[l].add(it);
        }
        P.prolong[l].cells = P.restr[l].cells = P.smooth[l].cells;
    }
    std::vector<CoarseArgs<float>> co(count);
    std::vector<Resid64Item> rs(count);
    std::vector<FinalItem> fi(count);
    std::vector<AxpyItem> ax(count);
    std::vector<DevScalars*> ds(count);
    int at = 0;
    std::vector<int> bmap;
    for (int i = 0; i < count; ++i) {
        mg_handle* h = hs[i];
        CoarseArgs<float>& A = co[i];
        memset(&A, 0, sizeof A);
        A.nlev = h->nlev - lc[i];
        for (int l = lc[i]; l < h->nlev; ++l) {
            A.L[l - lc[i]] = cview<float>(h, l);
            A.x[l - lc[i]] = h->lev[l].x32;
            A.b[l - lc[i]] = h->lev[l].b32;
        }
        A.Minv = h->Minv;
        A.Nd = h->Nd;
        A.nu1 = h->opt.nu1;
        A.nu2 = h->opt.nu2;
        A.order = h->opt.interp_order;
        A.zero_first = 1;
        const long long quads = (long long)(h->lev[0].nvec / 4);
        const int nvb = (int)std::min<long long>(kRedBlocks, (quads + kThreads - 1) / kThreads);
        rs[i] = Resid64Item{cview<double>(h, 0), h->phi_int, h->f64, h->lev[0].b32, &h->d->fscale, h->partials,
                            i, (int)bmap.size(), nvb, 0};
        bmap.resize(bmap.size() + nvb, i);
        fi[i] = FinalItem{h->partials, &h->d->rnorm2, &h->d->rscale2, i, 0};
        const int n4 = (int)(h->lev[0].nvec / 4);
        ax[i] = AxpyItem{h->phi_int, h->lev[0].x32, &h->d->fscale, i, at, n4, 0};
        at += (n4 + kThreads - 1) / kThreads;
        ds[i] = h->d;
        P.cells0 += (double)h->lev[0].ncell;
    }
    P.axpy_tiles = at;
    P.axpy_grid = axpy_batch_grid(at);
    P.resid_blocks = (int)bmap.size();
    // one allocation, 256-byte aligned tables
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t o_run = take(sizeof(int) * kMaxInner * count), o_ds = take(sizeof(DevScalars*) * count),
                 o_ctr = take(sizeof(BatchCounters)), o_co = take(sizeof(CoarseArgs<float>) * count),
                 o_rs = take(sizeof(Resid64Item) * count), o_fi = take(sizeof(FinalItem) * count),
                 o_ax = take(sizeof(AxpyItem) * count), o_bm = take(sizeof(int) * bmap.size());
    MG_CK(cudaMalloc(&P.dmem, off));
    MG_CK(cudaHostAlloc(&P.hctr, sizeof(BatchCounters), cudaHostAllocMapped));
    MG_CK(cudaHostGetDevicePointer((void**)&P.hctr_dev, P.hctr, 0));
    memset(P.hctr, 0, sizeof(BatchCounters));
    std::vector<char> host(off, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) { if (bytes) memcpy(host.data() + o, src, bytes); };
    put(o_ds, ds.data(), sizeof(DevScalars*) * count);
    put(o_co, co.data(), sizeof(CoarseArgs<float>) * count);
    put(o_rs, rs.data(), sizeof(Resid64Item) * count);
    put(o_fi, fi.data(), sizeof(FinalItem) * count);
    put(o_ax, ax.data(), sizeof(AxpyItem) * count);
    put(o_bm, bmap.data(), sizeof(int) * bmap.size());
    MG_CK(cudaMemcpy(P.dmem, host.data(), off, cudaMemcpyHostToDevice));
    P.run = reinterpret_cast<int*>(P.dmem + o_run);
    P.ds = reinterpret_cast<DevScalars**>(P.dmem + o_ds);
    P.ctr = reinterpret_cast<BatchCounters*>(P.dmem + o_ctr);
    P.coarse = reinterpret_cast<CoarseArgs<float>*>(P.dmem + o_co);
    P.resid = reinterpret_cast<Resid64Item*>(P.dmem + o_rs);
    P.fin = reinterpret_cast<FinalItem*>(P.dmem + o_fi);
    P.axpy = reinterpret_cast<AxpyItem*>(P.dmem + o_ax);
    P.resid_bmap = reinterpret_cast<int*>(P.dmem + o_bm);
    return MG_OK;
}

// V-cycle v + 1 of a refinement step for every solve whose run flag for it is
// set, in lockstep from the finest level (level 0 from zero when v == 0; the
// other levels always from zero, which the first colour pass of each level
// takes without loading x).
void batch_vcycle(const BatchPlan& P, int v, cudaStream_t s)
{
    const int* run = P.run + (size_t)v * P.count;
    auto pass = [&](const BatchPlan::Step& st, int op, int color, int zx) {
        if (st.launches.empty()) return;
        // algorithmic words per fine cell (as the single-solve classes)
        const double w = op == BATCH_GSRB ? 2.0 : op == BATCH_RESTRICT ? 3.125 : 2.125;
        const int id = op == BATCH_GSRB ? (&st == &P.smooth[0] ? MG_PROF_BATCH_SMOOTH : MG_PROF_BATCH_SMOOTH_COARSE)
                                        : op == BATCH_RESTRICT ? MG_PROF_BATCH_RESTRICT : MG_PROF_BATCH_PROLONG;
        const int pr = prof_begin(id, w * sizeof(float) * st.cells, s);
        for (const BatchLaunch& B : st.launches) batch_level(op, B, run, color, zx, s);
        prof_end(pr, s);
    };
    for (int l = 0; l < P.nsteps; ++l) {
        for (int k = 0; k < P.nu1; ++k)
            for (int color = 0; color < 2; ++color)
                pass(P.smooth[l], BATCH_GSRB, color, k == 0 && color == 0 && (l > 0 || v == 0));
        pass(P.restr[l], BATCH_RESTRICT, 0, 0);
    }
    const int pc = prof_begin(MG_PROF_BATCH_COARSE, 0.0, s);
    coarse_cycle_batch(P.coarse, P.count, run, s);
    prof_end(pc, s);
    for (int l = P.nsteps - 1; l >= 0; --l) {
        pass(P.prolong[l], BATCH_PROLONG, 0, 0);
        for (int k = 0; k < P.nu2; ++k)
            for (int color = 0; color < 2; ++color) pass(P.smooth[l], BATCH_GSRB, color, 0);
    }
}

// The FP64 refinement update, residuals and norms of a batched loop.
void batch_update(const BatchPlan& P, cudaStream_t s)
{
    axpy_f32_batch(P.axpy, P.count, P.axpy_tiles, P.run, P.axpy_grid, s);
    const int pr = prof_begin(MG_PROF_BATCH_RESID64, (24.0 + 4.0) * P.cells0, s, kCellResidFlops * P.cells0);
    cell_resid64_batch(P.resid, P.resid_bmap, P.resid_blocks, P.run, s);
    reduce_finalize_batch(P.fin, P.count, P.run, s);
    prof_end(pr, s);
}

// Capture a batched graph (see above) with one lockstep loop per group of
// solves, the groups as concurrent branches: while one group runs its FP64
// residuals or its latency-bound small levels, another streams its finest
// levels.  fixed: launches that run once per graph launch; each plan's body
// and ifb: per iteration of its loop and per run of one of its IF nodes.
mg_status build_batched_graph(std::vector<std::unique_ptr<BatchPlan>>& plans, mg_handle* const* branch,
                              int nbranch, bool rhs_from_io, cudaGraphExec_t* exec, long long& fixed,
                              long long* bfixed, long long* bbody, long long* bifb)
{
    CaptureStreams cs;
    mg_status rc = cs.make();
    if (rc != MG_OK) return rc;
    const long long c0 = launch_count();
    long long loops = 0;   // launches inside the loops and the branches (not fixed)
    MG_CK(cudaStreamBeginCapture(cs.main, cudaStreamCaptureModeRelaxed));
    std::vector<cudaGraphNode_t> sinks, all;
    cudaGraph_t g = nullptr;
    for (size_t gi = 0; gi < plans.size() && rc == MG_OK; ++gi) {
        BatchPlan& P = *plans[gi];
        const int count = P.count;
        std::vector<cudaGraphNode_t> join;
        for (int i = 0; i < count && rc == MG_OK; ++i) {
            cudaStreamUpdateCaptureDependencies(cs.main, nullptr, nullptr, 0, cudaStreamSetCaptureDependencies);
            cudaStream_t saved = P.hs[i]->stream;
            P.hs[i]->stream = cs.main;
            capture_prologue(P.hs[i], rhs_from_io);
            P.hs[i]->stream = saved;
            rc = capture_deps(cs.main, &g, sinks);
            join.insert(join.end(), sinks.begin(), sinks.end());
        }
        cudaGraphConditionalHandle cond{};
        cudaGraphNode_t wnode{};
        if (rc == MG_OK) {
            cudaStreamUpdateCaptureDependencies(cs.main, join.data(), nullptr, join.size(),
                                                cudaStreamSetCaptureDependencies);
            rc = capture_deps(cs.main, &g, sinks);
        }
        if (rc == MG_OK && cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
            rc = fail(MG_ERR_CUDA, "cudaGraphConditionalHandleCreate");
        if (rc == MG_OK) {
            MGP_LAUNCH(k_batch_check<<<1, kThreads, 0, cs.main>>>(P.ds, P.run, count, cond, 1, P.ctr, 1));
            rc = capture_deps(cs.main, &g, sinks);
        }
        cudaGraphNodeParams prm = {};
        if (rc == MG_OK) {
            prm.type = cudaGraphNodeTypeConditional;
            prm.conditional.handle = cond;
            prm.conditional.type = cudaGraphCondTypeWhile;
            prm.conditional.size = 1;
            if (cudaGraphAddNode(&wnode, g, sinks.data(), nullptr, sinks.size(), &prm) != cudaSuccess ||
                cudaStreamUpdateCaptureDependencies(cs.main, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
                    cudaSuccess)
                rc = fail(MG_ERR_CUDA, "adding the batched WHILE node");
        }
        if (rc == MG_OK) {
            const long long c1 = launch_count();
            long long if_total = 0;
            cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
            cudaStream_t b = cs.body;
            if (cudaStreamBeginCaptureToGraph(b, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
                cudaSuccess)
                rc = fail(MG_ERR_CUDA, "capturing the batched loop body");
            if (rc == MG_OK) {
                batch_vcycle(P, 0, b);
                for (int v = 1; v < kMaxInner && rc == MG_OK; ++v) {
                    cudaGraph_t bg;
                    std::vector<cudaGraphNode_t> deps;
                    rc = capture_deps(b, &bg, deps);
                    cudaGraphConditionalHandle ifh{};
                    if (rc == MG_OK && cudaGraphConditionalHandleCreate(&ifh, bg, 0, 0) != cudaSuccess)
                        rc = fail(MG_ERR_CUDA, "cudaGraphConditionalHandleCreate");
                    if (rc != MG_OK) break;
                    MGP_LAUNCH(k_batch_gate<<<1, kThreads, 0, b>>>(P.ds, P.run, P.run + (size_t)v * count, count, ifh,
                                                                   v, P.ctr, 1));
                    rc = capture_deps(b, &bg, deps);
                    if (rc != MG_OK) break;
                    cudaGraphNodeParams ip = {};
                    ip.type = cudaGraphNodeTypeConditional;
                    ip.conditional.handle = ifh;
                    ip.conditional.type = cudaGraphCondTypeIf;
                    ip.conditional.size = 1;
                    cudaGraphNode_t ifnode;
                    if (cudaGraphAddNode(&ifnode, bg, deps.data(), nullptr, deps.size(), &ip) != cudaSuccess ||
                        cudaStreamUpdateCaptureDependencies(b, &ifnode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
                            cudaSuccess) {
                        rc = fail(MG_ERR_CUDA, "adding a batched IF node");
                        break;
                    }
                    cudaGraph_t ifg = ip.conditional.phGraph_out[0];
                    if (cudaStreamBeginCaptureToGraph(cs.inner, ifg, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                        rc = fail(MG_ERR_CUDA, "capturing a batched IF body");
                        break;
                    }
                    const long long i0 = launch_count();
                    batch_vcycle(P, v, cs.inner);
                    P.ifb = launch_count() - i0;
                    if_total += P.ifb;
                    if (cudaStreamEndCapture(cs.inner, &ifg) != cudaSuccess) rc = fail(MG_ERR_CUDA, "end of IF capture");
                }
                if (rc == MG_OK) {
                    batch_update(P, b);
                    MGP_LAUNCH(k_batch_check<<<1, kThreads, 0, b>>>(P.ds, P.run, count, cond, 0, P.ctr, 1));
                }
                cudaGraph_t tmp = bodyg;
                if (cudaStreamEndCapture(b, &tmp) != cudaSuccess && rc == MG_OK)
                    rc = fail(MG_ERR_CUDA, "end of body capture");
            }
            const long long c2 = launch_count();
            P.body = (c2 - c1) - if_total;
            loops += c2 - c1;
        }
        for (int i = 0; i < count && rc == MG_OK; ++i) {
            cudaStreamUpdateCaptureDependencies(cs.main, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            cudaStream_t saved = P.hs[i]->stream;
            P.hs[i]->stream = cs.main;
            rc = capture_epilogue(P.hs[i]);
            P.hs[i]->stream = saved;
            if (rc == MG_OK) rc = capture_deps(cs.main, &g, sinks);
            all.insert(all.end(), sinks.begin(), sinks.end());
        }
    }
    // the solves that run as their own branches (each its own loop, as build_graph)
    for (int i = 0; i < nbranch && rc == MG_OK; ++i) {
        cudaStreamUpdateCaptureDependencies(cs.main, nullptr, nullptr, 0, cudaStreamSetCaptureDependencies);
        const long long b0 = launch_count();
        cudaStream_t saved = branch[i]->stream;
        branch[i]->stream = cs.main;
        rc = capture_solve(branch[i], rhs_from_io, cs.body, cs.inner, bfixed[i], bbody[i], bifb[i]);
        branch[i]->stream = saved;
        loops += launch_count() - b0;
        if (rc == MG_OK) rc = capture_deps(cs.main, &g, sinks);
        all.insert(all.end(), sinks.begin(), sinks.end());
    }
    if (rc == MG_OK) {
        cudaStreamUpdateCaptureDependencies(cs.main, all.data(), nullptr, all.size(), cudaStreamSetCaptureDependencies);
        for (auto& P : plans) put_host(P->hctr_dev, P->ctr, sizeof(BatchCounters), cs.main);
    }
    const long long c3 = launch_count();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs.main, &graph);
    add_launches(-(c3 - c0));   // capture enqueues nothing; replays are counted after each run
    if (rc != MG_OK) { if (graph) cudaGraphDestroy(graph); cudaGetLastError(); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    fixed = (c3 - c0) - loops;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return MG_OK;
}

// The batched loop driven from the host (graphs off, or profiling): the
// launches of the graph's body, with V-cycles 2 .. kMaxInner of a step always
// launched (a solve that does not take one has its run flag clear) and one
// read-back of the check per iteration.  Same decisions, same results.
mg_status batch_host_loop(mg_handle* const* hs, int count, bool rhs_from_io, cudaStream_t s)
{
    BatchPlan P;
    mg_status rc = make_batch_plan(hs, count, P);
    if (rc != MG_OK) return rc;
    for (int i = 0; i < count; ++i) {
        cudaStream_t saved = hs[i]->stream;
        hs[i]->stream = s;
        capture_prologue(hs[i], rhs_from_io);
        hs[i]->stream = saved;
    }
    MGP_LAUNCH(k_batch_check<<<1, kThreads, 0, s>>>(P.ds, P.run, count, 0, 1, P.ctr, 0));
    for (;;) {
        put_host(P.hctr_dev, P.ctr, sizeof(BatchCounters), s);
        MG_CK(cudaStreamSynchronize(s));
        if (!P.hctr->any) break;
        batch_vcycle(P, 0, s);
        for (int v = 1; v < kMaxInner; ++v) {
            MGP_LAUNCH(k_batch_gate<<<1, kThreads, 0, s>>>(P.ds, P.run, P.run + (size_t)v * count, count, 0, v,
                                                           P.ctr, 0));
            batch_vcycle(P, v, s);
        }
        batch_update(P, s);
        MGP_LAUNCH(k_batch_check<<<1, kThreads, 0, s>>>(P.ds, P.run, count, 0, 0, P.ctr, 0));
    }
    for (int i = 0; i < count && rc == MG_OK; ++i) {
        cudaStream_t saved = hs[i]->stream;
        hs[i]->stream = s;
        rc = capture_epilogue(hs[i]);
        hs[i]->stream = saved;
    }
    MG_CK(cudaStreamSynchronize(s));
    return rc;
}

// Solves of at most this many fine cells share the batched loops; larger ones
// run as their own branches of the batch graph.  Measured on one GB300 (64
// solves of 32^3: the loop 2.8x faster than branches; 64^3: 1.35x; 16 of
// 96^3: even; 16 of 128^3: 12 % slower): a large solve keeps its own working
// set in L2 from one pass to the next when it runs as a branch, which a step
// over the finest levels of all solves at once cannot.
constexpr size_t kBatchLockstepCells = (size_t)1 << 18;

// Concurrent batched loops a batch of count solves is split into
// (mg_set_batch_groups; 0: automatic, one loop: measured on one GB300, 64
// solves of 32^3 took 3.1 ms per batch in one loop against 6.3 ms in four,
// and the uneven 64-solve batch 31.0 ms in one against 32.3, 34.0 and 38.7 ms
// in 2, 4 and 8).
std::atomic<int> g_batch_groups{0};
int batch_groups(int)
{
    const int g = g_batch_groups.load(std::memory_order_relaxed);
    return g > 0 ? g : 1;
}

// Batch graphs, cached by the exact ordered list of handles.
struct BatchGraph {
    std::vector<mg_handle*> hs;
    bool rhs_io = true;   // right-hand sides from the callers (solves) or already in f64 (projections)
    int groups = 1;       // concurrent batched loops asked for when the graph was built
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> fixed, body, ifb;
    std::vector<std::unique_ptr<BatchPlan>> plans;   // set when the solves share batched loops
    long long b_fixed = 0;
    // launches of the last run (batched loops), from the device counters
    long long launches() const
    {
        if (plans.empty()) return 0;
        long long n = b_fixed;
        for (const auto& P : plans) {
            n += P->body * P->hctr->loops;
            for (int v = 1; v < kMaxInner; ++v) n += P->ifb * P->hctr->ifruns[v];
        }
        return n;
    }
};

constexpr size_t kMaxBatchGraphs = 64;   // cached batch graphs; the least recently used goes first
std::mutex g_batch_mu;
std::vector<BatchGraph*> g_batches;

void drop_batches_of(mg_handle* h)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batches.size();) {
        BatchGraph* b = g_batches[i];
        bool has = false;
        for (mg_handle* x : b->hs) has = has || x == h;
        if (has) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            delete b;
            g_batches.erase(g_batches.begin() + i);
        } else {
            ++i;
        }
    }
}

// The cached batch graph of this ordered list of handles and mode (built on
// first use); the list keeps the most recently used last and at most
// kMaxBatchGraphs entries.
mg_status batch_graph(mg_handle* const* hs, int count, bool rhs_io, BatchGraph** out)
{
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (size_t i = 0; i < g_batches.size(); ++i) {
            BatchGraph* b = g_batches[i];
            if (b->rhs_io == rhs_io && b->groups == batch_groups(count) && (int)b->hs.size() == count &&
                std::equal(b->hs.begin(), b->hs.end(), hs)) {
                g_batches.erase(g_batches.begin() + i);
                g_batches.push_back(b);
                *out = b;
                return MG_OK;
            }
        }
    }
    std::unique_ptr<BatchGraph> nb(new BatchGraph());
    nb->hs.assign(hs, hs + count);
    nb->rhs_io = rhs_io;
    nb->groups = batch_groups(count);
    // solves of at most kBatchLockstepCells fine cells share batched loops
    // (when at least two do); the others run as their own branches
    std::vector<mg_handle*> lock, branch;
    std::vector<int> branch_at;
    for (int i = 0; i < count; ++i) {
        if (batch_kernels_ok(hs[i]) && hs[i]->lev[0].ncell <= kBatchLockstepCells &&
            hs[i]->opt.nu1 == hs[0]->opt.nu1 && hs[i]->opt.nu2 == hs[0]->opt.nu2) {
            lock.push_back(hs[i]);
        } else {
            branch.push_back(hs[i]);
            branch_at.push_back(i);
        }
    }
    if (lock.size() < 2) {
        lock.clear();
        branch.assign(hs, hs + count);
        branch_at.resize(count);
        for (int i = 0; i < count; ++i) branch_at[i] = i;
    }
    mg_status rc = MG_OK;
    if (!lock.empty()) {
        // groups balanced by cells: the largest solves first, each to the lightest group
        const int nl = (int)lock.size();
        const int G = std::max(1, std::min(batch_groups(nl), nl));
        std::vector<int> order(nl);
        for (int i = 0; i < nl; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return lock[a]->lev[0].ncell > lock[b]->lev[0].ncell; });
        std::vector<std::vector<mg_handle*>> members(G);
        std::vector<double> load(G, 0.0);
        for (int i : order) {
            const int gi = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            members[gi].push_back(lock[i]);
            load[gi] += (double)lock[i]->lev[0].ncell;
        }
        for (int gi = 0; gi < G && rc == MG_OK; ++gi) {
            if (members[gi].empty()) continue;
            nb->plans.emplace_back(new BatchPlan());
            rc = make_batch_plan(members[gi].data(), (int)members[gi].size(), *nb->plans.back());
        }
        const int nbr = (int)branch.size();
        std::vector<long long> bf(nbr, 0), bb(nbr, 0), bi(nbr, 0);
        if (rc == MG_OK)
            rc = build_batched_graph(nb->plans, branch.data(), nbr, rhs_io, &nb->exec, nb->b_fixed, bf.data(),
                                     bb.data(), bi.data());
        if (rc == MG_OK) {
            nb->fixed.assign(count, 0);
            nb->body.assign(count, 0);
            nb->ifb.assign(count, 0);
            for (int k = 0; k < nbr; ++k) {
                nb->fixed[branch_at[k]] = bf[k];
                nb->body[branch_at[k]] = bb[k];
                nb->ifb[branch_at[k]] = bi[k];
            }
        }
    } else {
        rc = build_graph(hs, count, rhs_io, &nb->exec, nb->fixed, nb->body, nb->ifb);
    }
    if (rc != MG_OK) return rc;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    // evict from the least recently used end, skipping graphs whose handles are
    // in use (their caller may be launching the graph right now)
    for (size_t i = 0; g_batches.size() >= kMaxBatchGraphs && i < g_batches.size();) {
        BatchGraph* old = g_batches[i];
        bool busy = false;
        for (mg_handle* x : old->hs) busy = busy || x->busy.load() != 0;
        if (busy) {
            ++i;
            continue;
        }
        if (old->exec) cudaGraphExecDestroy(old->exec);
        delete old;
        g_batches.erase(g_batches.begin() + i);
    }
    *out = nb.release();
    g_batches.push_back(*out);
    return MG_OK;
}

struct BusyGuard {
    mg_handle* h;
    bool ok;
    explicit BusyGuard(mg_handle* hh) : h(hh), ok(hh->busy.exchange(1) == 0) {}
    ~BusyGuard()
    {
        if (ok) h->busy.store(0);
    }
};

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---- smoother kernel autotuner (MG_FLAG_AUTOTUNE)
//
// For every FP32 level but the coarsest, the candidate smoother kernels -- the
// four-cell / four-node passes with 8, 16 or 32 quads per block row (for nodes
// also marching four planes per thread), and the
// shared-memory pipelined (cells) or tiled (nodes) kernel where the level
// allows it -- each run two sweeps (the default smoothing count, so that a
// ping-ponging kernel ends in place) on the level's scratch vectors, timed with
// CUDA events on the handle's stream (one untimed call, then the best of
// three), and the fastest is kept in Level::kind.  All candidates compute the
// same arithmetic, so the choice changes no result.  Choices are cached per
// (location, dimension, grid, boundary kinds) for the process: handles of a
// size already seen are not timed again.
struct TuneKey {
    int v[11];
    bool operator<(const TuneKey& o) const { return std::lexicographical_compare(v, v + 11, o.v, o.v + 11); }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

mg_status autotune(mg_handle* h)
{
    if (h->prec != MG_PREC_MIXED || (h->opt.flags & MG_FLAG_NO_FUSED)) return MG_OK;
    cudaStream_t s = h->stream;
    const bool nodal = h->loc == MG_LOC_NODAL;
    cudaEvent_t e0, e1;
    MG_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(MG_ERR_CUDA, "cudaEventCreate"); }
    mg_status rc = MG_OK;
    for (int l = 0; l < h->nlev - 1 && rc == MG_OK; ++l) {
        Level& v = h->lev[l];
        const TuneKey key{{h->loc, h->dim, v.n[0], v.n[1], v.n[2], h->bc.lo[0], h->bc.lo[1], h->bc.lo[2], h->bc.hi[0],
                           h->bc.hi[1], h->bc.hi[2]}};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) { v.kind = it->second; continue; }
        }
        float *x = v.x32, *t = v.t32, *b = v.b32;
        if (!x || !t || !b) continue;
        std::vector<int> cand;
        if (nodal) {
            if (node_v4_ok(h->dim, nview<float>(h, l), x, t, b))
                for (int k = 1; k <= 3; ++k)
                    if ((4 << k) <= v.N[0] / 4) {
                        cand.push_back(k);
                        cand.push_back(k + 4);   // the same shape marching four planes
                        cand.push_back(k + 8);   // and eight
                    }
            if (h->dim == 3 && v.N[0] >= 32 && v.N[1] >= 8) cand.push_back(4);
        } else {
            const CellLevel<float> V = cview<float>(h, l);
            if (cell_gsrb_v4_ok(h->dim, V, x, b))
                for (int k = 1; k <= 3; ++k)
                    if ((4 << k) <= v.n[0] / 4) cand.push_back(k);
            if (cell_gsrb_fused_ok<float>(h->dim, V)) cand.push_back(4);
            if (cell_gsrb_tma_ok(h->dim, V, x, t, b) && cell_gsrb_tma_fits(V.nx)) cand.push_back(8);
        }
        int best = 0;
        if (cand.size() > 1) {
            cudaMemsetAsync(x, 0, v.nvec * sizeof(float), s);
            cudaMemsetAsync(b, 0, v.nvec * sizeof(float), s);
            float best_ms = 1e30f;
            for (int k : cand) {
                v.kind = k;
                float ms = 1e30f;
                for (int rep = 0; rep < 4 && rc == MG_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    if (nodal) node_smooth<float>(h, l, x, b, 2);
                    else cell_smooth<float>(h, l, cview<float>(h, l), x, b, 2);
                    cudaEventRecord(e1, s);
                    float m = 0.f;
                    const cudaError_t e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess || cudaEventElapsedTime(&m, e0, e1) != cudaSuccess) {
                        rc = cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown, "autotune timing");
                        break;
                    }
                    if (rep > 0 && m < ms) ms = m;   // the first call is an untimed warm-up
                }
                if (ms < best_ms) { best_ms = ms; best = k; }
            }
            cudaMemsetAsync(x, 0, v.nvec * sizeof(float), s);
            cudaMemsetAsync(b, 0, v.nvec * sizeof(float), s);
            cudaMemsetAsync(t, 0, v.nvec * sizeof(float), s);
        }
        v.kind = rc == MG_OK ? best : 0;
        if (rc == MG_OK) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

void mg_default_options(mg_options* o)
{
    if (!o) return;
    o->prec = MG_PREC_MIXED;
    o->nu1 = 2;
    o->nu2 = 2;
    o->max_iters = 100;
    o->coarsest_max = 8;
    o->interp_order = 1;
    o->omega = 0.9;
    o->stream = nullptr;
    o->flags = 0;
    o->inner_cycles = 0;
}

static mg_status init_handle(mg_handle* h, const mg_geometry* g, const mg_bc* bc, const mg_options* o)
{
    h->geo = *g;
    h->bcin = *bc;
    h->opt = *o;
    h->dim = g->dim;
    h->loc = g->loc;
    h->prec = o->prec;
    h->singular = 1;
    for (int d = 0; d < 3; ++d) {
        h->bc.lo[d] = d < g->dim ? bc->lo[d] : BCN;
        h->bc.hi[d] = d < g->dim ? bc->hi[d] : BCN;
        if (d < g->dim && (bc->lo[d] == MG_BC_DIRICHLET || bc->hi[d] == MG_BC_DIRICHLET)) h->singular = 0;
    }
    h->stream = (cudaStream_t)o->stream;
    return MG_OK;
}

mg_status mg_hierarchy_bytes(const mg_geometry* g, const mg_bc* bc, const mg_options* o, size_t* bytes)
{
    mg_status rc = check_problem(g, bc, o);
    if (rc != MG_OK) return rc;
    if (!bytes) return fail(MG_ERR_INVALID_ARG, "bytes is null");
    mg_handle* h = new (std::nothrow) mg_handle();
    if (!h) return fail(MG_ERR_OOM, "host allocation failed");
    init_handle(h, g, bc, o);
    Bump B;
    rc = plan(h, B);
    *bytes = B.off + 256;
    delete h;
    return rc;
}

mg_status mg_setup(const mg_coeff* c, const mg_geometry* g, const mg_bc* bc, const mg_options* o, void* workspace,
                   size_t workspace_bytes, mg_handle** out)
{
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    mg_status rc = check_problem(g, bc, o);
    if (rc != MG_OK) return rc;
    mg_handle* h = new (std::nothrow) mg_handle();
    if (!h) return fail(MG_ERR_OOM, "host allocation failed");
    init_handle(h, g, bc, o);
    Bump dry;
    rc = plan(h, dry);
    if (rc != MG_OK) { delete h; return rc; }
    const size_t need = dry.off + 256;
    if (workspace) {
        if (workspace_bytes < need) { delete h; return fail(MG_ERR_OOM, "workspace smaller than mg_hierarchy_bytes()"); }
        if (((uintptr_t)workspace & 255) != 0) { delete h; return fail(MG_ERR_INVALID_ARG, "workspace must be 256-byte aligned"); }
        h->ws = workspace;
        h->own_ws = false;
    } else {
        cudaError_t e = cudaMalloc(&h->ws, need);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaMalloc(workspace)"); }
        h->own_ws = true;
    }
    h->ws_bytes = need;
    if (cudaHostAlloc((void**)&h->hs, sizeof(DevScalars), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&h->hs_dev, h->hs, 0) != cudaSuccess) {
        if (h->hs) cudaFreeHost(h->hs);
        if (h->own_ws) cudaFree(h->ws);
        delete h;
        return fail(MG_ERR_OOM, "pinned host allocation failed");
    }
    Bump real;
    real.base = (char*)h->ws;
    plan(h, real);
    cudaMemsetAsync(h->d, 0, sizeof(DevScalars), h->stream);
    // zero every work vector once (Dirichlet planes of nodal vectors stay 0)
    cudaMemsetAsync(h->ws, 0, need - 256, h->stream);
    rc = build_coefficients(h, c);
    // one-time limits of the TMA-staged sweep, here rather than inside a stream capture
    if (rc == MG_OK && h->prec == MG_PREC_MIXED && h->loc == MG_LOC_CELL && h->dim == 3)
        (void)cell_gsrb_tma_fits(h->lev[0].n[0]);
    if (rc == MG_OK && h->pipe_ctr) (void)cell_pipe_grid();
    if (rc == MG_OK && (h->opt.flags & MG_FLAG_AUTOTUNE)) rc = autotune(h);
    if (rc != MG_OK) { mg_destroy(h); return rc; }
    *out = h;
    return MG_OK;
}

mg_status mg_update_coeff(mg_handle* h, const mg_coeff* c)
{
    if (!h) return fail(MG_ERR_INVALID_ARG, "null handle");
    BusyGuard g(h);
    if (!g.ok) return fail(MG_ERR_BUSY, "handle in use");
    return build_coefficients(h, c);
}

mg_status mg_set_stream(mg_handle* h, void* stream)
{
    if (!h) return fail(MG_ERR_INVALID_ARG, "null handle");
    h->stream = (cudaStream_t)stream;
    h->opt.stream = stream;
    return MG_OK;
}

mg_status mg_solve(mg_handle* h, const double* rhs, double* phi, double tol, mg_stats* st)
{
    if (!h || !rhs || !phi) return fail(MG_ERR_INVALID_ARG, "null handle, rhs or phi");
    if (!(tol > 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be positive");
    BusyGuard g(h);
    if (!g.ok) return fail(MG_ERR_BUSY, "handle in use");
    const double t0 = now_ms();
    cudaStream_t s = h->stream;
    const size_t n = h->lev[0].nvec;
    mg_stats local;
    memset(&local, 0, sizeof local);
    mg_status rc;
    if (use_graph(h)) {
        rc = ensure_graph(h, 0);
        if (rc != MG_OK) return rc;
        MGP_LAUNCH(k_set_io<<<1, 1, 0, s>>>(h->d, rhs, phi, tol, h->opt.max_iters));
        MG_CK(cudaGraphLaunch(h->gx[0], s));
        MG_CK(cudaStreamSynchronize(s));
        rc = graph_result(h, h->g_fixed[0], h->g_body[0], h->g_if[0], &local);
    } else {
        vec_copy_f64(h->f64, rhs, n, s);
        if (h->loc == MG_LOC_NODAL) node_zero_dirichlet<double>(h->dim, nview<double>(h, 0), h->f64, s);
        vec_sum_sq(h->f64, n, h->partials, s);
        reduce_finalize(h->partials, 2, h->d->red, s);
        finish_rhs(h, 1, -1);
        rc = solve_core(h, phi, tol, &local);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mg_solve");
    local.ms = now_ms() - t0;
    local.status = rc;
    if (st) *st = local;
    return rc;
}

mg_status mg_project(mg_handle* h, double* const U[3], const mg_beta0* b0, const double* S, double* phi, double tol,
                     mg_stats* st)
{
    if (!h || !U || !b0 || !b0->cell || !S) return fail(MG_ERR_INVALID_ARG, "null argument");
    for (int d = 0; d < h->dim; ++d) {
        if (!U[d]) return fail(MG_ERR_INVALID_ARG, "U[d] is null");
        if (h->loc == MG_LOC_CELL && !b0->face[d]) return fail(MG_ERR_INVALID_ARG, "beta0 faces are required (MAC)");
    }
    if (!(tol > 0.0)) return fail(MG_ERR_INVALID_ARG, "tol must be positive");
    BusyGuard g(h);
    if (!g.ok) return fail(MG_ERR_BUSY, "handle in use");
    const double t0 = now_ms();
    cudaStream_t s = h->stream;
    const int dim = h->dim;
    const Level& v0 = h->lev[0];
    const double* Uc[3] = {U[0], U[1], dim == 3 ? U[2] : nullptr};
    if (phi == nullptr) {
        phi = h->phi_int;
        zero(phi, v0.nvec, s);
    }
    // a2: f = D(beta0 U) - beta0 S
    if (h->loc == MG_LOC_CELL) cell_rhs(dim, cview<double>(h, 0), v0.h, Uc, b0->face, b0->cell, S, h->f64, h->partials, s);
    else node_rhs(dim, nview<double>(h, 0), v0.h[0], Uc, b0->cell, S, h->f64, h->partials, s);
    reduce_finalize(h->partials, 3, h->d->red, s);
    finish_rhs(h, 2, 1);
    mg_stats local;
    memset(&local, 0, sizeof local);
    // a3-a8
    mg_status rc;
    if (use_graph(h)) {
        rc = ensure_graph(h, 1);
        if (rc != MG_OK) return rc;
        MGP_LAUNCH(k_set_io<<<1, 1, 0, s>>>(h->d, nullptr, phi, tol, h->opt.max_iters));
        if (h->loc == MG_LOC_CELL) MGP_LAUNCH(k_constraint_tol<<<1, 1, 0, s>>>(h->d));
        MG_CK(cudaGraphLaunch(h->gx[1], s));
        MG_CK(cudaStreamSynchronize(s));
        rc = graph_result(h, h->g_fixed[1], h->g_body[1], h->g_if[1], &local);
    } else {
        rc = solve_core(h, phi, tol, &local, h->loc == MG_LOC_CELL);
    }
    if (rc == MG_OK || rc == MG_ERR_NOT_CONVERGED) {
        // a9: projection update; a10: constraint
        if (h->loc == MG_LOC_CELL) {
            cell_project(dim, cview<double>(h, 0), v0.h, phi, b0->face, U, s);
            cell_rhs(dim, cview<double>(h, 0), v0.h, Uc, b0->face, b0->cell, S, nullptr, h->partials, s);
        } else {
            node_project(dim, nview<double>(h, 0), v0.h[0], phi, b0->cell, U, s);
            // the nodal projection is approximate: its constraint is a diagnostic,
            // formed in FP32 where the tiled kernel applies (||S_N|| from the FP64 RHS)
            if (!node_constraint32(dim, nview<double>(h, 0), v0.h[0], Uc, b0->cell, S, h->partials, s))
                node_rhs(dim, nview<double>(h, 0), v0.h[0], Uc, b0->cell, S, nullptr, h->partials, s);
        }
        reduce_finalize(h->partials, 3, h->d->red, s);
        mg_status r2 = readback(h);
        if (r2 != MG_OK) return r2;
        const double src2 = h->loc == MG_LOC_CELL ? h->hs->red[1] : h->hs->src2, con2 = h->hs->red[2];
        local.src_norm = sqrt(src2);
        local.rel_constraint = src2 > 0.0 ? sqrt(con2 / src2) : sqrt(con2);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mg_project");
    local.ms = now_ms() - t0;
    local.status = rc;
    if (st) *st = local;
    return rc;
}

mg_status mg_rhs(mg_handle* h, const double* const U[3], const mg_beta0* b0, const double* S, double* f)
{
    if (!h || !U || !b0 || !b0->cell || !S || !f) return fail(MG_ERR_INVALID_ARG, "null argument");
    for (int d = 0; d < h->dim; ++d) {
        if (!U[d]) return fail(MG_ERR_INVALID_ARG, "U[d] is null");
        if (h->loc == MG_LOC_CELL && !b0->face[d]) return fail(MG_ERR_INVALID_ARG, "beta0 faces are required (MAC)");
    }
    BusyGuard g(h);
    if (!g.ok) return fail(MG_ERR_BUSY, "handle in use");
    cudaStream_t s = h->stream;
    const Level& v0 = h->lev[0];
    const double* Uc[3] = {U[0], U[1], h->dim == 3 ? U[2] : nullptr};
    if (h->loc == MG_LOC_CELL) cell_rhs(h->dim, cview<double>(h, 0), v0.h, Uc, b0->face, b0->cell, S, f, h->partials, s);
    else node_rhs(h->dim, nview<double>(h, 0), v0.h[0], Uc, b0->cell, S, f, h->partials, s);
    if (h->singular) {
        reduce_finalize(h->partials, 1, h->d->red, s);
        vec_sub_mean(f, v0.nvec, &h->d->red[0], (double)v0.nvec, s);
    }
    MG_CK(cudaGetLastError());
    MG_CK(cudaStreamSynchronize(s));
    return MG_OK;
}

mg_status mg_solve_batch(mg_handle* const* hs, const double* const* rhs, double* const* phi, const double* tol,
                         int count, mg_stats* st)
{
    if (count < 0 || (count > 0 && (!hs || !rhs || !phi || !tol))) return fail(MG_ERR_INVALID_ARG, "bad batch");
    if (count == 0) return MG_OK;
    bool graph = true;
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || !rhs[i] || !phi[i] || !(tol[i] > 0.0)) return fail(MG_ERR_INVALID_ARG, "bad batch entry");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(MG_ERR_INVALID_ARG, "a handle appears twice in the batch");
        graph = graph && use_graph(hs[i]);
    }
    mg_status worst = MG_OK;
    const bool host_batched = !graph && batch_eligible(hs, count);
    if (!graph && !host_batched) {
        for (int i = 0; i < count; ++i) {
            mg_status rc = mg_solve(hs[i], rhs[i], phi[i], tol[i], st ? &st[i] : nullptr);
            if (rc != MG_OK && worst == MG_OK) worst = rc;
        }
        return worst;
    }
    std::vector<std::unique_ptr<BusyGuard>> guards;
    for (int i = 0; i < count; ++i) {
        guards.emplace_back(new BusyGuard(hs[i]));
        if (!guards.back()->ok) return fail(MG_ERR_BUSY, "handle in use");
    }
    const double t0 = now_ms();
    BatchGraph* bg = nullptr;
    if (!host_batched) {
        mg_status brc = batch_graph(hs, count, true, &bg);
        if (brc != MG_OK) return brc;
    }
    cudaStream_t s = hs[0]->stream;
    for (int i = 0; i < count; ++i)
        MGP_LAUNCH(k_set_io<<<1, 1, 0, s>>>(hs[i]->d, rhs[i], phi[i], tol[i], hs[i]->opt.max_iters));
    if (host_batched) {
        mg_status hrc = batch_host_loop(hs, count, true, s);
        if (hrc != MG_OK) return hrc;
    } else {
        MG_CK(cudaGraphLaunch(bg->exec, s));
        MG_CK(cudaStreamSynchronize(s));
        add_launches(bg->launches());
    }
    const double ms = now_ms() - t0;
    for (int i = 0; i < count; ++i) {
        mg_stats local;
        memset(&local, 0, sizeof local);
        mg_status rc = bg ? graph_result(hs[i], bg->fixed[i], bg->body[i], bg->ifb[i], &local)
                          : graph_result(hs[i], 0, 0, 0, &local);
        local.ms = ms;
        local.status = rc;
        if (st) st[i] = local;
        if (rc != MG_OK && worst == MG_OK) worst = rc;
    }
    return worst;
}

mg_status mg_project_batch(mg_handle* const* hs, double* const* U, const mg_beta0* b0, const double* const* S,
                           double* const* phi, const double* tol, int count, mg_stats* st)
{
    if (count < 0 || (count > 0 && (!hs || !U || !b0 || !S || !tol))) return fail(MG_ERR_INVALID_ARG, "bad batch");
    if (count == 0) return MG_OK;
    bool graph = true;
    for (int i = 0; i < count; ++i) {
        mg_handle* h = hs[i];
        if (!h || !S[i] || !b0[i].cell || !(tol[i] > 0.0)) return fail(MG_ERR_INVALID_ARG, "bad batch entry");
        for (int d = 0; d < h->dim; ++d) {
            if (!U[3 * i + d]) return fail(MG_ERR_INVALID_ARG, "U[d] is null");
            if (h->loc == MG_LOC_CELL && !b0[i].face[d]) return fail(MG_ERR_INVALID_ARG, "beta0 faces are required (MAC)");
        }
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) return fail(MG_ERR_INVALID_ARG, "a handle appears twice in the batch");
        graph = graph && use_graph(h);
    }
    mg_status worst = MG_OK;
    const bool host_batched = !graph && batch_eligible(hs, count);
    if (!graph && !host_batched) {
        for (int i = 0; i < count; ++i) {
            mg_status rc = mg_project(hs[i], U + 3 * i, &b0[i], S[i], phi ? phi[i] : nullptr, tol[i], st ? &st[i] : nullptr);
            if (rc != MG_OK && worst == MG_OK) worst = rc;
        }
        return worst;
    }
    std::vector<std::unique_ptr<BusyGuard>> guards;
    for (int i = 0; i < count; ++i) {
        guards.emplace_back(new BusyGuard(hs[i]));
        if (!guards.back()->ok) return fail(MG_ERR_BUSY, "handle in use");
    }
    const double t0 = now_ms();
    BatchGraph* bg = nullptr;
    if (!host_batched) {
        mg_status rc = batch_graph(hs, count, false, &bg);
        if (rc != MG_OK) return rc;
    }
    cudaStream_t s = hs[0]->stream;
    std::vector<double*> ph(count);
    // a2 on each handle's own stream (after whatever the caller queued there:
    // uploads, a coefficient update); the batch stream waits for all of them
    for (int i = 0; i < count; ++i) {
        mg_handle* h = hs[i];
        cudaStream_t hsx = h->stream;
        const Level& v0 = h->lev[0];
        const double* Uc[3] = {U[3 * i], U[3 * i + 1], h->dim == 3 ? U[3 * i + 2] : nullptr};
        ph[i] = phi && phi[i] ? phi[i] : h->phi_int;
        if (ph[i] == h->phi_int) zero(ph[i], v0.nvec, hsx);
        if (h->loc == MG_LOC_CELL)
            cell_rhs(h->dim, cview<double>(h, 0), v0.h, Uc, b0[i].face, b0[i].cell, S[i], h->f64, h->partials, hsx);
        else
            node_rhs(h->dim, nview<double>(h, 0), v0.h[0], Uc, b0[i].cell, S[i], h->f64, h->partials, hsx);
        reduce_finalize(h->partials, 3, h->d->red, hsx);
        finish_rhs(h, 2, 1);
        if (hsx != s) {
            if (!h->ev) MG_CK(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
            MG_CK(cudaEventRecord(h->ev, hsx));
            MG_CK(cudaStreamWaitEvent(s, h->ev, 0));
        }
    }
    // a3-a8: every solve a branch of one graph
    for (int i = 0; i < count; ++i) {
        MGP_LAUNCH(k_set_io<<<1, 1, 0, s>>>(hs[i]->d, nullptr, ph[i], tol[i], hs[i]->opt.max_iters));
        if (hs[i]->loc == MG_LOC_CELL) MGP_LAUNCH(k_constraint_tol<<<1, 1, 0, s>>>(hs[i]->d));
    }
    if (host_batched) {
        mg_status hrc = batch_host_loop(hs, count, false, s);
        if (hrc != MG_OK) return hrc;
    } else {
        MG_CK(cudaGraphLaunch(bg->exec, s));
        MG_CK(cudaStreamSynchronize(s));
        add_launches(bg->launches());
    }
    // a9-a10 on each handle's stream (concurrently), then the read-backs
    std::vector<mg_stats> local(count);
    std::vector<mg_status> rcs(count);
    for (int i = 0; i < count; ++i) {
        mg_handle* h = hs[i];
        memset(&local[i], 0, sizeof(mg_stats));
        rcs[i] = bg ? graph_result(h, bg->fixed[i], bg->body[i], bg->ifb[i], &local[i])
                    : graph_result(h, 0, 0, 0, &local[i]);
        if (rcs[i] != MG_OK && rcs[i] != MG_ERR_NOT_CONVERGED) continue;
        cudaStream_t hsx = h->stream;
        const Level& v0 = h->lev[0];
        double* const Ui[3] = {U[3 * i], U[3 * i + 1], h->dim == 3 ? U[3 * i + 2] : nullptr};
        const double* Uc[3] = {Ui[0], Ui[1], Ui[2]};
        if (h->loc == MG_LOC_CELL) {
            cell_project(h->dim, cview<double>(h, 0), v0.h, ph[i], b0[i].face, Ui, hsx);
            cell_rhs(h->dim, cview<double>(h, 0), v0.h, Uc, b0[i].face, b0[i].cell, S[i], nullptr, h->partials, hsx);
        } else {
            node_project(h->dim, nview<double>(h, 0), v0.h[0], ph[i], b0[i].cell, Ui, hsx);
            if (!node_constraint32(h->dim, nview<double>(h, 0), v0.h[0], Uc, b0[i].cell, S[i], h->partials, hsx))
                node_rhs(h->dim, nview<double>(h, 0), v0.h[0], Uc, b0[i].cell, S[i], nullptr, h->partials, hsx);
        }
        reduce_finalize(h->partials, 3, h->d->red, hsx);
    }
    for (int i = 0; i < count; ++i) {
        mg_handle* h = hs[i];
        if (rcs[i] == MG_OK || rcs[i] == MG_ERR_NOT_CONVERGED) {
            const mg_status r2 = readback(h);
            if (r2 != MG_OK) {
                rcs[i] = r2;
            } else {
                const double src2 = h->loc == MG_LOC_CELL ? h->hs->red[1] : h->hs->src2, con2 = h->hs->red[2];
                local[i].src_norm = sqrt(src2);
                local[i].rel_constraint = src2 > 0.0 ? sqrt(con2 / src2) : sqrt(con2);
            }
        }
        if (rcs[i] != MG_OK && worst == MG_OK) worst = rcs[i];
    }
    const double ms = now_ms() - t0;
    for (int i = 0; i < count; ++i) {
        local[i].ms = ms;
        local[i].status = rcs[i];
        if (st) st[i] = local[i];
    }
    return worst;
}

mg_status mg_apply(mg_handle* h, const double* phi, double* out)
{
    if (!h || !phi || !out) return fail(MG_ERR_INVALID_ARG, "null argument");
    if (h->loc == MG_LOC_CELL) cell_apply64(h->dim, cview<double>(h, 0), phi, out, h->stream);
    else node_apply64(h->dim, nview<double>(h, 0), phi, out, h->stream);
    MG_CK(cudaGetLastError());
    MG_CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

mg_status mg_set_batch_groups(int groups)
{
    if (groups < 0 || groups > 64) return fail(MG_ERR_INVALID_ARG, "batch groups must be in 0 .. 64");
    g_batch_groups.store(groups, std::memory_order_relaxed);
    return MG_OK;
}

void mg_destroy(mg_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    drop_batches_of(h);
    for (int i = 0; i < 2; ++i) {
        if (h->gx[i]) cudaGraphExecDestroy(h->gx[i]);
        if (h->cg[i]) cudaGraphExecDestroy(h->cg[i]);
    }
    if (h->ev) cudaEventDestroy(h->ev);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->hs) cudaFreeHost(h->hs);
    delete h;
}

const char* mg_strerror(mg_status s)
{
    switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_DIVERGED: return "diverged";
    case MG_ERR_INCOMPATIBLE_RHS: return "incompatible right-hand side";
    case MG_ERR_TIMEOUT: return "timeout";
    case MG_ERR_BUSY: return "handle busy";
    case MG_ERR_UNSUPPORTED: return "unsupported problem";
    }
    return "unknown status";
}

const char* mg_last_error(void) { return g_last_error.c_str(); }

mg_status mg_convert_f64_to_f32(const double* x, float* y, size_t n, void* stream)
{
    if (n == 0) return MG_OK;
    if (!x || !y) return fail(MG_ERR_INVALID_ARG, "null array");
    vec_to_f32(y, x, n, (cudaStream_t)stream);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_convert_f64_to_f32_pow2(const double* x, float* y, size_t n, int shift, void* stream)
{
    if (n == 0) return MG_OK;
    if (!x || !y) return fail(MG_ERR_INVALID_ARG, "null array");
    if (shift < -1022 || shift > 1023) return fail(MG_ERR_INVALID_ARG, "shift out of range");
    vec_to_f32_pow2(y, x, n, shift, (cudaStream_t)stream);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_convert_f32_to_f64(const float* x, double* y, size_t n, void* stream)
{
    if (n == 0) return MG_OK;
    if (!x || !y) return fail(MG_ERR_INVALID_ARG, "null array");
    vec_to_f64(y, x, n, (cudaStream_t)stream);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_reciprocal_f64(const double* x, double* y, size_t n, void* stream)
{
    if (n == 0) return MG_OK;
    if (!x || !y) return fail(MG_ERR_INVALID_ARG, "null array");
    vec_recip(y, x, n, (cudaStream_t)stream);
    MG_CK(cudaGetLastError());
    return MG_OK;
}

int mg_smoother_kind(const mg_handle* h, int level)
{
    if (!h || level < 0 || level >= h->nlev) return -1;
    return h->lev[level].kind;
}

long long mg_launch_count(void) { return launch_count(); }

void mg_prof_enable(int on)
{
    Prof& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    P.used = 0;
    P.on = on != 0;
}

mg_status mg_prof_query(int kernel, double* total_ms, int* launches, double* bytes, double* flops)
{
    if (kernel < 0 || kernel >= MG_PROF_COUNT) return fail(MG_ERR_INVALID_ARG, "unknown kernel class");
    Prof& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    double ms = 0.0, by = 0.0, fl = 0.0;
    int cnt = 0;
    for (size_t i = 0; i < P.used; ++i) {
        const ProfRec& r = P.recs[i];
        if (r.id != kernel) continue;
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        ms += t;
        by += r.bytes;
        fl += r.flops;
        cnt += r.count;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = cnt;
    if (bytes) *bytes = by;
    if (flops) *flops = fl;
    return MG_OK;
}

}  // extern "C"
