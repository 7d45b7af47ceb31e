// mg_internal.cuh -- shared declarations of the CUDA projection-solve library.
//
// Everything here is internal to libmgproj.so; the public surface is include/mg.h.
// Kernels are plain CUDA C++ for sm_103a: the multigrid path is a sparse stencil,
// so it is bound by HBM bandwidth (FP32 levels) or the FP64 pipe (FP64 residual),
// never by a dense contraction; no tensor-core instruction appears anywhere.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/mg.h"

namespace mgp {

enum { BCP = 0, BCN = 1, BCD = 2 };

constexpr int kNumSMs = 152;        // SMs of a GB300 (two dies of 76)
constexpr int kRedBlocks = 608;     // 4 x 152 SMs: fixed grid of every reduction kernel
constexpr int kRedSlots = 4;        // quantities one reduction pass may accumulate
constexpr int kMaxLevels = 16;
constexpr int kMaxDense = 512;      // unknowns of the coarsest (dense) level

struct BC3 {
    int lo[3];
    int hi[3];
};

// One cell-centred level: n cells per axis, face coefficients pre-scaled by 1/h_d^2.
template <typename T>
struct CellLevel {
    int nx, ny, nz;
    BC3 bc;
    const T* bx;
    const T* by;
    const T* bz;
    const T* invd;  // optional 1/diagonal (FP64 levels); nullptr -> computed
    const T* diag;  // optional diagonal for the FP64 residual; nullptr -> computed
};

// One nodal level: n cells per axis, N nodes per axis, sigma per cell, h^-2.
template <typename T>
struct NodeLevel {
    int nx, ny, nz;     // cells
    int Nx, Ny, Nz;     // stored nodes
    BC3 bc;
    const T* sigma;
    T ih2;
    const T* invd;      // optional 1/diagonal; nullptr -> computed
    const T* diag;      // optional diagonal for the FP64 residual; nullptr -> computed
};

// Device scalars of one solve (reduction results and the iteration state that
// the graph-resident solve loop keeps on the device).
struct DevScalars {
    double red[kRedSlots];     // last reduction results
    double fnorm2;             // ||f||^2 of the system being solved
    double rnorm2;             // ||f - L phi||^2 / ||f||^2, latest (squared relative residual)
    double fscale;             // r32 = (f - L phi) / fscale in mixed refinement: the power of two <= ||f||
    double rscale2;            // (fscale / ||f||)^2: turns the sum of r32^2 into ||f - L phi||^2 / ||f||^2
    double mean;               // mean removed from f (singular problems)
    double src2;               // ||beta0 S||^2 or ||S_N||^2
    double con2;               // post-projection constraint^2
    double tol;                // relative tolerance of the current solve
    double rel, rel0, best;    // relative residual: latest, initial, best
    int info;                  // dense coarsest factorisation: 0 ok, k > 0 zero pivot
    int iters, stall, status;  // iteration count, stalled iterations, mg_status
    int maxit;
    const double* rhs_in;      // caller rhs of the current call (graph mode)
    double* phi_io;            // caller phi of the current call (graph mode)
    double prev_rel;           // relative residual before the last refinement step
    int ncyc;                  // V-cycles of the next refinement step (automatic inner cycles)
    int n_extra;               // V-cycles run beyond the first of each refinement step (launch accounting)
    int async_err;             // set by a kernel whose bounded wait for an asynchronous copy gave up
};

// Every kernel launch of the library goes through MGP_LAUNCH, which counts it
// (mg_launch_count reports the total).
// sets the message mg_last_error() returns on this thread
void set_last_error(const char* msg);
// geometry, boundary kinds and stream of a handle (for entry points outside the engine)
void handle_info(const mg_handle* h, mg_geometry* g, mg_bc* bc, cudaStream_t* s);
void note_launch();
void add_launches(long long n);
long long launch_count();
#define MGP_LAUNCH(...) (::mgp::note_launch(), __VA_ARGS__)

// ---------------------------------------------------------------- launchers
// Cell-centred (MAC) system.  dim = 2 or 3.  All launches are asynchronous on s.
void cell_faces_from_sigma(int dim, const CellLevel<double>& L, const double* sigma, const double* h,
                           double* bx, double* by, double* bz, cudaStream_t s);
void cell_scale_faces(int dim, const CellLevel<double>& L, const double* const face[3], const double* h,
                      double* bx, double* by, double* bz, cudaStream_t s);
void cell_coarsen_faces(int dim, const CellLevel<double>& F, const CellLevel<double>& C, double* bx, double* by,
                        double* bz, cudaStream_t s);
void cell_invdiag(int dim, const CellLevel<double>& L, double* invd, cudaStream_t s);
void cell_diag(int dim, const CellLevel<double>& L, double* diag, cudaStream_t s);
template <typename T>
void cell_gsrb(int dim, const CellLevel<T>& L, T* x, const T* b, int color, cudaStream_t s);
// one full red-then-black sweep xin -> xout in a single launch (when ok)
template <typename T>
bool cell_gsrb_fused_ok(int dim, const CellLevel<T>& L);
// one colour pass, four cells per thread with 16-byte accesses (FP32, nx % 4 == 0,
// 16-byte aligned x, b and face arrays); same arithmetic as cell_gsrb
bool cell_gsrb_v4_ok(int dim, const CellLevel<float>& L, const float* x, const float* b);
// bxw: quads per block row (8, 16 or 32; 0 picks by the level's width)
void cell_gsrb_v4(int dim, const CellLevel<float>& L, float* x, const float* b, int color, cudaStream_t s,
                  int bxw = 0);
// one full red-black sweep in one pass over memory, operands staged in shared
// memory by bulk asynchronous copies (xin -> xout; same results as two
// cell_gsrb passes); err: a device word set if a bounded wait gave up
bool cell_gsrb_tma_ok(int dim, const CellLevel<float>& L, const float* xin, const float* xout, const float* b);
bool cell_gsrb_tma_fits(int nx);
void cell_gsrb_tma(const CellLevel<float>& L, const float* xin, float* xout, const float* b, int* err,
                   cudaStream_t s);
// The down leg (nu1 sweeps, residual, restriction) or the up leg (linear
// prolongation, nu2 sweeps) of a cell V-cycle on a 3-D FP32 level as one
// persistent launch whose passes are pipelined through L2 (mg_cellpipe.cu);
// same results as the pass-by-pass kernels.  S: per-handle ticket / exit /
// epoch counters (3 words) and cell_pipe_flag_words() item flags, zeroed once
// at setup; S.err is set if a bounded wait gave up.
enum { PIPE_RED = 0, PIPE_BLACK = 1, PIPE_RESTRICT = 2, PIPE_PROLONG = 3 };
constexpr int kPipeBand = 8;       // fine rows per work item
constexpr int kPipeZ = 2;          // planes per step
constexpr int kPipeMaxNu = 4;      // sweeps per leg
constexpr int kPipeMaxPass = 2 * kPipeMaxNu + 1;
constexpr size_t kPipeMinCells = (size_t)1 << 14;   // finest levels of 2^14 cells and more
constexpr int kPipeK = 3;          // slots between a pass and the next one (steps in flight)
struct CellPipe {
    int npass, Z, nband, nstep, zero_first, yper, K, nslot;
    int op[kPipeMaxPass];
    int lag[kPipeMaxPass];
    int dep[kPipeMaxPass];
};
struct PipeSync {
    unsigned* ctr;
    unsigned* flags;
    int* err;
};
bool cell_pipe_ok(const CellLevel<float>& F, const float* x, const float* b);
int cell_pipe_grid();   // resident CTAs of the pipelined kernel (first call: outside stream capture)
size_t cell_pipe_flag_words(int ny, int nz, int nu_max);
void cell_pipe_down(const CellLevel<float>& F, float* x, const float* b, float* bc, int nu1, bool zero_first,
                    const PipeSync& S, cudaStream_t s);
void cell_pipe_up(const CellLevel<float>& F, const CellLevel<float>& C, float* x, const float* b, const float* xc,
                  int nu2, const PipeSync& S, cudaStream_t s);
// 3-D residual + restriction, vectorised like cell_gsrb_v4; same results as cell_resid_restrict
bool cell_resid_restrict_v4_ok(int dim, const CellLevel<float>& F, const float* x, const float* b, const float* bc);
void cell_resid_restrict_v4(const CellLevel<float>& F, const float* x, const float* b, float* bc, cudaStream_t s);
// 3-D linear prolongation and correction, four fine cells per thread
bool cell_prolong_v4_ok(int dim, const CellLevel<float>& F, const float* xf, const float* xc);
void cell_prolong_v4(const CellLevel<float>& F, const CellLevel<float>& C, float* xf, const float* xc, cudaStream_t s);
template <typename T>
void cell_gsrb_sweep(int dim, const CellLevel<T>& L, const T* xin, T* xout, const T* b, cudaStream_t s);
template <typename T>
void cell_resid_restrict(int dim, const CellLevel<T>& F, const T* x, const T* b, T* bc, cudaStream_t s);
template <typename T>
void cell_prolong_add(int dim, const CellLevel<T>& F, const CellLevel<T>& C, T* xf, const T* xc, int order,
                      cudaStream_t s);
// r = b - L x in FP64; optional FP32 copy r/scale; partials of sum (r/scale)^2
// (accumulated in FP32: the norm only steers convergence decisions)
// vec: the four-cells-per-thread kernel where the level allows it (same results)
void cell_resid64(int dim, const CellLevel<double>& L, const double* x, const double* b, float* r32,
                  const double* scale, double* partials, cudaStream_t s, bool vec = true);
void cell_apply64(int dim, const CellLevel<double>& L, const double* x, double* out, cudaStream_t s);
// f = D(beta0 U) - beta0 S with partials {sum f, sum (beta0 S)^2, sum f^2}; f may be null
void cell_rhs(int dim, const CellLevel<double>& L, const double* h, const double* const U[3],
              const double* const b0f[3], const double* b0c, const double* S, double* f, double* partials,
              cudaStream_t s);
void cell_project(int dim, const CellLevel<double>& L, const double* h, const double* phi,
                  const double* const b0f[3], double* const U[3], cudaStream_t s);
template <typename T>
void cell_dense_assemble(int dim, const CellLevel<T>& L, double* A, int lda, cudaStream_t s);

// The coarse end of a cell V-cycle in one CTA (levels of at most kCoarseCells
// cells, at most kCoarseMaxLevels of them): zero (all but the first level
// unless zero_first), nu1 colour sweeps, residual restriction, dense bottom
// solve, prolongation, nu2 sweeps; same arithmetic as the launched kernels.
constexpr int kCoarseCells = 512;
constexpr int kCoarseMaxLevels = 8;
template <typename T>
void coarse_cycle(int dim, int nlev, const CellLevel<T>* L, T* const* x, T* const* b, const double* Minv, int Nd,
                  int nu1, int nu2, int order, bool zero_first, cudaStream_t s);
// The arguments of one coarse end (levels of the sub-cycle, coarsest last).
template <typename T>
struct CoarseArgs {
    int nlev;                          // levels of the sub-cycle; the last is the coarsest
    CellLevel<T> L[kCoarseMaxLevels];
    T* x[kCoarseMaxLevels];
    T* b[kCoarseMaxLevels];            // b[0]: the sub-cycle's right-hand side (read only)
    const double* Minv;
    int Nd, nu1, nu2, order, zero_first;
};

// ---- batched solves: the same steps of many independent cell solves (3-D,
// FP32 V-cycles in FP64 refinement) share one launch per step.  Each launch
// reads a table of work items in device memory -- one per solve that has work
// in that step -- and its CTAs stay resident and walk the items' tiles; a
// solve's items run while its run flag (run[solve]) is set, so solves that
// have converged drop out without the launch sequence changing.  Every item
// computes with the per-quad, per-cell and per-block functions of the
// single-solve kernels, over the same partition where a reduction is formed,
// so each solve's result equals its result alone bit for bit.
enum { BATCH_GSRB = 0, BATCH_RESTRICT = 1, BATCH_PROLONG = 2 };
constexpr int kBatchTile = 32;               // work units per (warp) tile
constexpr size_t kBatchCoarseCells = 512;    // batched coarse ends start at the first level this small
// One solve's share of a batched level launch: a colour pass, the residual +
// restriction to C, or the linear prolongation from C, on level F (3-D FP32,
// nx % 4 == 0, ny and nz even).  units: quads (colour pass, prolongation) or
// quad columns of 2 x 2 rows and planes (restriction); tile0: first tile.  A
// launch also takes the item index of each of its tiles (tmap).
struct BatchItem {
    CellLevel<float> F, C;
    float* x;
    const float* b;
    float* bc;
    const float* xc;
    int solve, tile0, units;
    int sq, sy;        // multiply-shift divisors (batch_magic): nx / 4, and ny (ny / 2 for the restriction)
    unsigned mq, my;
};
// (m, s) with floor(n / d) = (n m) >> s for 0 <= n < 2^31
void batch_magic(int d, unsigned* m, int* s);
// The parameter of one batched level launch: its items (sorted by first tile)
// and its warp tiles; it fits the 32 KB kernel-parameter space.
constexpr int kBatchLaunchItems = 96;
struct BatchLaunch {
    int nitems, tiles;
    BatchItem items[kBatchLaunchItems];
};
void batch_level(int op, const BatchLaunch& B, const int* run, int color, int zx, cudaStream_t s);
// the coarse ends of count solves, one 1024-thread CTA each (A[i] belongs to solve i)
void coarse_cycle_batch(const CoarseArgs<float>* A, int count, const int* run, cudaStream_t s);
// FP64 residual, FP32 copy and norm partials of many cell solves (the
// four-cells-per-thread kernel's traversal and block partition per solve):
// blocks vb0 .. vb0 + nvb - 1 of the launch are a solve's blocks with quads
// (nvb = min(kRedBlocks, quads / kThreads rounded up)); bmap gives the item of
// each block.
struct Resid64Item {
    CellLevel<double> L;
    const double* x;
    const double* b;
    float* r32;
    const double* scale;
    double* partials;
    int solve, vb0, nvb, pad;
};
bool cell_resid64_batch_ok(const CellLevel<double>& L, const double* x, const double* b, const float* r32);
void cell_resid64_batch(const Resid64Item* items, const int* bmap, int blocks, const int* run, cudaStream_t s);
// *out = (sum of the partials of slot 0) * *mul per solve, in reduce_finalize's order
struct FinalItem {
    const double* partials;
    double* out;
    const double* mul;
    int solve, pad;
};
void reduce_finalize_batch(const FinalItem* items, int count, const int* run, cudaStream_t s);
// phi += (*scale) e per solve; n4: groups of four entries (n % 4 == 0, 16-byte aligned)
struct AxpyItem {
    double* phi;
    const float* e;
    const double* scale;
    int solve, tile0, n4, pad;
};
int axpy_batch_grid(int tiles);
void axpy_f32_batch(const AxpyItem* items, int count, int tiles, const int* run, int grid, cudaStream_t s);
// The coarse end of a nodal V-cycle in one CTA (levels of at most kCoarseNodes
// stored nodes): zero, nu1 Jacobi sweeps (ping-pong with t), residual into r,
// restriction, dense bottom solve, prolongation, nu2 sweeps; same arithmetic
// as the launched kernels.
constexpr int kCoarseNodes = 1024;
template <typename T>
void node_coarse_cycle(int dim, int nlev, const NodeLevel<T>* L, T* const* x, T* const* b, T* const* t, T* const* r,
                       const double* Minv, int Nd, int nu1, int nu2, T omega, bool zero_first, cudaStream_t s);

// Nodal system.
void node_coarsen_sigma(int dim, const NodeLevel<double>& F, const NodeLevel<double>& C, double* sc,
                        cudaStream_t s);
void node_invdiag(int dim, const NodeLevel<double>& L, double* invd, cudaStream_t s);
void node_diag(int dim, const NodeLevel<double>& L, double* diag, cudaStream_t s);
// tiled: allow the shared-memory tiled kernel (3-D levels of at least 32 x 8 nodes)
// kind: 0 the default choice; 1..3 the four-node kernel with 8/16/32 quads per
// block row, one plane per thread; 4 the shared-memory tiled kernel; 5..7 the
// four-node kernel with 8/16/32 quads per block row marching four planes (when
// the level allows each)
template <typename T>
void node_jacobi(int dim, const NodeLevel<T>& L, const T* x, T* xo, const T* b, T omega, bool tiled, cudaStream_t s,
                 int kind = 0);
template <typename T>
void node_resid(int dim, const NodeLevel<T>& L, const T* x, const T* b, T* r, bool tiled, cudaStream_t s,
                int kind = 0);
template <typename T>
void node_restrict(int dim, const NodeLevel<T>& F, const NodeLevel<T>& C, const T* rf, T* bc, cudaStream_t s);
template <typename T>
void node_prolong_add(int dim, const NodeLevel<T>& F, const NodeLevel<T>& C, T* xf, const T* xc, cudaStream_t s);
// FP32 3-D levels with x periodic and nx % 4 == 0: Jacobi sweep / residual with
// four nodes per thread (same results as the plain kernels); bxw quads per
// block row (0: by the row length), kz node planes marched per thread (1 or 4;
// 0: by the level size)
bool node_v4_ok(int dim, const NodeLevel<float>& L, const float* x, const float* out, const float* b);
void node_v4(const NodeLevel<float>& L, const float* x, float* out, const float* b, float omega, bool resid,
             cudaStream_t s, int bxw = 0, int kz = 0);
bool node_prolong_v4_ok(int dim, const NodeLevel<float>& F, const float* xf, const float* xc);
// full-weighting restriction of FP32 3-D nodal levels with x periodic, two
// coarse nodes per thread (same results as k_node_restrict)
bool node_restrict_v4_ok(int dim, const NodeLevel<float>& F, const float* rf, const float* bc);
void node_restrict_v4(const NodeLevel<float>& F, const NodeLevel<float>& C, const float* rf, float* bc,
                      cudaStream_t s);
void node_prolong_v4(const NodeLevel<float>& F, const NodeLevel<float>& C, float* xf, const float* xc, cudaStream_t s);
void node_resid64(int dim, const NodeLevel<double>& L, const double* x, const double* b, float* r32,
                  const double* scale, double* partials, cudaStream_t s);
// Level-0 data of the sum-factorised FP64 nodal residual (3-D): per node the
// sigma sums over the cells around its +x, +y and +z edges (w), and
// dq = -(5/12) sum(sigma of its cells) / h^2 (0 at Dirichlet nodes).
struct NodeEdges {
    double* w[3];
    double* dq;
};
void node_edges(const NodeLevel<double>& L, const NodeEdges& E, cudaStream_t s);
void node_resid64_sf(const NodeLevel<double>& L, const NodeEdges& E, const double* x, const double* b, float* r32,
                     const double* scale, double* partials, cudaStream_t s);
void node_apply64(int dim, const NodeLevel<double>& L, const double* x, double* out, cudaStream_t s);
void node_rhs(int dim, const NodeLevel<double>& L, double h, const double* const U[3], const double* b0,
              const double* S, double* f, double* partials, cudaStream_t s);
// the post-projection diagnostic D_N(beta0 U) - S_N of the nodal projection
// with FP32 arithmetic (FP64 inputs rounded as loaded; partial sums in FP64):
// partials {sum v, sum lump^2, sum v^2} like node_rhs; false (nothing
// launched) where the tiled kernel does not apply
bool node_constraint32(int dim, const NodeLevel<double>& L, double h, const double* const U[3], const double* b0,
                       const double* S, double* partials, cudaStream_t s);
void node_project(int dim, const NodeLevel<double>& L, double h, const double* phi, const double* b0,
                  double* const U[3], cudaStream_t s);
template <typename T>
void node_dense_assemble(int dim, const NodeLevel<T>& L, double* A, int lda, cudaStream_t s);
// zero the Dirichlet node planes of x
template <typename T>
void node_zero_dirichlet(int dim, const NodeLevel<T>& L, T* x, cudaStream_t s);

// Generic helpers.
// out[q] = sum of the partials of slot q (times *mul when mul is given)
void reduce_finalize(const double* partials, int nslots, double* out, cudaStream_t s, const double* mul = nullptr);
// partials {sum v, sum v^2} of v[0..n)
void vec_sum_sq(const double* v, size_t n, double* partials, cudaStream_t s);
// v[i] -= *mean (mean = sum / count read from a device scalar)
void vec_sub_mean(double* v, size_t n, const double* sum, double count, cudaStream_t s);
void vec_copy_f64(double* dst, const double* src, size_t n, cudaStream_t s);
void vec_to_f32(float* dst, const double* src, size_t n, cudaStream_t s);
// dst = src * 2^shift rounded to binary32 (the FP64 residual kernels' scaled conversion)
void vec_to_f32_pow2(float* dst, const double* src, size_t n, int shift, cudaStream_t s);
void vec_to_f64(double* dst, const float* src, size_t n, cudaStream_t s);
void vec_recip(double* dst, const double* src, size_t n, cudaStream_t s);
// r32 = f / scale and partials of its squared norm: the residual of x = 0
void vec_init_zero_guess(const double* f, float* r32, const double* scale, double* partials, size_t n,
                         cudaStream_t s);
void vec_zero_f32(float* v, size_t n, cudaStream_t s);
void vec_zero_f64(double* v, size_t n, cudaStream_t s);
// phi += (*scale) * e
void vec_axpy_f32(double* phi, const float* e, const double* scale, size_t n, cudaStream_t s);
// dense coarsest solve: A holds the assembled N x N operator with row stride
// 2 (N + singular); Minv = leading N x N block of the (bordered) inverse
int dense_invert(double* A, int N, int singular, double* Minv, int* info, cudaStream_t s);
template <typename T>
void dense_apply(const double* Minv, int N, const T* b, T* x, cudaStream_t s);
// scalars: s->fscale = sqrt(s->fnorm2) (or 1 if 0)
void scalars_set_fscale(DevScalars* d, cudaStream_t s);

}  // namespace mgp
