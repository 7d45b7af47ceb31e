/*
 * mg.h -- C ABI of the GB300 projection-solve library (libmgproj.so).
 *
 * The library solves the variable-coefficient elliptic problem that enforces the
 * velocity constraint of the low Mach number equations (Eq. 6, S2, with the
 * base state frozen so that dp0/dt = 0):
 *
 *     div( sigma grad phi ) = div(beta0 U) - beta0 S,      sigma = beta0 / rho,
 *
 * by geometric multigrid V-cycles (S3 solves the projections with multigrid), and
 * applies the projection U <- U - (sigma/beta0) grad phi that the gradient term of
 * the momentum equation (Eq. 2) implies.  Two discretisations are offered, one per
 * projection of the second-order projection method of S3:
 *
 *   MG_LOC_CELL   MAC projection: phi at cell centres, U on faces.  The discrete
 *                 operator is L = D B G with B the harmonic mean of sigma on faces,
 *                 so the projected face velocity satisfies the discrete constraint
 *                 D(beta0 U) - beta0 S = (solver residual) exactly.
 *   MG_LOC_NODAL  nodal projection: phi at nodes, U at cell centres, Q1 finite
 *                 elements with sigma constant per cell (27-point operator in 3-D,
 *                 9-point in 2-D).  This projection is approximate.
 *
 * Grids are uniform, 2-D or 3-D, on [0, n_d h_d].  Array layout (all arrays):
 * x fastest, C order, double precision, DEVICE memory owned by the caller:
 *   cells   nx*ny*nz                   index (k*ny + j)*nx + i
 *   x faces (nx+1)*ny*nz               index (k*ny + j)*(nx+1) + i   (face i is the low face of cell i)
 *   y faces nx*(ny+1)*nz               index (k*(ny+1) + j)*nx + i
 *   z faces nx*ny*(nz+1)               index (k*ny + j)*nx + i
 *   nodes   Nx*Ny*Nz, N_d = n_d on periodic axes (node n_d is node 0), n_d + 1 otherwise
 * 2-D problems set dim = 2 and n[2] = 1 and have no z faces.  On periodic axes the
 * face arrays still hold n_d + 1 planes; planes 0 and n_d are the same face and
 * the library writes both.
 *
 * Boundary conditions per domain face: periodic (paired), Neumann (a wall: no
 * flux, the wall-normal velocity is left unchanged), Dirichlet (phi = 0, an
 * outflow boundary).  A problem with no Dirichlet face is singular: the library
 * removes the mean of the right-hand side and returns the zero-mean solution.
 *
 * Errors: every call returns an mg_status; outputs are valid only on MG_OK,
 * except MG_ERR_NOT_CONVERGED, which still writes the best phi (and U) and the
 * stats.  No exception or signal crosses the ABI.  mg_last_error() returns a
 * thread-local message for the last failure.
 *
 * Streams and threading: all work of a handle is enqueued on the handle's CUDA
 * stream.  mg_solve/mg_project synchronise that stream (residual norms are read
 * back to decide convergence) and only that stream.  A handle must not be used
 * from two host threads at once (MG_ERR_BUSY).
 */
#ifndef MGPROJ_MG_H
#define MGPROJ_MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,      /* bad pointer, size, boundary pairing, option */
    MG_ERR_OOM = 2,              /* device allocation failed or workspace too small */
    MG_ERR_CUDA = 3,             /* a CUDA runtime call failed (see mg_last_error) */
    MG_ERR_NOT_CONVERGED = 4,    /* iteration cap or round-off floor reached above tol */
    MG_ERR_DIVERGED = 5,         /* NaN/Inf or a growing residual */
    MG_ERR_INCOMPATIBLE_RHS = 6, /* reserved: singular problem with incompatible data */
    MG_ERR_TIMEOUT = 7,          /* a bounded wait expired */
    MG_ERR_BUSY = 8,             /* the handle is in use by another thread */
    MG_ERR_UNSUPPORTED = 9       /* grid does not coarsen to a dense-solvable size, etc. */
} mg_status;

typedef enum { MG_BC_PERIODIC = 0, MG_BC_NEUMANN = 1, MG_BC_DIRICHLET = 2 } mg_bc_kind;
typedef enum { MG_LOC_CELL = 0, MG_LOC_NODAL = 1 } mg_location;
typedef enum { MG_PREC_FP64 = 0, MG_PREC_MIXED = 1 } mg_precision;

/* Grid: dim 2 or 3; n[d] cells per axis (n[2] = 1 in 2-D); h[d] spacing (> 0).
 * The nodal discretisation requires h[0] = h[1] (= h[2]). */
typedef struct {
    int dim;
    int n[3];
    double h[3];
    int loc; /* mg_location */
} mg_geometry;

/* lo[d] / hi[d]: mg_bc_kind of the low / high face of axis d.  Periodic must be
 * paired; entries for axes >= dim are ignored. */
typedef struct {
    int lo[3];
    int hi[3];
} mg_bc;

/* Coefficient sigma = beta0/rho (Eq. 6), cell-centred, device, required, > 0.
 * face[d]: optional explicit MAC face coefficients (device, face layout); when
 * all are NULL the library uses the harmonic mean of the adjacent sigma
 * (boundary faces: the interior sigma; periodic: the mean across the wrap).
 * Ignored for the nodal discretisation.  Copied into the hierarchy: the caller
 * may free them after the call returns (and the stream has progressed). */
typedef struct {
    const double* sigma;
    const double* face[3];
} mg_coeff;

/* beta0 of Eq. 5 at cell centres (both projections) and at face centres (MAC
 * only: it divides the face update).  Device pointers. */
typedef struct {
    const double* cell;
    const double* face[3];
} mg_beta0;

/* Solver options; mg_default_options() fills sensible values.
 *   prec          MG_PREC_FP64: FP64 V-cycles throughout.
 *                 MG_PREC_MIXED: FP32 smoothing, restriction, prolongation and
 *                 coarse levels inside an FP64 iterative-refinement loop that
 *                 recomputes the fine residual and the update in FP64; the
 *                 coarsest dense solve is FP64 in both modes.
 *   nu1, nu2      pre/post smoothing sweeps (red-black Gauss-Seidel for cells,
 *                 damped Jacobi for nodes)
 *   max_iters     cap on V-cycles (FP64) or refinement steps (mixed)
 *   coarsest_max  stop coarsening once a level has at most this many cells (default 8)
 *   interp_order  cell prolongation: 0 piecewise constant, 1 linear
 *   omega         nodal Jacobi damping
 *   stream        cudaStream_t (NULL: the legacy default stream)
 *   flags         MG_FLAG_* bits (0 by default)
 *   inner_cycles  mixed precision: FP32 V-cycles per FP64 refinement step
 *                 (0: automatic -- three, or the fewest (one or two) that the
 *                 last step's rate per V-cycle predicts to bring the residual
 *                 below half the tolerance; the graph path decides this on the
 *                 device with the same rule) */
typedef struct {
    int prec;
    int nu1;
    int nu2;
    int max_iters;
    int coarsest_max;
    int interp_order;
    double omega;
    void* stream;
    int flags;
    int inner_cycles;
} mg_options;

/* flags: run every smoothing sweep with the plain one-thread-per-cell kernels,
 * never the tiled or vectorised ones (same arithmetic, slower; for testing). */
#define MG_FLAG_NO_FUSED 1
/* flags: drive the iterations from the host (one scalar read-back per
 * iteration) instead of the graph-resident loop (same decisions, same phi).
 * The host loop is also used while mg_prof_enable(1) is in effect. */
#define MG_FLAG_NO_GRAPH 2
/* flags: FP32 cell levels sweep with the shared-memory pipelined one-launch
 * kernel (red and black of a sweep in one pass over memory) instead of two
 * vectorised colour passes (same arithmetic). */
#define MG_FLAG_SWEEP_PIPE 4
/* flags (mixed precision): at mg_setup, time the candidate smoother kernels of
 * every FP32 level -- the vectorised passes with 8, 16 or 32 quads per block
 * row and the shared-memory pipelined or tiled kernel -- and keep the fastest.
 * All candidates compute the same arithmetic.  Choices are cached per grid and
 * boundary kinds for the process; mg_smoother_kind reports them.  The timing
 * synchronises the handle's stream during mg_setup. */
#define MG_FLAG_AUTOTUNE 8
/* flags: solves ignore phi's input and start from phi = 0; the first residual
 * is then f itself and costs no operator application (one FP64 residual fewer
 * per solve).  phi is still written with the solution. */
#define MG_FLAG_ZERO_GUESS 16
/* flags: FP32 3-D cell levels with 32 <= nx <= 256, nx % 4 == 0, ny % 4 == 0
 * and z not periodic sweep with the one-pass kernel whose operands are staged
 * in shared memory by bulk asynchronous (TMA) copies: red and black of a sweep
 * in one pass over memory (same arithmetic).  A stage copy that does not
 * complete within about two seconds makes the solve return MG_ERR_CUDA. */
#define MG_FLAG_SWEEP_TMA 32
/* flags (mixed precision, 3-D cell grids of at least 2^14 cells, z not
 * periodic): run each leg of a V-cycle on the finest level -- the nu1 sweeps
 * with the residual restriction, and the prolongation with the nu2 sweeps --
 * as ONE persistent launch whose colour passes are pipelined through L2 (same
 * results as the pass-by-pass kernels, which are the default).  A pipelined
 * pass that waits for its predecessor longer than about a second makes the
 * solve return MG_ERR_CUDA. */
#define MG_FLAG_CELL_PIPE 64
/* flags: in mg_solve_batch / mg_project_batch, run this handle's solve as its
 * own branch of the batch graph.  By default, when every solve of a batch is a
 * 3-D mixed-precision cell solve with linear prolongation and automatic inner
 * cycles (and the same nu1, nu2), the solves share one iteration loop whose
 * steps -- each colour pass, restriction and prolongation of "level l" of all
 * solves, their coarse ends, FP64 residuals, norms and updates -- are one
 * launch each, driven by tables of per-solve work items; solves that have
 * converged drop out of the launches.  Both forms give every solve the result
 * it has alone, bit for bit.  One handle with this flag makes the whole batch
 * use per-solve branches. */
#define MG_FLAG_BATCH_BRANCHES 128

/* Per-solve statistics.  rel_resid = ||f - L phi||_2/||f||_2 over the unknowns;
 * rel_constraint (projections only): MAC ||D(beta0 U) - beta0 S||/||beta0 S||
 * over cells, nodal ||D_N(beta0 U) - S_N||/||S_N|| over unknown nodes (a
 * diagnostic: the nodal projection is approximate).  ms: wall time of the call.
 * iters: refinement steps (mixed) or V-cycles (FP64); vcycles: V-cycles run. */
typedef struct {
    int iters;
    double rel_resid;
    double rel_constraint;
    double rhs_norm;
    double src_norm;
    double ms;
    int status;
    int vcycles;
} mg_stats;

typedef struct mg_handle mg_handle;

/* Fill *opt with defaults (mixed precision, V(2,2), linear interpolation).  The
 * paper names multigrid for the projections (S3) but none of its parameters;
 * these defaults are this library's. */
void mg_default_options(mg_options* opt);

/* Device bytes that mg_setup needs for this problem (hierarchy, work arrays,
 * dense coarsest inverse, reduction scratch).  Used for admission control.  No
 * counterpart in the paper (its solver ran on the host, S4); the hierarchy sized
 * here is the one S3's multigrid needs.  MG_ERR_INVALID_ARG for a null or
 * invalid argument, MG_ERR_UNSUPPORTED for a grid that does not coarsen. */
mg_status mg_hierarchy_bytes(const mg_geometry* geom, const mg_bc* bc, const mg_options* opt, size_t* bytes);

/* Build a resident multigrid hierarchy for the projection solves of S3 (the
 * pressure projections are solved by multigrid): the coefficient sigma = beta0/rho
 * of Eq. 6 (beta0 from Eq. 5, the 1/rho from the gradient term of Eq. 2), face or
 * nodal coefficients on every level, FP32 copies in mixed mode, the dense inverse
 * of the coarsest operator.  workspace: optional caller-owned device buffer of at least
 * mg_hierarchy_bytes() bytes (e.g. from the PyTorch caching allocator); NULL
 * makes the library cudaMalloc its own, freed by mg_destroy.  The handle owns
 * nothing else on the device. */
mg_status mg_setup(const mg_coeff* coeff, const mg_geometry* geom, const mg_bc* bc, const mg_options* opt,
                   void* workspace, size_t workspace_bytes, mg_handle** out);

/* Recompute every level's coefficients from new sigma = beta0/rho (Eq. 6; the
 * base state and density change from one time step to the next, S2-S3) on the
 * same grid, in place.  Asynchronous on the handle's stream. */
mg_status mg_update_coeff(mg_handle* h, const mg_coeff* coeff);

/* Solve L phi = rhs, the elliptic problem of the projection (S3: multigrid
 * V-cycles; L = div(sigma grad) discretised as above), to
 * ||rhs - L phi|| <= tol ||rhs||.  rhs: device, unknown
 * layout (cells or nodes; Dirichlet nodes ignored).  phi: device, in: initial
 * guess, out: solution (Dirichlet nodes set to 0).  stats may be NULL. */
mg_status mg_solve(mg_handle* h, const double* rhs, double* phi, double tol, mg_stats* stats);

/* Projection enforcing the constraint div(beta0 U) = beta0 S of Eq. 6 (S2, with
 * dp0/dt = 0) by the projection method of S3: f = D(beta0 U) - beta0 S, solve
 * L phi = f by multigrid to tol, update U <- U - (sigma/beta0) G phi in place (the
 * gradient form -(beta0/rho) grad(pi/beta0) of Eq. 2), report the constraint.  MAC: U[d] face arrays, beta0->face required;
 * the constraint after the update equals the solver residual, and the solve
 * stops when ||f - L phi|| <= tol * min(||f||, ||beta0 S||), so that
 * ||D(beta0 U) - beta0 S|| <= tol ||beta0 S|| holds as well.  Nodal: U[d] cell
 * arrays (approximate projection: the constraint is reported only).  phi:
 * optional device output (and initial guess) of the solution; NULL uses an
 * internal buffer started from zero. */
mg_status mg_project(mg_handle* h, double* const U[3], const mg_beta0* beta0, const double* S, double* phi,
                     double tol, mg_stats* stats);

/* Right-hand side of the projection system (Eq. 6: the divergence of beta0 U
 * minus beta0 S) into a caller buffer f
 * (device, unknown layout: cells for MAC, nodes for nodal):
 *   MAC    f = D(beta0 U) - beta0 S     (beta0->face required)
 *   nodal  f = D_N(beta0 U) - S_N       (Dirichlet nodes 0)
 * with the mean removed when the problem is singular.  Synchronises the
 * handle's stream. */
mg_status mg_rhs(mg_handle* h, const double* const U[3], const mg_beta0* beta0, const double* S, double* f);

/* Base state on the device (Eq. 5).  beta0 on a radial grid from tabulated
 * p0 > 0 (device, nr values, increasing radius), Gamma1 per point (device, or
 * NULL to use gamma1_const) and rho0 at the first point:
 *   beta0_0 = rho0_base,
 *   beta0_{k+1} = rho0_base exp( sum_{m<=k} (1/2)(1/Gamma1_m + 1/Gamma1_{m+1}) (ln p0_{m+1} - ln p0_m) ),
 * the trapezoid rule for the integral of (1/Gamma1) d(ln p0) = dp0/dr / (Gamma1 p0) dr of
 * Eq. 5 (exact when Gamma1 is constant).  beta0: device, nr values.  Asynchronous on stream. */
mg_status mg_base_state_beta0(const double* p0, const double* gamma1, double gamma1_const, double rho0_base, int nr,
                              double* beta0, void* stream);

/* Map radial base-state tables (beta0_r, rho0_r: device, nr values at r0 + k dr)
 * onto the grid by linear interpolation (clamped to the end values): every cell
 * or face centre gets r = its distance to center (spherical != 0) or its height
 * (the last axis; center ignored).  Writes sigma = beta0/rho0 and beta0 at cell
 * centres and beta0 at the face centres of each axis (device arrays in the
 * layouts above; any output may be NULL).  Asynchronous on stream. */
mg_status mg_base_state_map(const mg_geometry* geom, int spherical, const double center[3], double r0, double dr,
                            int nr, const double* beta0_r, const double* rho0_r, double* sigma, double* beta0_cell,
                            double* const beta0_face[3], void* stream);

/* Solve count independent problems of the kind mg_solve solves (S3 multigrid;
 * batching many of them has no counterpart in the paper) -- any mix of grids,
 * precisions and locations, each handle at most once -- as ONE CUDA graph launch on the first
 * handle's stream: every solve is a branch of the graph with its own
 * device-side convergence loop, so the branches run concurrently and each
 * stops on its own tolerance tol[i].  The graph is captured on the first call
 * for a given ordered list of handles and cached until one of them is
 * destroyed.  rhs[i] and phi[i] follow mg_solve; stats may be NULL or hold
 * count entries (ms is the wall time of the whole batch).  Returns the first
 * non-OK status of the batch, MG_OK if every solve converged. */
mg_status mg_solve_batch(mg_handle* const* hs, const double* const* rhs, double* const* phi, const double* tol,
                         int count, mg_stats* stats);

/* count projections (as mg_project; any mix of grids, precisions and locations,
 * each handle at most once) whose elliptic solves run as ONE CUDA graph launch:
 * the right-hand side of each (Eq. 6, a2) is formed on its handle's own stream,
 * after whatever the caller has queued there (uploads of its inputs, a
 * coefficient update), the solves (S3 multigrid) run as the branches of one
 * graph on the first handle's stream, and each projection update (Eq. 2's
 * gradient form) and constraint is then applied on its handle's stream.
 * Batching projections has no counterpart in the paper; it serves many
 * independent requests at once.
 *   hs      count handles
 *   U       3 * count device pointers: U[3 i + d] is component d of entry i
 *           (faces for MAC, cells for nodal; unused entries of 2-D grids NULL);
 *           updated in place
 *   beta0   count entries, as for mg_project
 *   S       count device pointers (cells)
 *   phi     NULL, or count device pointers (each NULL: internal buffer)
 *   tol     count tolerances (> 0), as for mg_project
 *   stats   NULL or count entries (ms: wall time of the whole batch)
 * The graph of an ordered list of handles is captured on first use and cached
 * (at most 64 batch graphs; the least recently used is dropped first).
 * Returns the first non-OK status; synchronises the handles' streams. */
mg_status mg_project_batch(mg_handle* const* hs, double* const* U, const mg_beta0* beta0, const double* const* S,
                           double* const* phi, const double* tol, int count, mg_stats* stats);

/* Change the handle's stream (cudaStream_t; NULL: the legacy default stream).
 * No counterpart in the paper.  Work already enqueued stays on the old stream:
 * synchronise it first if the new stream does not wait for it.
 * MG_ERR_INVALID_ARG for a null handle. */
mg_status mg_set_stream(mg_handle* h, void* stream);

/* Concurrent batched loops (section 3's V-cycles of many independent solves):
 * a batch whose solves share batched loops (see MG_FLAG_BATCH_BRANCHES) is
 * split into this many groups of about equal total cells, each group one
 * lockstep loop, the groups concurrent branches of the batch graph, so one
 * group's FP64 residuals and latency-bound small levels overlap another's
 * bandwidth-bound finest levels.  0 (the default) means one group, which
 * measured fastest.  Results do not depend on it.  Takes effect for batch
 * graphs built afterwards (they are cached per list of handles and setting).
 * MG_ERR_INVALID_ARG outside 0 .. 64. */
mg_status mg_set_batch_groups(int groups);

/* out = L phi with the FP64 fine-level operator of the projection system (S3,
 * Eq. 6's elliptic operator; diagnostics and tests).  Device arrays in the
 * unknown layout; synchronises the handle's stream. */
mg_status mg_apply(mg_handle* h, const double* phi, double* out);

/* Free the handle (and its workspace when the library allocated it).  No
 * counterpart in the paper.  Null is ignored. */
void mg_destroy(mg_handle* h);

/* Static text naming a status (never NULL; "unknown status" for other values),
 * and the calling thread's message for its last failing call ("" if none).
 * No counterpart in the paper. */
const char* mg_strerror(mg_status s);
const char* mg_last_error(void);

/* Live per-kernel timing (diagnostics, used by the benchmark's roofline).
 * mg_prof_enable(1) clears the record and starts bracketing the launches of
 * the kernels below with pairs of CUDA events on the launching stream: one
 * pair per launch, or per run of consecutive launches of one class (the colour
 * passes or sweeps of one smoothing step), which then counts as that many
 * launches (solves use the host-driven loop meanwhile: a graph replay cannot
 * be bracketed per launch); mg_prof_enable(0) stops.  mg_prof_query (call
 * after the stream has been synchronised) returns, for one kernel class, the
 * summed event time, the launch count and the summed ALGORITHMIC bytes and
 * FP64 flops of those launches (what the method must move and compute, see
 * each class).  Returns MG_ERR_INVALID_ARG for an unknown class.  Recording
 * stops silently after 65536 brackets. */
typedef enum {
    MG_PROF_CELL_SMOOTH_FINE = 0, /* on the finest cell level, one colour pass of the
                                     vectorised or plain smoother (half a sweep: 2 words/cell),
                                     or one red-black sweep of the pipelined or TMA-staged
                                     smoother (phi, f, sigma read, phi written: 4 words/cell) */
    MG_PROF_RESID64 = 1,          /* FP64 fine residual of a cell system (+ FP32 copy in mixed
                                     mode): phi, f, sigma in FP64 (+ r in FP32) per cell;
                                     15 FP64 flops per cell (6 face FMAs, the diagonal FMA,
                                     one subtraction) */
    MG_PROF_NODE_SMOOTH_FINE = 2, /* one Jacobi sweep on the finest nodal level: phi, f, sigma read, phi written */
    MG_PROF_CELL_RESTRICT_FINE = 3, /* fused residual + restriction on the finest cell level:
                                       phi, f, sigma read, 1/2^dim word written per cell */
    MG_PROF_NODE_RESID64 = 4,     /* FP64 fine residual of a nodal system (+ FP32 copy):
                                     phi, f, sigma in FP64 (+ r in FP32) per node; FP64 flops
                                     per node of the form evaluated: 44 for the row assembled
                                     from 8 sigma (2-D, small 3-D grids), about 25.8 for the
                                     sum-factorised 3-D form (edge sigma sums set up once) */
    MG_PROF_CELL_PIPE_DOWN = 5,   /* down leg of a V-cycle on the finest cell level as one
                                     pipelined launch: nu1 sweeps (4 words/cell each) and the
                                     residual + restriction (3 + 1/8 words/cell) */
    MG_PROF_CELL_PIPE_UP = 6,     /* up leg as one pipelined launch: the prolongation fused
                                     into the first of nu2 sweeps (4 + 1/8 words/cell), 4 words
                                     per further sweep */
    /* the batched loop of mg_solve_batch / mg_project_batch (host-driven while
     * profiling): one launch each, over every solve with work in that step */
    MG_PROF_BATCH_SMOOTH = 7,     /* a colour pass of the finest level step (level 0 of every
                                     solve): 2 words per cell */
    MG_PROF_BATCH_RESTRICT = 8,   /* residual + restriction of one level step: 3 + 1/8 words per fine cell */
    MG_PROF_BATCH_PROLONG = 9,    /* prolongation + correction of one level step: x read and
                                     written, 1/8 word of coarse x per fine cell */
    MG_PROF_BATCH_COARSE = 10,    /* the solves' coarse ends (one CTA each; latency-bound, no bytes counted) */
    MG_PROF_BATCH_RESID64 = 11,   /* FP64 residuals and norms of the solves: 15 FP64 flops per cell */
    MG_PROF_BATCH_SMOOTH_COARSE = 12, /* a colour pass of a coarser level step: 2 words per cell */
    MG_PROF_COUNT = 13
} mg_prof_kernel;

/* Allocation-free check of the MAC constraint.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at the
 * moment they need the answer -- code running while a CUDA graph is being
 * captured, or a process whose device-memory budget is already handed out --
 * and it calls no cudaMalloc, cudaFree or allocating library routine.  For MAC
 * face velocities U it writes, for v = D(beta0 U) - beta0 S over the cells,
 *   out[0] = sum v,   out[1] = sum (beta0 S)^2,   out[2] = sum v^2
 * (the relative constraint reported by mg_project is sqrt(out[2] / out[1])).
 *   geom    cell grid (loc MG_LOC_CELL), at most MG_NOALLOC_MAX_CELLS cells;
 *           larger grids return MG_ERR_UNSUPPORTED (the scratch holds one
 *           partial sum per 2048 cells)
 *   U, beta0, S   device arrays as for mg_project (beta0->face required)
 *   out     device, 3 doubles, written by the call
 *   stream  cudaStream_t (NULL: the legacy default stream); asynchronous
 * Its reduction scratch is a fixed device array of 3 * MG_NOALLOC_MAX_CELLS /
 * 2048 doubles (384 KiB) that every GPU loading the library holds until the
 * process exits.  Each call overwrites every slot it reads, so nothing needs
 * clearing between calls; but all calls share that one array, so calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The first call on a device looks up the array's
 * device address (once per device, with that device current): make that first
 * call before any stream capture.  The address is kept for the life of the
 * process, so a cudaDeviceReset of that device after the first call is not
 * supported (later calls would write through the stale address). */
#define MG_NOALLOC_MAX_CELLS (1 << 25)
mg_status mg_mac_constraint_noalloc(const mg_geometry* geom, const double* const U[3], const mg_beta0* beta0,
                                    const double* S, double* out, void* stream);

/* One time step around the two projections (S2-S3; NEXT to the projection
 * path), in the order of the method:
 *   1. face velocities Uadv from the cell velocities U (mean of the two cells
 *      beside a face; periodic faces wrap; wall faces 0; outflow faces the
 *      interior cell's value),
 *   2. MAC projection of Uadv (mg_project on mac, phi internal),
 *   3. Unew = U - dt (Uadv . grad) U with upwind face values (zero gradient
 *      where the upwind cell is outside a boundary), plus dt times the rotation
 *      accelerations of mg_rotation_forces when omega is not NULL,
 *   4. nodal projection of Unew (mg_project on nodal, phi internal).
 *   mac, nodal  handles of the same grid, boundary kinds and stream (loc
 *               MG_LOC_CELL and MG_LOC_NODAL)
 *   U           device, cell-centred components of U^n (not modified)
 *   Unew        device, cell-centred output U^{n+1}; must not alias U
 *   Uadv        device, face arrays: scratch, and on return the projected face
 *               velocities
 *   beta0       cell and face values (both required); S: cells
 *   dt >= 0; omega (3 doubles, host) or NULL; center (host) when centrifugal
 *   tol         for both projections; stats: NULL or 2 entries (MAC, nodal)
 * Returns the first failing status (MG_ERR_NOT_CONVERGED still completes the
 * step with the best phi); synchronises the handles' stream. */
mg_status mg_step(mg_handle* mac, mg_handle* nodal, const double* const U[3], double* const Unew[3],
                  double* const Uadv[3], const mg_beta0* beta0, const double* S, double dt, const double omega[3],
                  const double center[3], int centrifugal, double tol, mg_stats stats[2]);

/* Rotation (S5, the rotating form of the velocity equation): at every cell
 * centre x, with r = x - center, accumulate the Coriolis and (if centrifugal
 * is nonzero) centrifugal accelerations
 *     F[d] += alpha * ( -2 Omega x U  -  Omega x (Omega x r) )_d ,   d < dim.
 *   geom     cell grid (its loc is ignored); 2-D grids use the in-plane
 *            components (U_z = 0, r_z = 0)
 *   omega    host, 3 doubles: the angular velocity
 *   center   host, 3 doubles: the rotation axis passes through it (may be NULL
 *            when centrifugal is 0)
 *   alpha    scale (1: the acceleration; dt: the explicit velocity update)
 *   U, F     device, cell-centred components, x-fastest; F may alias U
 *   stream   cudaStream_t (NULL: legacy default stream); asynchronous
 * MG_ERR_INVALID_ARG for null or missing arguments. */
mg_status mg_rotation_forces(const mg_geometry* geom, const double omega[3], const double center[3], int centrifugal,
                             double alpha, const double* const U[3], double* const F[3], void* stream);

/* Precision conversions of the mixed-precision path, exposed so that they can
 * be checked against the hardware conversions.  The paper has no counterpart.
 * mg_convert_f64_to_f32 rounds to nearest, ties to even; mg_convert_f32_to_f64
 * is exact.  x, y: device arrays of n elements (no overlap); stream as
 * cudaStream_t (NULL: legacy default stream); asynchronous.  Both are
 * computed with 32-bit integer operations for normal results and zeros (the
 * hardware conversion for the rest), as in the library's FP64 kernels.
 * MG_ERR_INVALID_ARG for null pointers with n > 0. */
mg_status mg_convert_f64_to_f32(const double* x, float* y, size_t n, void* stream);
mg_status mg_convert_f32_to_f64(const float* x, double* y, size_t n, void* stream);
/* y = x * 2^shift rounded to binary32, the exponent shift folded into the
 * conversion (how the FP64 residual kernels scale the residual by a power of
 * two near 1/||f|| without an FP64 multiply); -1022 <= shift <= 1023, else
 * MG_ERR_INVALID_ARG; arguments otherwise as above. */
mg_status mg_convert_f64_to_f32_pow2(const double* x, float* y, size_t n, int shift, void* stream);
/* y = 1/x as the library's FP64 kernels compute it where they divide (face
 * coefficients, projection updates): Newton's method from a binary32 estimate,
 * within about one ulp of the quotient; arguments as above. */
mg_status mg_reciprocal_f64(const double* x, double* y, size_t n, void* stream);

/* The smoother kernel a level uses: 0 the default rule, 1..3 the vectorised
 * passes with 8/16/32 quads per block row, 4 the shared-memory kernel, 5..7
 * (nodal levels) the vectorised passes with 8/16/32 quads per block row
 * marching four node planes per thread, 9..11 (nodal) the same marching eight
 * planes, 8 (cell levels) the TMA-staged one-pass sweep; -1 for a null handle
 * or a level out of range. */
int mg_smoother_kind(const mg_handle* h, int level);

/* FP64 throughput probe (measurement support; no counterpart in the paper).
 * Launches blocks x 256 threads, each running eight independent chains of iters
 * FP64 fused multiply-adds, on stream (cudaStream_t; NULL: the legacy default
 * stream), asynchronously, and stores the flop count of the launch (2 per FMA)
 * in *flops (host).  The caller times the launch with CUDA events on the same
 * stream; flops / time is the FP64 rate the solver's FP64 kernels are judged
 * against.  sink: device, one double, written only in a case that never occurs.
 * Reads no memory and changes no GPU setting.  MG_ERR_INVALID_ARG for
 * non-positive sizes or null pointers. */
mg_status mg_fp64_fma_probe(int blocks, int iters, double* sink, void* stream, double* flops);

void mg_prof_enable(int on);
/* Total number of CUDA kernels this library has launched in the process. */
long long mg_launch_count(void);
mg_status mg_prof_query(int kernel, double* total_ms, int* launches, double* bytes, double* flops);

#ifdef __cplusplus
}
#endif

#endif /* MGPROJ_MG_H */
