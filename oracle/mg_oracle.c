/*
 * mg_oracle.c -- FP64 CPU oracle for the variable-coefficient projection solve
 *
 *     div( (beta0/rho) grad phi ) = div(beta0 U) - beta0 S          (Eq. 6, S2;
 *                                                                    dp0/dt = 0)
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * reference that the GPU path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * The paper (S3) states only that the pressure projections are solved with
 * multigrid and that a second-order projection method enforces the constraint
 * of Eq. 6; it gives no discretisation.  The readings taken here are:
 *
 *   MAC / cell-centred system
 *     (L phi)_c = sum_d h_d^-2 [ B_{c+1/2}(phi_{c+e_d}-phi_c) - B_{c-1/2}(phi_c-phi_{c-e_d}) ]
 *     B on faces = harmonic mean of the two adjacent sigma = beta0/rho
 *     (boundary face: the interior sigma; periodic: harmonic mean across the wrap)
 *     BCs: periodic wraps; Neumann (wall) drops the flux; Dirichlet phi=0 on the
 *     face uses the ghost value -phi_c.
 *     D(V)_c = sum_d h_d^-1 (V_{c+1/2} - V_{c-1/2});  (G phi)_f = (phi_+ - phi_-)/h
 *     so that L = D B G holds exactly.  Projection: U_f -= (B_f/beta0_f) (G phi)_f.
 *
 *   Nodal system (Q1 finite elements, sigma constant per cell)
 *     (L phi)_I = -(1/V) sum_{cells c touching I} sigma_c sum_{J in c} K_c(I,J) phi_J
 *     with the Q1 element stiffness K_c built as the tensor product of the 1-D
 *     stiffness [[1,-1],[-1,1]]/h and mass [[1/3,1/6],[1/6,1/3]] h, V = prod h.
 *     D_N(V)_I = sum_{c} sum_d s_d(c,I) V_{d,c} / (2^(d-1) h_d)   (cells inside
 *     the domain only: natural boundary condition), lumped source
 *     sum_c g_c / 2^d, G_N(phi)_{d,c} = sum_{J in c} s_d(J,c) phi_J / (2^(d-1) h_d).
 *     Dirichlet nodes are fixed at 0 and are not unknowns; periodic nodes are
 *     identified.  Projection: U_c -= (sigma_c/beta0_c) G_N(phi)_c (approximate).
 *
 *   Singular problems (no Dirichlet boundary): f <- f - mean(f), and the
 *   returned phi has zero mean over the unknowns.
 *
 * Solvers: (1) dense LU with partial pivoting on the assembled matrix (the
 * plain definition, tiny grids; bordered [A 1; 1^T 0] when singular);
 * (2) V(2,2) multigrid with LEXICOGRAPHIC Gauss-Seidel, cell-mean restriction
 * and piecewise-constant prolongation (cell) / full weighting and trilinear
 * prolongation (nodal), rediscretised coarse operators and a dense LU bottom
 * solve, iterated to the FP64 round-off floor.
 *
 * Array layout: x fastest.  Cells (nz,ny,nx); x faces (nz,ny,nx+1);
 * y faces (nz,ny+1,nx); z faces (nz+1,ny,nx); nodes (Nz,Ny,Nx) with
 * N_d = n_d on periodic axes (node n == node 0) and n_d + 1 otherwise.
 * 2-D problems use nz = 1 and no z faces.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The CPU-baseline build (mg_oracle_omp.c) compiles this file with
 * ORC_PARALLEL: loops whose iterations write only their own element run on
 * OpenMP threads, and the multigrid smoothers are replaced by colour-ordered
 * ones (declared below, defined there).  The oracle itself is built without
 * it: ORC_PARALLEL_FOR is then empty and the smoothers are the lexicographic
 * sweeps of this file. */
#ifdef ORC_PARALLEL
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PARALLEL_FOR
#endif

enum { BC_PERIODIC = 0, BC_NEUMANN = 1, BC_DIRICHLET = 2 };

typedef struct {
    int dim;
    int n[3];
    double h[3];
    int bclo[3];
    int bchi[3];
} orc_grid;

typedef struct {
    int iters;
    double relres;      /* ||f - L phi||_2 / ||f||_2 */
    double constraint;  /* post-projection constraint, see the project routines */
    double rhs_norm;    /* ||f||_2 */
    double src_norm;    /* ||beta0 S||_2 (MAC) or ||S_N||_2 (nodal) */
} orc_stats;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static long ncells(const orc_grid* g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static long cell_index(const orc_grid* g, const int c[3])
{
    return ((long)c[2] * g->n[1] + c[1]) * g->n[0] + c[0];
}

/* face array of direction d has n_d + 1 entries along d */
static long face_index(const orc_grid* g, int d, const int f[3])
{
    int m[3] = { g->n[0], g->n[1], g->n[2] };
    m[d] += 1;
    return ((long)f[2] * m[1] + f[1]) * m[0] + f[0];
}

static long nfaces(const orc_grid* g, int d)
{
    long m[3] = { g->n[0], g->n[1], g->n[2] };
    m[d] += 1;
    return m[0] * m[1] * m[2];
}

static int is_singular(const orc_grid* g)
{
    for (int d = 0; d < g->dim; ++d)
        if (g->bclo[d] == BC_DIRICHLET || g->bchi[d] == BC_DIRICHLET) return 0;
    return 1;
}

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

/* ------------------------------------------------------------------------ */
/* dense LU with partial pivoting                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    double* a;  /* n*n, row major, holds L and U */
    int* piv;
} orc_lu;

static int lu_factor(orc_lu* lu)
{
    int n = lu->n;
    double* a = lu->a;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[(long)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(a[(long)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        lu->piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = a[(long)k * n + j];
                a[(long)k * n + j] = a[(long)p * n + j];
                a[(long)p * n + j] = t;
            }
        for (int i = k + 1; i < n; ++i) {
            double l = a[(long)i * n + k] / a[(long)k * n + k];
            a[(long)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[(long)i * n + j] -= l * a[(long)k * n + j];
        }
    }
    return 0;
}

static void lu_solve(const orc_lu* lu, double* x)
{
    int n = lu->n;
    const double* a = lu->a;
    for (int k = 0; k < n; ++k) {
        int p = lu->piv[k];
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) x[i] -= a[(long)i * n + j] * x[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) x[i] -= a[(long)i * n + j] * x[j];
        x[i] /= a[(long)i * n + i];
    }
}

static void lu_free(orc_lu* lu)
{
    free(lu->a);
    free(lu->piv);
    lu->a = NULL;
    lu->piv = NULL;
}

/* ======================================================================== */
/* MAC (cell-centred) system                                                 */
/* ======================================================================== */

/* Face coefficients from cell sigma: harmonic mean of the two neighbours. */
int orc_mac_faces(const orc_grid* g, const double* sigma, double* bx, double* by, double* bz)
{
    double* B[3] = { bx, by, bz };
    for (int d = 0; d < g->dim; ++d) {
        int f[3];
        for (f[2] = 0; f[2] < g->n[2] + (d == 2); ++f[2])
            for (f[1] = 0; f[1] < g->n[1] + (d == 1); ++f[1])
                for (f[0] = 0; f[0] < g->n[0] + (d == 0); ++f[0]) {
                    int lo[3] = { f[0], f[1], f[2] }, hi[3] = { f[0], f[1], f[2] };
                    lo[d] -= 1; /* cell on the low side of the face */
                    double v;
                    if (f[d] == 0 || f[d] == g->n[d]) {
                        if (g->bclo[d] == BC_PERIODIC) {
                            lo[d] = g->n[d] - 1;
                            hi[d] = 0;
                            v = harmonic(sigma[cell_index(g, lo)], sigma[cell_index(g, hi)]);
                        } else if (f[d] == 0) {
                            v = sigma[cell_index(g, hi)];
                        } else {
                            v = sigma[cell_index(g, lo)];
                        }
                    } else {
                        v = harmonic(sigma[cell_index(g, lo)], sigma[cell_index(g, hi)]);
                    }
                    B[d][face_index(g, d, f)] = v;
                }
    }
    return 0;
}

/* (L phi)_c at one cell, and the coefficient of phi_c in it (the diagonal). */
static double mac_row(const orc_grid* g, const double* const B[3], const double* phi,
                      const int c[3], double* diag)
{
    long ic = cell_index(g, c);
    double acc = 0.0, dg = 0.0;
    for (int d = 0; d < g->dim; ++d) {
        double ih2 = 1.0 / (g->h[d] * g->h[d]);
        /* high face */
        {
            int f[3] = { c[0], c[1], c[2] };
            f[d] += 1;
            double b = B[d][face_index(g, d, f)];
            if (c[d] == g->n[d] - 1) {
                if (g->bchi[d] == BC_PERIODIC) {
                    int nb[3] = { c[0], c[1], c[2] };
                    nb[d] = 0;
                    long inb = cell_index(g, nb);
                    if (inb != ic) { acc += b * ih2 * (phi[inb] - phi[ic]); dg -= b * ih2; }
                } else if (g->bchi[d] == BC_DIRICHLET) {
                    acc += b * ih2 * (-phi[ic] - phi[ic]);
                    dg -= 2.0 * b * ih2;
                }
            } else {
                int nb[3] = { c[0], c[1], c[2] };
                nb[d] += 1;
                acc += b * ih2 * (phi[cell_index(g, nb)] - phi[ic]);
                dg -= b * ih2;
            }
        }
        /* low face */
        {
            int f[3] = { c[0], c[1], c[2] };
            double b = B[d][face_index(g, d, f)];
            if (c[d] == 0) {
                if (g->bclo[d] == BC_PERIODIC) {
                    int nb[3] = { c[0], c[1], c[2] };
                    nb[d] = g->n[d] - 1;
                    long inb = cell_index(g, nb);
                    if (inb != ic) { acc -= b * ih2 * (phi[ic] - phi[inb]); dg -= b * ih2; }
                } else if (g->bclo[d] == BC_DIRICHLET) {
                    acc -= b * ih2 * (phi[ic] - (-phi[ic]));
                    dg -= 2.0 * b * ih2;
                }
            } else {
                int nb[3] = { c[0], c[1], c[2] };
                nb[d] -= 1;
                acc -= b * ih2 * (phi[ic] - phi[cell_index(g, nb)]);
                dg -= b * ih2;
            }
        }
    }
    if (diag) *diag = dg;
    return acc;
}

int orc_mac_apply(const orc_grid* g, const double* bx, const double* by, const double* bz,
                  const double* phi, double* out)
{
    const double* B[3] = { bx, by, bz };
    ORC_PARALLEL_FOR
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                int c[3] = { i, j, k };
                out[cell_index(g, c)] = mac_row(g, B, phi, c, NULL);
            }
    return 0;
}

/* D(V)_c = sum_d (V_{d,c+1/2} - V_{d,c-1/2}) / h_d */
int orc_mac_div(const orc_grid* g, const double* vx, const double* vy, const double* vz, double* out)
{
    const double* V[3] = { vx, vy, vz };
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                double acc = 0.0;
                for (int d = 0; d < g->dim; ++d) {
                    int fl[3] = { c[0], c[1], c[2] }, fh[3] = { c[0], c[1], c[2] };
                    fh[d] += 1;
                    acc += (V[d][face_index(g, d, fh)] - V[d][face_index(g, d, fl)]) / g->h[d];
                }
                out[cell_index(g, c)] = acc;
            }
    return 0;
}

/* f = D(beta0 U) - beta0 S (Eq. 6 with dp0/dt = 0); no mean removal here. */
int orc_mac_rhs(const orc_grid* g, const double* beta0_cell, const double* const beta0_face[3],
                const double* const U[3], const double* S, double* f)
{
    double* W[3] = { NULL, NULL, NULL };
    for (int d = 0; d < g->dim; ++d) {
        long m = nfaces(g, d);
        W[d] = (double*)malloc(sizeof(double) * m);
        for (long i = 0; i < m; ++i) W[d][i] = beta0_face[d][i] * U[d][i];
    }
    orc_mac_div(g, W[0], W[1], W[2], f);
    long N = ncells(g);
    for (long i = 0; i < N; ++i) f[i] -= beta0_cell[i] * S[i];
    for (int d = 0; d < g->dim; ++d) free(W[d]);
    return 0;
}

/* U_f -= (B_f / beta0_f) (G phi)_f, every face of every direction. */
int orc_mac_grad_update(const orc_grid* g, const double* const B[3], const double* const beta0_face[3],
                        const double* phi, double* const U[3])
{
    for (int d = 0; d < g->dim; ++d) {
        int f[3];
        double h = g->h[d];
        for (f[2] = 0; f[2] < g->n[2] + (d == 2); ++f[2])
            for (f[1] = 0; f[1] < g->n[1] + (d == 1); ++f[1])
                for (f[0] = 0; f[0] < g->n[0] + (d == 0); ++f[0]) {
                    int lo[3] = { f[0], f[1], f[2] }, hi[3] = { f[0], f[1], f[2] };
                    lo[d] -= 1;
                    double grad;
                    if (f[d] == 0 || f[d] == g->n[d]) {
                        if (g->bclo[d] == BC_PERIODIC) {
                            lo[d] = g->n[d] - 1;
                            hi[d] = 0;
                            grad = (phi[cell_index(g, hi)] - phi[cell_index(g, lo)]) / h;
                        } else {
                            int bc = (f[d] == 0) ? g->bclo[d] : g->bchi[d];
                            if (bc == BC_NEUMANN) {
                                grad = 0.0;
                            } else if (f[d] == 0) { /* phi = 0 on the face, cell at h/2 above */
                                grad = (phi[cell_index(g, hi)] - 0.0) / (0.5 * h);
                            } else {
                                grad = (0.0 - phi[cell_index(g, lo)]) / (0.5 * h);
                            }
                        }
                    } else {
                        grad = (phi[cell_index(g, hi)] - phi[cell_index(g, lo)]) / h;
                    }
                    long i = face_index(g, d, f);
                    U[d][i] -= B[d][i] / beta0_face[d][i] * grad;
                }
    }
    return 0;
}

/* --- dense direct solve of the MAC system ------------------------------- */

static int dense_solve_generic(long N, int singular,
                               void (*apply)(const void*, const double*, double*), const void* ctx,
                               const double* f, double* x)
{
    int n = (int)N + (singular ? 1 : 0);
    orc_lu lu;
    lu.n = n;
    lu.a = (double*)calloc((size_t)n * n, sizeof(double));
    lu.piv = (int*)malloc(sizeof(int) * n);
    double* e = (double*)calloc(N, sizeof(double));
    double* col = (double*)calloc(N, sizeof(double));
    /* assemble column j = L e_j */
    for (long j = 0; j < N; ++j) {
        e[j] = 1.0;
        apply(ctx, e, col);
        e[j] = 0.0;
        for (long i = 0; i < N; ++i) lu.a[i * n + j] = col[i];
    }
    if (singular) {
        for (long i = 0; i < N; ++i) { lu.a[i * n + N] = 1.0; lu.a[N * n + i] = 1.0; }
        lu.a[N * n + N] = 0.0;
    }
    int rc = lu_factor(&lu);
    if (rc == 0) {
        double* rhs = (double*)calloc(n, sizeof(double));
        for (long i = 0; i < N; ++i) rhs[i] = f[i];
        lu_solve(&lu, rhs);
        for (long i = 0; i < N; ++i) x[i] = rhs[i];
        free(rhs);
    }
    free(e);
    free(col);
    lu_free(&lu);
    return rc;
}

typedef struct {
    const orc_grid* g;
    const double* B[3];
} mac_ctx;

static void mac_apply_cb(const void* p, const double* x, double* y)
{
    const mac_ctx* c = (const mac_ctx*)p;
    orc_mac_apply(c->g, c->B[0], c->B[1], c->B[2], x, y);
}

static void remove_mean(double* v, long N)
{
    double s = 0.0;
    for (long i = 0; i < N; ++i) s += v[i];
    s /= (double)N;
    for (long i = 0; i < N; ++i) v[i] -= s;
}

static double norm2(const double* v, long N)
{
    double s = 0.0;
    for (long i = 0; i < N; ++i) s += v[i] * v[i];
    return sqrt(s);
}

/* Exact solution of L phi = f by LU.  f is made compatible (mean removed) when
 * the problem is singular; the solution then has zero mean. */
int orc_mac_solve_dense(const orc_grid* g, const double* bx, const double* by, const double* bz,
                        const double* f_in, double* phi)
{
    long N = ncells(g);
    int sing = is_singular(g);
    double* f = (double*)malloc(sizeof(double) * N);
    memcpy(f, f_in, sizeof(double) * N);
    if (sing) remove_mean(f, N);
    mac_ctx ctx = { g, { bx, by, bz } };
    int rc = dense_solve_generic(N, sing, mac_apply_cb, &ctx, f, phi);
    if (sing && rc == 0) remove_mean(phi, N);
    free(f);
    return rc;
}

/* --- MAC multigrid ------------------------------------------------------- */

#define ORC_MAX_LEVELS 24

typedef struct {
    orc_grid g;
    double* B[3];
    double* x;
    double* b;
    double* r;
} mac_level;

typedef struct {
    int nlev;
    mac_level lev[ORC_MAX_LEVELS];
    orc_lu bottom;
    int bottom_singular;
} mac_mg;

/* coarsen while every active axis is even and at least 4 cells, until the
 * level has at most 64 cells */
static int can_coarsen(const orc_grid* g, long max_bottom)
{
    if (ncells(g) <= max_bottom) return 0;
    for (int d = 0; d < g->dim; ++d)
        if (g->n[d] % 2 != 0 || g->n[d] < 4) return 0;
    return 1;
}

static void mac_coarse_faces(const orc_grid* gf, const double* const Bf[3], const orc_grid* gc,
                             double* const Bc[3])
{
    for (int d = 0; d < gc->dim; ++d) {
        int f[3];
        int nsub = 1 << (gc->dim - 1);
        for (f[2] = 0; f[2] < gc->n[2] + (d == 2); ++f[2])
            for (f[1] = 0; f[1] < gc->n[1] + (d == 1); ++f[1])
                for (f[0] = 0; f[0] < gc->n[0] + (d == 0); ++f[0]) {
                    /* the fine faces covering coarse face f: index 2 f along d,
                     * 2 f + {0,1} along the other active axes */
                    double s = 0.0;
                    for (int q = 0; q < nsub; ++q) {
                        int ff[3] = { 2 * f[0], 2 * f[1], (gc->dim == 3) ? 2 * f[2] : 0 };
                        int bit = 0;
                        for (int e = 0; e < gc->dim; ++e) {
                            if (e == d) continue;
                            ff[e] += (q >> bit) & 1;
                            ++bit;
                        }
                        s += Bf[d][face_index(gf, d, ff)];
                    }
                    Bc[d][face_index(gc, d, f)] = s / nsub;
                }
    }
}

static void mac_mg_free(mac_mg* mg)
{
    for (int l = 0; l < mg->nlev; ++l) {
        for (int d = 0; d < 3; ++d) free(mg->lev[l].B[d]);
        free(mg->lev[l].x);
        free(mg->lev[l].b);
        free(mg->lev[l].r);
    }
    lu_free(&mg->bottom);
}

static int mac_mg_build(mac_mg* mg, const orc_grid* g, const double* const B[3])
{
    memset(mg, 0, sizeof(*mg));
    mg->lev[0].g = *g;
    int l = 0;
    for (;;) {
        mac_level* L = &mg->lev[l];
        long N = ncells(&L->g);
        for (int d = 0; d < L->g.dim; ++d) {
            L->B[d] = (double*)malloc(sizeof(double) * nfaces(&L->g, d));
            if (l == 0) memcpy(L->B[d], B[d], sizeof(double) * nfaces(&L->g, d));
        }
        L->x = (double*)calloc(N, sizeof(double));
        L->b = (double*)calloc(N, sizeof(double));
        L->r = (double*)calloc(N, sizeof(double));
        if (l > 0) mac_coarse_faces(&mg->lev[l - 1].g, (const double* const*)mg->lev[l - 1].B, &L->g, L->B);
        if (!can_coarsen(&L->g, 64) || l + 1 >= ORC_MAX_LEVELS) break;
        orc_grid gc = L->g;
        for (int d = 0; d < gc.dim; ++d) { gc.n[d] /= 2; gc.h[d] *= 2.0; }
        mg->lev[l + 1].g = gc;
        ++l;
    }
    mg->nlev = l + 1;
    /* dense LU of the coarsest operator (bordered when singular) */
    mac_level* C = &mg->lev[mg->nlev - 1];
    long N = ncells(&C->g);
    int sing = is_singular(&C->g);
    int n = (int)N + (sing ? 1 : 0);
    mg->bottom.n = n;
    mg->bottom.a = (double*)calloc((size_t)n * n, sizeof(double));
    mg->bottom.piv = (int*)malloc(sizeof(int) * n);
    mg->bottom_singular = sing;
    double* e = (double*)calloc(N, sizeof(double));
    double* col = (double*)calloc(N, sizeof(double));
    for (long j = 0; j < N; ++j) {
        e[j] = 1.0;
        orc_mac_apply(&C->g, C->B[0], C->B[1], C->B[2], e, col);
        e[j] = 0.0;
        for (long i = 0; i < N; ++i) mg->bottom.a[i * n + j] = col[i];
    }
    if (sing) {
        for (long i = 0; i < N; ++i) { mg->bottom.a[i * n + N] = 1.0; mg->bottom.a[N * n + i] = 1.0; }
    }
    free(e);
    free(col);
    return lu_factor(&mg->bottom);
}

/* one lexicographic Gauss-Seidel sweep: x_c += (b_c - (Lx)_c) / L_cc */
static void mac_gs_lex(const mac_level* L)
{
    const double* B[3] = { L->B[0], L->B[1], L->B[2] };
    int c[3];
    for (c[2] = 0; c[2] < L->g.n[2]; ++c[2])
        for (c[1] = 0; c[1] < L->g.n[1]; ++c[1])
            for (c[0] = 0; c[0] < L->g.n[0]; ++c[0]) {
                double dg;
                double Lx = mac_row(&L->g, B, L->x, c, &dg);
                long i = cell_index(&L->g, c);
                if (dg != 0.0) L->x[i] += (L->b[i] - Lx) / dg;
            }
}

static void mac_residual(const mac_level* L)
{
    orc_mac_apply(&L->g, L->B[0], L->B[1], L->B[2], L->x, L->r);
    long N = ncells(&L->g);
    ORC_PARALLEL_FOR
    for (long i = 0; i < N; ++i) L->r[i] = L->b[i] - L->r[i];
}

/* coarse b = mean of the 2^dim fine residuals */
static void mac_restrict(const mac_level* F, mac_level* C)
{
    int nch = 1 << C->g.dim;
    ORC_PARALLEL_FOR
    for (int k = 0; k < C->g.n[2]; ++k)
        for (int j = 0; j < C->g.n[1]; ++j)
            for (int i = 0; i < C->g.n[0]; ++i) {
                int c[3] = { i, j, k };
                double s = 0.0;
                for (int q = 0; q < nch; ++q) {
                    int fc[3] = { 2 * c[0] + (q & 1), 2 * c[1] + ((q >> 1) & 1),
                                  (C->g.dim == 3) ? 2 * c[2] + ((q >> 2) & 1) : 0 };
                    s += F->r[cell_index(&F->g, fc)];
                }
                C->b[cell_index(&C->g, c)] = s / nch;
            }
}

/* fine x += coarse x, piecewise constant */
static void mac_prolong(const mac_level* C, mac_level* F)
{
    ORC_PARALLEL_FOR
    for (int k = 0; k < F->g.n[2]; ++k)
        for (int j = 0; j < F->g.n[1]; ++j)
            for (int i = 0; i < F->g.n[0]; ++i) {
                int c[3] = { i, j, k };
                int cc[3] = { c[0] / 2, c[1] / 2, (F->g.dim == 3) ? c[2] / 2 : 0 };
                F->x[cell_index(&F->g, c)] += C->x[cell_index(&C->g, cc)];
            }
}

#ifdef ORC_PARALLEL
static void mac_gs_colour(const mac_level* L);   /* red-black sweep, mg_oracle_omp.c */
#define ORC_MAC_SMOOTH mac_gs_colour
#else
#define ORC_MAC_SMOOTH mac_gs_lex
#endif

static void mac_vcycle(mac_mg* mg, int l)
{
    mac_level* L = &mg->lev[l];
    long N = ncells(&L->g);
    if (l == mg->nlev - 1) {
        int n = mg->bottom.n;
        double* rhs = (double*)calloc(n, sizeof(double));
        for (long i = 0; i < N; ++i) rhs[i] = L->b[i];
        lu_solve(&mg->bottom, rhs);
        for (long i = 0; i < N; ++i) L->x[i] = rhs[i];
        free(rhs);
        return;
    }
    for (int s = 0; s < 2; ++s) ORC_MAC_SMOOTH(L);
    mac_residual(L);
    mac_level* C = &mg->lev[l + 1];
    mac_restrict(L, C);
    memset(C->x, 0, sizeof(double) * ncells(&C->g));
    mac_vcycle(mg, l + 1);
    mac_prolong(C, L);
    for (int s = 0; s < 2; ++s) ORC_MAC_SMOOTH(L);
}

/* Multigrid solve to relative residual <= tol, or until the residual stops
 * falling (the FP64 round-off floor).  phi holds the initial guess on entry. */
int orc_mac_solve_mg(const orc_grid* g, const double* bx, const double* by, const double* bz,
                     const double* f_in, double* phi, double tol, int max_cycles, orc_stats* st)
{
    const double* B[3] = { bx, by, bz };
    mac_mg mg;
    if (mac_mg_build(&mg, g, B) != 0) { mac_mg_free(&mg); return -1; }
    long N = ncells(g);
    int sing = is_singular(g);
    mac_level* L = &mg.lev[0];
    memcpy(L->b, f_in, sizeof(double) * N);
    if (sing) remove_mean(L->b, N);
    memcpy(L->x, phi, sizeof(double) * N);
    double fn = norm2(L->b, N);
    if (fn == 0.0) fn = 1.0;
    mac_residual(L);
    double rel = norm2(L->r, N) / fn, best = rel;
    int it = 0, stall = 0;
    while (rel > tol && it < max_cycles) {
        mac_vcycle(&mg, 0);
        if (sing) remove_mean(L->x, N);
        mac_residual(L);
        rel = norm2(L->r, N) / fn;
        ++it;
        if (rel < 0.5 * best) { best = rel; stall = 0; }
        else if (++stall >= 3) break;
        if (rel < best) best = rel;
    }
    memcpy(phi, L->x, sizeof(double) * N);
    if (st) { st->iters = it; st->relres = rel; st->rhs_norm = norm2(L->b, N); }
    mac_mg_free(&mg);
    return 0;
}

/* Full MAC projection: faces from sigma, f = D(beta0 U) - beta0 S, solve,
 * U_f -= (B_f/beta0_f) G phi, then ||D(beta0 U) - beta0 S|| / ||beta0 S||.
 * dense != 0 selects the LU solve. */
int orc_mac_project(const orc_grid* g, const double* sigma, const double* beta0_cell,
                    const double* const beta0_face[3], double* const U[3], const double* S,
                    double* phi, double tol, int dense, orc_stats* st)
{
    long N = ncells(g);
    double* B[3] = { NULL, NULL, NULL };
    for (int d = 0; d < g->dim; ++d) B[d] = (double*)malloc(sizeof(double) * nfaces(g, d));
    orc_mac_faces(g, sigma, B[0], B[1], B[2]);
    double* f = (double*)malloc(sizeof(double) * N);
    orc_mac_rhs(g, beta0_cell, beta0_face, (const double* const*)U, S, f);
    orc_stats s0;
    memset(&s0, 0, sizeof(s0));
    int rc;
    if (dense) {
        rc = orc_mac_solve_dense(g, B[0], B[1], B[2], f, phi);
    } else {
        memset(phi, 0, sizeof(double) * N);
        rc = orc_mac_solve_mg(g, B[0], B[1], B[2], f, phi, tol, 200, &s0);
    }
    if (rc == 0) {
        /* relative residual of the (mean-removed when singular) system */
        double* r = (double*)malloc(sizeof(double) * N);
        double* fb = (double*)malloc(sizeof(double) * N);
        memcpy(fb, f, sizeof(double) * N);
        if (is_singular(g)) remove_mean(fb, N);
        orc_mac_apply(g, B[0], B[1], B[2], phi, r);
        for (long i = 0; i < N; ++i) r[i] = fb[i] - r[i];
        double fn = norm2(fb, N);
        s0.relres = norm2(r, N) / (fn > 0 ? fn : 1.0);
        s0.rhs_norm = fn;
        orc_mac_grad_update(g, (const double* const*)B, beta0_face, phi, U);
        orc_mac_rhs(g, beta0_cell, beta0_face, (const double* const*)U, S, r);
        for (long i = 0; i < N; ++i) fb[i] = beta0_cell[i] * S[i];
        s0.src_norm = norm2(fb, N);
        s0.constraint = norm2(r, N) / (s0.src_norm > 0 ? s0.src_norm : 1.0);
        free(r);
        free(fb);
    }
    if (st) *st = s0;
    free(f);
    for (int d = 0; d < g->dim; ++d) free(B[d]);
    return rc;
}

/* ======================================================================== */
/* Nodal (Q1 finite element) system                                          */
/* ======================================================================== */

static int node_extent(const orc_grid* g, int d)
{
    if (d >= g->dim) return 1;
    return g->bclo[d] == BC_PERIODIC ? g->n[d] : g->n[d] + 1;
}

static long nnodes(const orc_grid* g)
{
    return (long)node_extent(g, 0) * node_extent(g, 1) * node_extent(g, 2);
}

static long node_index(const orc_grid* g, const int p[3])
{
    return ((long)p[2] * node_extent(g, 1) + p[1]) * node_extent(g, 0) + p[0];
}

static int node_is_dirichlet(const orc_grid* g, const int p[3])
{
    for (int d = 0; d < g->dim; ++d) {
        if (g->bclo[d] == BC_DIRICHLET && p[d] == 0) return 1;
        if (g->bchi[d] == BC_DIRICHLET && p[d] == g->n[d]) return 1;
    }
    return 0;
}

/* the node at lattice position q (0..n_d along each axis) in storage, with
 * periodic wrap of position n_d to 0 */
static void node_wrap(const orc_grid* g, int q[3])
{
    for (int d = 0; d < g->dim; ++d)
        if (g->bclo[d] == BC_PERIODIC) q[d] = ((q[d] % g->n[d]) + g->n[d]) % g->n[d];
}

/* cell at lattice position c (may be -1 or n_d): returns 0 if outside the domain */
static int cell_wrap(const orc_grid* g, int c[3])
{
    for (int d = 0; d < g->dim; ++d) {
        if (c[d] < 0 || c[d] >= g->n[d]) {
            if (g->bclo[d] != BC_PERIODIC) return 0;
            c[d] = ((c[d] % g->n[d]) + g->n[d]) % g->n[d];
        }
    }
    return 1;
}

/* Q1 element stiffness between local corners a and b (bit d = position along
 * axis d), for a cell of size h: sum_d (V/h_d^2) k(a_d,b_d) prod_{e!=d} m(a_e,b_e)
 * with the unit-interval stiffness k = [[1,-1],[-1,1]] and mass m = [[1/3,1/6],[1/6,1/3]]. */
static double q1_stiffness(const orc_grid* g, int a, int b)
{
    double V = 1.0;
    for (int d = 0; d < g->dim; ++d) V *= g->h[d];
    double s = 0.0;
    for (int d = 0; d < g->dim; ++d) {
        double t = V / (g->h[d] * g->h[d]);
        for (int e = 0; e < g->dim; ++e) {
            int same = (((a >> e) & 1) == ((b >> e) & 1));
            if (e == d) t *= same ? 1.0 : -1.0;
            else t *= same ? (1.0 / 3.0) : (1.0 / 6.0);
        }
        s += t;
    }
    return s;
}

/* (L phi)_I and its diagonal coefficient at node p (not Dirichlet) */
static double nodal_row(const orc_grid* g, const double* sigma, const double* phi, const int p[3],
                        double* diag)
{
    double V = 1.0;
    for (int d = 0; d < g->dim; ++d) V *= g->h[d];
    int ncorner = 1 << g->dim;
    double acc = 0.0, dg = 0.0;
    long ip = node_index(g, p);
    /* the cells touching node p: p - 1 + corner offsets */
    for (int a = 0; a < ncorner; ++a) {
        /* node p is local corner a of cell c = p - a */
        int c[3] = { p[0], p[1], p[2] };
        for (int d = 0; d < g->dim; ++d) c[d] -= (a >> d) & 1;
        if (!cell_wrap(g, c)) continue;
        double sg = sigma[cell_index(g, c)];
        for (int b = 0; b < ncorner; ++b) {
            int q[3] = { p[0], p[1], p[2] };
            for (int d = 0; d < g->dim; ++d) q[d] += ((b >> d) & 1) - ((a >> d) & 1);
            double k = q1_stiffness(g, a, b);
            int qq[3] = { q[0], q[1], q[2] };
            node_wrap(g, qq);
            if (node_is_dirichlet(g, q)) continue;
            long iq = node_index(g, qq);
            acc -= sg * k * phi[iq] / V;
            if (iq == ip) dg -= sg * k / V;
        }
    }
    if (diag) *diag = dg;
    return acc;
}

int orc_nodal_apply(const orc_grid* g, const double* sigma, const double* phi, double* out)
{
    ORC_PARALLEL_FOR
    for (int k = 0; k < node_extent(g, 2); ++k)
        for (int j = 0; j < node_extent(g, 1); ++j)
            for (int i = 0; i < node_extent(g, 0); ++i) {
                int p[3] = { i, j, k };
                out[node_index(g, p)] = node_is_dirichlet(g, p) ? 0.0 : nodal_row(g, sigma, phi, p, NULL);
            }
    return 0;
}

/* D_N(V)_I for cell-centred V (3 arrays); 0 on Dirichlet nodes */
int orc_nodal_div(const orc_grid* g, const double* const V[3], double* out)
{
    int p[3];
    int ncorner = 1 << g->dim;
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0]) {
                double acc = 0.0;
                if (!node_is_dirichlet(g, p)) {
                    for (int a = 0; a < ncorner; ++a) {
                        int c[3] = { p[0], p[1], p[2] };
                        for (int d = 0; d < g->dim; ++d) c[d] -= (a >> d) & 1;
                        if (!cell_wrap(g, c)) continue;
                        long ic = cell_index(g, c);
                        for (int d = 0; d < g->dim; ++d) {
                            /* corner bit 0 => the cell lies on the + side of the node */
                            double s = ((a >> d) & 1) ? -1.0 : 1.0;
                            acc += s * V[d][ic] / ((double)(1 << (g->dim - 1)) * g->h[d]);
                        }
                    }
                }
                out[node_index(g, p)] = acc;
            }
    return 0;
}

/* lumped cell source: sum over cells touching I of g_c / 2^dim */
int orc_nodal_lump(const orc_grid* g, const double* gc, double* out)
{
    int p[3];
    int ncorner = 1 << g->dim;
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0]) {
                double acc = 0.0;
                if (!node_is_dirichlet(g, p)) {
                    for (int a = 0; a < ncorner; ++a) {
                        int c[3] = { p[0], p[1], p[2] };
                        for (int d = 0; d < g->dim; ++d) c[d] -= (a >> d) & 1;
                        if (!cell_wrap(g, c)) continue;
                        acc += gc[cell_index(g, c)] / (double)ncorner;
                    }
                }
                out[node_index(g, p)] = acc;
            }
    return 0;
}

/* G_N(phi)_{d,c} = sum_{J in c} s_d(J,c) phi_J / (2^(dim-1) h_d), Dirichlet nodes = 0 */
int orc_nodal_grad(const orc_grid* g, const double* phi, double* const G[3])
{
    int c[3];
    int ncorner = 1 << g->dim;
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                long ic = cell_index(g, c);
                for (int d = 0; d < g->dim; ++d) G[d][ic] = 0.0;
                for (int b = 0; b < ncorner; ++b) {
                    int q[3] = { c[0], c[1], c[2] };
                    for (int d = 0; d < g->dim; ++d) q[d] += (b >> d) & 1;
                    if (node_is_dirichlet(g, q)) continue;
                    int qq[3] = { q[0], q[1], q[2] };
                    node_wrap(g, qq);
                    double v = phi[node_index(g, qq)];
                    for (int d = 0; d < g->dim; ++d) {
                        double s = ((b >> d) & 1) ? 1.0 : -1.0;
                        G[d][ic] += s * v / ((double)(1 << (g->dim - 1)) * g->h[d]);
                    }
                }
            }
    return 0;
}

/* f_I = D_N(beta0 U)_I - lumped(beta0 S)_I, Dirichlet nodes 0; no mean removal */
int orc_nodal_rhs(const orc_grid* g, const double* beta0, const double* const U[3], const double* S,
                  double* f)
{
    long N = ncells(g);
    long M = nnodes(g);
    double* W[3] = { NULL, NULL, NULL };
    for (int d = 0; d < g->dim; ++d) {
        W[d] = (double*)malloc(sizeof(double) * N);
        for (long i = 0; i < N; ++i) W[d][i] = beta0[i] * U[d][i];
    }
    double* bs = (double*)malloc(sizeof(double) * N);
    for (long i = 0; i < N; ++i) bs[i] = beta0[i] * S[i];
    double* lump = (double*)malloc(sizeof(double) * M);
    orc_nodal_div(g, (const double* const*)W, f);
    orc_nodal_lump(g, bs, lump);
    for (long i = 0; i < M; ++i) f[i] -= lump[i];
    for (int d = 0; d < g->dim; ++d) free(W[d]);
    free(bs);
    free(lump);
    return 0;
}

/* mean over the unknown (non-Dirichlet) nodes */
static void nodal_remove_mean(const orc_grid* g, double* v)
{
    int p[3];
    double s = 0.0;
    long cnt = 0;
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0])
                if (!node_is_dirichlet(g, p)) { s += v[node_index(g, p)]; ++cnt; }
    s /= (double)cnt;
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0])
                if (!node_is_dirichlet(g, p)) v[node_index(g, p)] -= s;
}

static double nodal_norm2(const orc_grid* g, const double* v)
{
    int p[3];
    double s = 0.0;
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0])
                if (!node_is_dirichlet(g, p)) { double x = v[node_index(g, p)]; s += x * x; }
    return sqrt(s);
}

/* --- nodal dense solve ---------------------------------------------------- */

typedef struct {
    const orc_grid* g;
    const double* sigma;
    long* map;      /* unknown k -> storage index */
    long nunk;
    double* full;
    double* fout;
} nodal_ctx;

static void nodal_apply_cb(const void* p, const double* x, double* y)
{
    const nodal_ctx* c = (const nodal_ctx*)p;
    long M = nnodes(c->g);
    memset(c->full, 0, sizeof(double) * M);
    for (long k = 0; k < c->nunk; ++k) c->full[c->map[k]] = x[k];
    orc_nodal_apply(c->g, c->sigma, c->full, c->fout);
    for (long k = 0; k < c->nunk; ++k) y[k] = c->fout[c->map[k]];
}

static long nodal_unknown_map(const orc_grid* g, long* map)
{
    int p[3];
    long k = 0;
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0])
                if (!node_is_dirichlet(g, p)) map[k++] = node_index(g, p);
    return k;
}

int orc_nodal_solve_dense(const orc_grid* g, const double* sigma, const double* f_in, double* phi)
{
    long M = nnodes(g);
    nodal_ctx ctx;
    ctx.g = g;
    ctx.sigma = sigma;
    ctx.map = (long*)malloc(sizeof(long) * M);
    ctx.nunk = nodal_unknown_map(g, ctx.map);
    ctx.full = (double*)malloc(sizeof(double) * M);
    ctx.fout = (double*)malloc(sizeof(double) * M);
    int sing = is_singular(g);
    double* f = (double*)malloc(sizeof(double) * M);
    memcpy(f, f_in, sizeof(double) * M);
    if (sing) nodal_remove_mean(g, f);
    double* fu = (double*)malloc(sizeof(double) * ctx.nunk);
    double* xu = (double*)malloc(sizeof(double) * ctx.nunk);
    for (long k = 0; k < ctx.nunk; ++k) fu[k] = f[ctx.map[k]];
    int rc = dense_solve_generic(ctx.nunk, sing, nodal_apply_cb, &ctx, fu, xu);
    memset(phi, 0, sizeof(double) * M);
    if (rc == 0) {
        for (long k = 0; k < ctx.nunk; ++k) phi[ctx.map[k]] = xu[k];
        if (sing) nodal_remove_mean(g, phi);
    }
    free(ctx.map); free(ctx.full); free(ctx.fout); free(f); free(fu); free(xu);
    return rc;
}

/* --- nodal multigrid ------------------------------------------------------ */

typedef struct {
    orc_grid g;
    double* sigma;
    double* x;
    double* b;
    double* r;
} nodal_level;

typedef struct {
    int nlev;
    nodal_level lev[ORC_MAX_LEVELS];
    orc_lu bottom;
    long* map;
    long nunk;
} nodal_mg;

static void nodal_mg_free(nodal_mg* mg)
{
    for (int l = 0; l < mg->nlev; ++l) {
        free(mg->lev[l].sigma);
        free(mg->lev[l].x);
        free(mg->lev[l].b);
        free(mg->lev[l].r);
    }
    free(mg->map);
    lu_free(&mg->bottom);
}

static int nodal_mg_build(nodal_mg* mg, const orc_grid* g, const double* sigma)
{
    memset(mg, 0, sizeof(*mg));
    mg->lev[0].g = *g;
    int l = 0;
    for (;;) {
        nodal_level* L = &mg->lev[l];
        long N = ncells(&L->g), M = nnodes(&L->g);
        L->sigma = (double*)malloc(sizeof(double) * N);
        L->x = (double*)calloc(M, sizeof(double));
        L->b = (double*)calloc(M, sizeof(double));
        L->r = (double*)calloc(M, sizeof(double));
        if (l == 0) {
            memcpy(L->sigma, sigma, sizeof(double) * N);
        } else {
            /* coarse sigma = mean of the 2^dim fine cells */
            nodal_level* F = &mg->lev[l - 1];
            int c[3];
            int nch = 1 << L->g.dim;
            for (c[2] = 0; c[2] < L->g.n[2]; ++c[2])
                for (c[1] = 0; c[1] < L->g.n[1]; ++c[1])
                    for (c[0] = 0; c[0] < L->g.n[0]; ++c[0]) {
                        double s = 0.0;
                        for (int q = 0; q < nch; ++q) {
                            int fc[3] = { 2 * c[0] + (q & 1), 2 * c[1] + ((q >> 1) & 1),
                                          (L->g.dim == 3) ? 2 * c[2] + ((q >> 2) & 1) : 0 };
                            s += F->sigma[cell_index(&F->g, fc)];
                        }
                        L->sigma[cell_index(&L->g, c)] = s / nch;
                    }
        }
        if (!can_coarsen(&L->g, 64) || l + 1 >= ORC_MAX_LEVELS) break;
        orc_grid gc = L->g;
        for (int d = 0; d < gc.dim; ++d) { gc.n[d] /= 2; gc.h[d] *= 2.0; }
        mg->lev[l + 1].g = gc;
        ++l;
    }
    mg->nlev = l + 1;
    nodal_level* C = &mg->lev[mg->nlev - 1];
    long M = nnodes(&C->g);
    mg->map = (long*)malloc(sizeof(long) * M);
    mg->nunk = nodal_unknown_map(&C->g, mg->map);
    int sing = is_singular(&C->g);
    int n = (int)mg->nunk + (sing ? 1 : 0);
    mg->bottom.n = n;
    mg->bottom.a = (double*)calloc((size_t)n * n, sizeof(double));
    mg->bottom.piv = (int*)malloc(sizeof(int) * n);
    nodal_ctx ctx = { &C->g, C->sigma, mg->map, mg->nunk,
                      (double*)malloc(sizeof(double) * M), (double*)malloc(sizeof(double) * M) };
    double* e = (double*)calloc(mg->nunk, sizeof(double));
    double* col = (double*)calloc(mg->nunk, sizeof(double));
    for (long j = 0; j < mg->nunk; ++j) {
        e[j] = 1.0;
        nodal_apply_cb(&ctx, e, col);
        e[j] = 0.0;
        for (long i = 0; i < mg->nunk; ++i) mg->bottom.a[i * n + j] = col[i];
    }
    if (sing)
        for (long i = 0; i < mg->nunk; ++i) {
            mg->bottom.a[i * n + mg->nunk] = 1.0;
            mg->bottom.a[mg->nunk * n + i] = 1.0;
        }
    free(e); free(col); free(ctx.full); free(ctx.fout);
    return lu_factor(&mg->bottom);
}

static void nodal_gs_lex(const nodal_level* L)
{
    int p[3];
    for (p[2] = 0; p[2] < node_extent(&L->g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(&L->g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(&L->g, 0); ++p[0]) {
                if (node_is_dirichlet(&L->g, p)) continue;
                double dg;
                double Lx = nodal_row(&L->g, L->sigma, L->x, p, &dg);
                long i = node_index(&L->g, p);
                if (dg != 0.0) L->x[i] += (L->b[i] - Lx) / dg;
            }
}

static void nodal_residual(const nodal_level* L)
{
    orc_nodal_apply(&L->g, L->sigma, L->x, L->r);
    long M = nnodes(&L->g);
    ORC_PARALLEL_FOR
    for (long i = 0; i < M; ++i) L->r[i] = L->b[i] - L->r[i];
    int p[3];
    for (p[2] = 0; p[2] < node_extent(&L->g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(&L->g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(&L->g, 0); ++p[0])
                if (node_is_dirichlet(&L->g, p)) L->r[node_index(&L->g, p)] = 0.0;
}

/* 1-D linear-interpolation weight for a fine lattice offset o from the fine
 * position 2C of coarse node C: 1 at o = 0, 1/2 at o = +-1 */
static double interp_w(int o)
{
    return o == 0 ? 1.0 : 0.5;
}

/* fine lattice position q on axis d, wrapped on periodic axes; returns 0 when
 * q lies outside a non-periodic axis */
static int fine_pos(const orc_grid* gf, int d, int q, int* out)
{
    if (gf->bclo[d] == BC_PERIODIC) {
        *out = ((q % gf->n[d]) + gf->n[d]) % gf->n[d];
        return 1;
    }
    if (q < 0 || q > gf->n[d]) return 0;
    *out = q;
    return 1;
}

/* b_C = 2^-dim sum_J P_{JC} r_J  (R = 2^-dim P^T, full weighting) */
static void nodal_restrict(const nodal_level* F, nodal_level* C)
{
    int dim = C->g.dim;
    double scale = 1.0 / (double)(1 << dim);
    int noff = (dim == 3) ? 27 : 9;
    ORC_PARALLEL_FOR
    for (int k = 0; k < node_extent(&C->g, 2); ++k)
        for (int j = 0; j < node_extent(&C->g, 1); ++j)
            for (int i = 0; i < node_extent(&C->g, 0); ++i) {
                int pc[3] = { i, j, k };
                double s = 0.0;
                if (!node_is_dirichlet(&C->g, pc)) {
                    for (int t = 0; t < noff; ++t) {
                        int o[3] = { t % 3 - 1, (t / 3) % 3 - 1, (dim == 3) ? t / 9 - 1 : 0 };
                        int pf[3] = { 0, 0, 0 };
                        double w = 1.0;
                        int inside = 1;
                        for (int d = 0; d < dim; ++d) {
                            inside &= fine_pos(&F->g, d, 2 * pc[d] + o[d], &pf[d]);
                            w *= interp_w(o[d]);
                        }
                        if (inside) s += w * F->r[node_index(&F->g, pf)];
                    }
                }
                C->b[node_index(&C->g, pc)] = scale * s;
            }
}

/* x_J += sum_C P_{JC} x_C over fine non-Dirichlet nodes (trilinear) */
static void nodal_prolong(const nodal_level* C, nodal_level* F)
{
    int dim = F->g.dim;
    ORC_PARALLEL_FOR
    for (int k = 0; k < node_extent(&F->g, 2); ++k)
        for (int j = 0; j < node_extent(&F->g, 1); ++j)
            for (int i = 0; i < node_extent(&F->g, 0); ++i) {
                int pf[3] = { i, j, k };
                if (node_is_dirichlet(&F->g, pf)) continue;
                /* per axis: even position -> one coarse node, odd -> two halves */
                int lo[3] = { 0, 0, 0 }, cnt[3] = { 1, 1, 1 };
                for (int d = 0; d < dim; ++d) {
                    lo[d] = pf[d] / 2;
                    cnt[d] = (pf[d] % 2 == 0) ? 1 : 2;
                }
                double s = 0.0;
                for (int a = 0; a < cnt[2]; ++a)
                    for (int b = 0; b < cnt[1]; ++b)
                        for (int e = 0; e < cnt[0]; ++e) {
                            int q[3] = { lo[0] + e, lo[1] + b, lo[2] + a };
                            double w = 1.0;
                            for (int d = 0; d < dim; ++d) {
                                if (cnt[d] == 2) w *= 0.5;
                                if (C->g.bclo[d] == BC_PERIODIC) q[d] %= C->g.n[d];
                            }
                            s += w * C->x[node_index(&C->g, q)];
                        }
                F->x[node_index(&F->g, pf)] += s;
            }
}

#ifdef ORC_PARALLEL
static void nodal_gs_colour(const nodal_level* L);   /* eight-colour sweep, mg_oracle_omp.c */
#define ORC_NODAL_SMOOTH nodal_gs_colour
#else
#define ORC_NODAL_SMOOTH nodal_gs_lex
#endif

static void nodal_vcycle(nodal_mg* mg, int l)
{
    nodal_level* L = &mg->lev[l];
    if (l == mg->nlev - 1) {
        int n = mg->bottom.n;
        double* rhs = (double*)calloc(n, sizeof(double));
        for (long k = 0; k < mg->nunk; ++k) rhs[k] = L->b[mg->map[k]];
        lu_solve(&mg->bottom, rhs);
        memset(L->x, 0, sizeof(double) * nnodes(&L->g));
        for (long k = 0; k < mg->nunk; ++k) L->x[mg->map[k]] = rhs[k];
        free(rhs);
        return;
    }
    for (int s = 0; s < 2; ++s) ORC_NODAL_SMOOTH(L);
    nodal_residual(L);
    nodal_level* C = &mg->lev[l + 1];
    nodal_restrict(L, C);
    memset(C->x, 0, sizeof(double) * nnodes(&C->g));
    nodal_vcycle(mg, l + 1);
    nodal_prolong(C, L);
    for (int s = 0; s < 2; ++s) ORC_NODAL_SMOOTH(L);
}

int orc_nodal_solve_mg(const orc_grid* g, const double* sigma, const double* f_in, double* phi,
                       double tol, int max_cycles, orc_stats* st)
{
    nodal_mg mg;
    if (nodal_mg_build(&mg, g, sigma) != 0) { nodal_mg_free(&mg); return -1; }
    long M = nnodes(g);
    int sing = is_singular(g);
    nodal_level* L = &mg.lev[0];
    memcpy(L->b, f_in, sizeof(double) * M);
    int p[3];
    for (p[2] = 0; p[2] < node_extent(g, 2); ++p[2])
        for (p[1] = 0; p[1] < node_extent(g, 1); ++p[1])
            for (p[0] = 0; p[0] < node_extent(g, 0); ++p[0])
                if (node_is_dirichlet(g, p)) L->b[node_index(g, p)] = 0.0;
    if (sing) nodal_remove_mean(g, L->b);
    memcpy(L->x, phi, sizeof(double) * M);
    double fn = nodal_norm2(g, L->b);
    if (fn == 0.0) fn = 1.0;
    nodal_residual(L);
    double rel = nodal_norm2(g, L->r) / fn, best = rel;
    int it = 0, stall = 0;
    while (rel > tol && it < max_cycles) {
        nodal_vcycle(&mg, 0);
        if (sing) nodal_remove_mean(g, L->x);
        nodal_residual(L);
        rel = nodal_norm2(g, L->r) / fn;
        ++it;
        if (rel < 0.5 * best) { best = rel; stall = 0; }
        else if (++stall >= 3) break;
        if (rel < best) best = rel;
    }
    memcpy(phi, L->x, sizeof(double) * M);
    if (st) { st->iters = it; st->relres = rel; st->rhs_norm = nodal_norm2(g, L->b); }
    nodal_mg_free(&mg);
    return 0;
}

/* Full nodal projection: f = D_N(beta0 U) - lump(beta0 S), solve,
 * U_c -= (sigma_c/beta0_c) G_N phi, then the diagnostic
 * ||D_N(beta0 U) - lump(beta0 S)|| / ||lump(beta0 S)|| over the unknowns. */
int orc_nodal_project(const orc_grid* g, const double* sigma, const double* beta0, double* const U[3],
                      const double* S, double* phi, double tol, int dense, orc_stats* st)
{
    long N = ncells(g), M = nnodes(g);
    double* f = (double*)malloc(sizeof(double) * M);
    orc_nodal_rhs(g, beta0, (const double* const*)U, S, f);
    orc_stats s0;
    memset(&s0, 0, sizeof(s0));
    int rc;
    if (dense) {
        rc = orc_nodal_solve_dense(g, sigma, f, phi);
    } else {
        memset(phi, 0, sizeof(double) * M);
        rc = orc_nodal_solve_mg(g, sigma, f, phi, tol, 200, &s0);
    }
    if (rc == 0) {
        double* r = (double*)malloc(sizeof(double) * M);
        double* fb = (double*)malloc(sizeof(double) * M);
        memcpy(fb, f, sizeof(double) * M);
        if (is_singular(g)) nodal_remove_mean(g, fb);
        orc_nodal_apply(g, sigma, phi, r);
        for (long i = 0; i < M; ++i) r[i] = fb[i] - r[i];
        double fn = nodal_norm2(g, fb);
        s0.relres = nodal_norm2(g, r) / (fn > 0 ? fn : 1.0);
        s0.rhs_norm = fn;
        double* G[3] = { NULL, NULL, NULL };
        for (int d = 0; d < g->dim; ++d) G[d] = (double*)malloc(sizeof(double) * N);
        orc_nodal_grad(g, phi, G);
        for (int d = 0; d < g->dim; ++d)
            for (long i = 0; i < N; ++i) U[d][i] -= sigma[i] / beta0[i] * G[d][i];
        orc_nodal_rhs(g, beta0, (const double* const*)U, S, r);
        double* bs = (double*)malloc(sizeof(double) * N);
        for (long i = 0; i < N; ++i) bs[i] = beta0[i] * S[i];
        orc_nodal_lump(g, bs, fb);
        s0.src_norm = nodal_norm2(g, fb);
        s0.constraint = nodal_norm2(g, r) / (s0.src_norm > 0 ? s0.src_norm : 1.0);
        for (int d = 0; d < g->dim; ++d) free(G[d]);
        free(bs); free(r); free(fb);
    }
    if (st) *st = s0;
    free(f);
    return rc;
}

/* ======================================================================== */
/* Base state (Eq. 5) and its mapping onto the grid                          */
/* ======================================================================== */

/* beta0 of Eq. 5 on a radial grid:
 *   beta0(r) = rho0(r_0) exp( int (1 / (Gamma1 p0)) dp0 ),
 * written as the integral of (1/Gamma1) d(ln p0) and evaluated by the
 * trapezoid rule in ln p0: the increment between r_k and r_{k+1} is
 *   (1/2)(1/Gamma1_k + 1/Gamma1_{k+1}) (ln p0_{k+1} - ln p0_k).
 * gamma1 may be NULL (then the constant g1 is used). */
int orc_beta0_eq5(const double* p0, const double* gamma1, double g1, double rho00, int nr, double* beta0)
{
    double acc = 0.0;
    beta0[0] = rho00;
    for (int k = 0; k + 1 < nr; ++k) {
        double ga = gamma1 ? gamma1[k] : g1, gb = gamma1 ? gamma1[k + 1] : g1;
        acc += 0.5 * (1.0 / ga + 1.0 / gb) * (log(p0[k + 1]) - log(p0[k]));
        beta0[k + 1] = rho00 * exp(acc);
    }
    return 0;
}

/* linear interpolation in a uniform radial table f(r0 + k dr), clamped to the ends */
static double radial_interp(const double* f, int nr, double r0, double dr, double r)
{
    double s = (r - r0) / dr;
    if (s <= 0.0) return f[0];
    if (s >= (double)(nr - 1)) return f[nr - 1];
    int k = (int)floor(s);
    double w = s - k;
    return (1.0 - w) * f[k] + w * f[k + 1];
}

/* radius of a point: distance to the centre (spherical) or its height z
 * (plane-parallel: the last axis) */
static double point_radius(int dim, int spherical, const double* c, double x, double y, double z)
{
    if (!spherical) return dim == 3 ? z : y;
    double dx = x - c[0], dy = y - c[1], dz = dim == 3 ? z - c[2] : 0.0;
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* sigma = beta0/rho0 and beta0 at cell centres, beta0 at face centres, from
 * uniform radial tables of beta0 and rho0.  Output pointers may be NULL. */
int orc_map_radial(const orc_grid* g, int spherical, const double* center, double r0, double dr, int nr,
                   const double* beta0_r, const double* rho0_r, double* sigma, double* beta0_cell,
                   double* const beta0_face[3])
{
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                double x = (c[0] + 0.5) * g->h[0], y = (c[1] + 0.5) * g->h[1], z = (c[2] + 0.5) * g->h[2];
                double r = point_radius(g->dim, spherical, center, x, y, z);
                double b = radial_interp(beta0_r, nr, r0, dr, r), rho = radial_interp(rho0_r, nr, r0, dr, r);
                long i = cell_index(g, c);
                if (sigma) sigma[i] = b / rho;
                if (beta0_cell) beta0_cell[i] = b;
            }
    for (int d = 0; d < g->dim; ++d) {
        if (!beta0_face || !beta0_face[d]) continue;
        int f[3];
        for (f[2] = 0; f[2] < g->n[2] + (d == 2); ++f[2])
            for (f[1] = 0; f[1] < g->n[1] + (d == 1); ++f[1])
                for (f[0] = 0; f[0] < g->n[0] + (d == 0); ++f[0]) {
                    double p[3];
                    for (int e = 0; e < 3; ++e) p[e] = (f[e] + (e == d ? 0.0 : 0.5)) * g->h[e];
                    double r = point_radius(g->dim, spherical, center, p[0], p[1], p[2]);
                    beta0_face[d][face_index(g, d, f)] = radial_interp(beta0_r, nr, r0, dr, r);
                }
    }
    return 0;
}

/* ======================================================================== */
/* Rotation: Coriolis and centrifugal accelerations (S5, the rotating form  */
/* of the momentum equation)                                                 */
/* ======================================================================== */

/* For cell-centred velocity components U[d] (d < dim; the missing component of
 * a 2-D grid is 0) and angular velocity omega (3 components), at every cell
 * centre x with r = x - center:
 *     a = -2 omega x U  -  [centrifugal] omega x (omega x r)
 * and F[d] += alpha a_d.  The cross products are written out component by
 * component.  F may alias U (each cell is read in full before it is written). */
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

int orc_rotation_forces(const orc_grid* g, const double* omega, const double* center, int centrifugal,
                        double alpha, const double* const U[3], double* const F[3])
{
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                size_t id = ((size_t)c[2] * g->n[1] + c[1]) * g->n[0] + c[0];
                double u[3] = {0.0, 0.0, 0.0}, r[3] = {0.0, 0.0, 0.0}, w[3], a[3];
                for (int d = 0; d < g->dim; ++d) {
                    u[d] = U[d][id];
                    r[d] = (c[d] + 0.5) * g->h[d] - center[d];
                }
                cross3(omega, u, w);
                for (int d = 0; d < 3; ++d) a[d] = -2.0 * w[d];
                if (centrifugal) {
                    double wr[3], wwr[3];
                    cross3(omega, r, wr);
                    cross3(omega, wr, wwr);
                    for (int d = 0; d < 3; ++d) a[d] -= wwr[d];
                }
                for (int d = 0; d < g->dim; ++d) F[d][id] += alpha * a[d];
            }
    return 0;
}

/* ======================================================================== */
/* One time step around the two projections (S2-S3): face velocities,        */
/* advection of the cell-centred velocity                                    */
/* ======================================================================== */

/* cell c moved by s along d: 1 and the (wrapped) index when it exists */
static int cell_shift(const orc_grid* g, const int c[3], int d, int s, int out[3])
{
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2];
    out[d] += s;
    if (out[d] >= 0 && out[d] < g->n[d]) return 1;
    if (g->bclo[d] != BC_PERIODIC) return 0;
    out[d] = out[d] < 0 ? out[d] + g->n[d] : out[d] - g->n[d];
    return 1;
}

/* Face velocities from cell-centred U: on every face of direction d the mean of
 * U_d in the two cells beside it; a periodic face takes its wrap neighbour; a
 * wall (Neumann) face carries 0; an outflow (Dirichlet) face the value of its
 * interior cell. */
int orc_face_average(const orc_grid* g, const double* const U[3], double* const Uf[3])
{
    for (int d = 0; d < g->dim; ++d) {
        int m[3] = { g->n[0], g->n[1], g->n[2] };
        m[d] += 1;
        int f[3];
        for (f[2] = 0; f[2] < m[2]; ++f[2])
            for (f[1] = 0; f[1] < m[1]; ++f[1])
                for (f[0] = 0; f[0] < m[0]; ++f[0]) {
                    int hi[3] = { f[0], f[1], f[2] }, lo[3];
                    int has_hi = hi[d] < g->n[d];
                    int has_lo = cell_shift(g, hi, d, -1, lo);
                    if (!has_hi && g->bclo[d] == BC_PERIODIC) { hi[d] = 0; has_hi = 1; }
                    double v;
                    if (has_hi && has_lo) {
                        v = 0.5 * (U[d][cell_index(g, lo)] + U[d][cell_index(g, hi)]);
                    } else {
                        int bc = has_hi ? g->bclo[d] : g->bchi[d];
                        v = bc == BC_NEUMANN ? 0.0 : U[d][cell_index(g, has_hi ? hi : lo)];
                    }
                    Uf[d][face_index(g, d, f)] = v;
                }
    }
    return 0;
}

/* Upwind advective derivative (U_adv . grad) q at cell centres, from face
 * velocities U_adv and a cell field q:
 *   A_c = sum_d (1/h_d) [ u_{d,+} (q~_{d,+} - q_c) - u_{d,-} (q~_{d,-} - q_c) ]
 * with q~ on a face the value of the upwind cell (the lower cell when u >= 0);
 * an upwind cell outside a non-periodic boundary takes q_c (zero gradient). */
int orc_advect(const orc_grid* g, const double* const Uf[3], const double* q, double* A)
{
    int c[3];
    for (c[2] = 0; c[2] < g->n[2]; ++c[2])
        for (c[1] = 0; c[1] < g->n[1]; ++c[1])
            for (c[0] = 0; c[0] < g->n[0]; ++c[0]) {
                long id = cell_index(g, c);
                double qc = q[id], a = 0.0;
                for (int d = 0; d < g->dim; ++d) {
                    int fl[3] = { c[0], c[1], c[2] }, fh[3] = { c[0], c[1], c[2] };
                    fh[d] += 1;
                    double ul = Uf[d][face_index(g, d, fl)], uh = Uf[d][face_index(g, d, fh)];
                    int nb[3];
                    double qlo = cell_shift(g, c, d, -1, nb) ? q[cell_index(g, nb)] : qc;
                    double qhi = cell_shift(g, c, d, +1, nb) ? q[cell_index(g, nb)] : qc;
                    double qt_hi = uh >= 0.0 ? qc : qhi;   /* upwind value on the high face */
                    double qt_lo = ul >= 0.0 ? qlo : qc;   /* and on the low face */
                    a += (uh * (qt_hi - qc) - ul * (qt_lo - qc)) / g->h[d];
                }
                A[id] = a;
            }
    return 0;
}
