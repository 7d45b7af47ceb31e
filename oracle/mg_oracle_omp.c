/*
 * mg_oracle_omp.c -- the CPU baseline on every host core.  TIMING ONLY: the
 * parity tests use the one-thread oracle (mg_oracle.c as it stands), never
 * this build.
 *
 * It is mg_oracle.c compiled with ORC_PARALLEL and OpenMP: the loops over
 * cells and nodes whose iterations each write only their own element run on
 * all threads, and the two multigrid smoothers are replaced by colour-ordered
 * Gauss-Seidel sweeps -- red-black for the cell system, eight colours (the
 * parities of the three node indices) for the 27-point nodal system -- whose
 * updates within one colour read only other colours, so they too run on all
 * threads.  Every sum across cells or nodes (norms, means, the dense bottom
 * solve) stays serial.  The result therefore does not depend on the number of
 * threads: a one-thread and an all-core run agree bit for bit.  The iteration
 * counts differ from the lexicographic oracle's (another smoother), the
 * converged solution does not.
 */
#define ORC_PARALLEL 1
#include "mg_oracle.c"

#include <omp.h>

/* one red-black sweep: red cells ((i+j+k) even), then black */
static void mac_gs_colour(const mac_level* L)
{
    const double* B[3] = { L->B[0], L->B[1], L->B[2] };
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < L->g.n[2]; ++k)
            for (int j = 0; j < L->g.n[1]; ++j)
                for (int i = (colour + j + k) & 1; i < L->g.n[0]; i += 2) {
                    int c[3] = { i, j, k };
                    double dg;
                    double Lx = mac_row(&L->g, B, L->x, c, &dg);
                    long id = cell_index(&L->g, c);
                    if (dg != 0.0) L->x[id] += (L->b[id] - Lx) / dg;
                }
    }
}

/* one eight-colour sweep: nodes grouped by the parities of their indices (two
 * nodes of one colour are never neighbours in the 27-point stencil; node
 * counts on periodic axes are even, so the colouring holds across the wrap) */
static void nodal_gs_colour(const nodal_level* L)
{
    const int ncol = L->g.dim == 3 ? 8 : 4;
    for (int colour = 0; colour < ncol; ++colour) {
        const int ci = colour & 1, cj = (colour >> 1) & 1, ck = (colour >> 2) & 1;
#pragma omp parallel for schedule(static)
        for (int k = ck; k < node_extent(&L->g, 2); k += (L->g.dim == 3 ? 2 : 1))
            for (int j = cj; j < node_extent(&L->g, 1); j += 2)
                for (int i = ci; i < node_extent(&L->g, 0); i += 2) {
                    int p[3] = { i, j, k };
                    if (node_is_dirichlet(&L->g, p)) continue;
                    double dg;
                    double Lx = nodal_row(&L->g, L->sigma, L->x, p, &dg);
                    long id = node_index(&L->g, p);
                    if (dg != 0.0) L->x[id] += (L->b[id] - Lx) / dg;
                }
    }
}

void orc_omp_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_omp_max_threads(void) { return omp_get_max_threads(); }
