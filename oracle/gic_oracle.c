/*
 * gic_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library. The GPU
 * product path never links, imports or calls it, and it shares no code,
 * header or table with the CUDA sources.
 *
 * Every routine restates one step of the method of "Deep Learning-Enhanced
 * Preconditioning for Efficient Conjugate Gradient Solvers in Large-Scale PDE
 * Systems" (arxiv 2412.07127) in the most literal sequential form: no
 * blocking, no fusion, no reordering beyond what the definition states.
 * Compiled with -ffp-contract=off so every a-b*c is two roundings.
 *
 * Parity status per function (what pins it, see tests/test_oracle_*.py):
 *   or_hex_element_stiffness  pinned: symmetry, 6 rigid-body null vectors,
 *                             uniform-strain patch test (closed form forces)
 *   or_fem_hex_assemble       pinned: closed-form nnz, symmetry, rigid modes
 *   or_fem_box_assemble       pinned: equals the cube for Nx = Ny = Nz = N;
 *                             the rows of its first m node planes equal the
 *                             cube's (a z-slab of the cube's elements)
 *   or_spmv_threads           pinned: identical to or_spmv
 *   or_lower_pattern/levels   pinned: closed-form level formula x+2y+4(z-1)
 *   or_ic0                    pinned: dense Cholesky on no-fill patterns,
 *                             (LL^T)_ij == a_ij on the pattern, dense masked
 *                             brute force at n<=200
 *   or_spmv/lsolve/ltsolve    pinned: dense numpy products/solves
 *   or_pcg                    pinned: <= n steps, 1 step with exact Cholesky,
 *                             Eq.(6) bound, dense solve
 *   or_features               pinned: hand-computed 4x4 cases
 *   or_gnn_forward            pinned: g = 0 => L = L_IC; GraphNorm output
 *                             moments in closed form; block-0 node sums =
 *                             full-row counts / row sums of A (each edge to
 *                             both endpoints, a self-loop once), means = sums
 *                             / incident-edge count; a hand-worked 2-node
 *                             graph; two disjoint copies in one graph give
 *                             the copy's output twice; an independent dense
 *                             restatement. The
 *                             layout itself is a reading (Figure 1 is missing
 *                             from the text): parity unpinned against the
 *                             paper for the architecture, not its arithmetic.
 *   or_correct(+backward)     pinned: g = 0 => L_IC; finite differences
 *   or_probe_loss(+grad)      pinned: unbiased vs dense ||LL^T-A||_F^2,
 *                             central finite differences
 *   or_gnn_backward           pinned: central finite differences
 *   or_adam_step              pinned: closed form of the first steps
 *   or_dropout                pinned: eps = 0 keeps L, a huge eps keeps the
 *                             diagonal only, hand-built 3x3 case
 *   or_factor_deviation       pinned: zero for equal factors, hand-built case
 *   or_row_groups             pinned: hex nodes (groups of 3), hand-built runs,
 *                             runs cut at their common length
 *   or_dropout_grouped        pinned: eps = 0 keeps L, reduces to or_dropout
 *                             on single-row groups, hand-built 2x2 blocks,
 *                             node blocks kept whole (hex)
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ======================================================================
 * A1. 3-D linear-elasticity stiffness on a structured trilinear hex mesh.
 * The paper's systems come from 3-D static structural FE analysis
 * (Experiments, Datasets; Supplementary 1). The synthetic stand-in is the
 * unit cube split into N^3 cubes of side h = 1/N.
 * ====================================================================== */

/* Element stiffness of one cube of side h, Young modulus 1, Poisson nu.
 * Ke is 24x24 row-major; local dof 3*a+c, local node a = ax + 2ay + 4az.
 * Ke = sum over the 2x2x2 Gauss points of B^T D B det(J). Engineering shear
 * strains in the order (xy, yz, zx). */
void or_hex_element_stiffness(double nu, double h, double *Ke)
{
    double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = 1.0 / (2.0 * (1.0 + nu));
    double D[6][6];
    memset(D, 0, sizeof D);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) D[i][j] = lam;
        D[i][i] = lam + 2.0 * mu;
        D[3 + i][3 + i] = mu;
    }
    memset(Ke, 0, sizeof(double) * 24 * 24);
    double gp = 1.0 / sqrt(3.0);
    double detJ = (h / 2.0) * (h / 2.0) * (h / 2.0);
    for (int q = 0; q < 8; ++q) {
        double xi = (q & 1) ? gp : -gp;
        double eta = (q & 2) ? gp : -gp;
        double zeta = (q & 4) ? gp : -gp;
        double B[6][24];
        memset(B, 0, sizeof B);
        for (int a = 0; a < 8; ++a) {
            double sx = (a & 1) ? 1.0 : -1.0;
            double sy = (a & 2) ? 1.0 : -1.0;
            double sz = (a & 4) ? 1.0 : -1.0;
            /* dN/dx = (2/h) dN/dxi */
            double dx = 0.125 * sx * (1.0 + eta * sy) * (1.0 + zeta * sz) * (2.0 / h);
            double dy = 0.125 * (1.0 + xi * sx) * sy * (1.0 + zeta * sz) * (2.0 / h);
            double dz = 0.125 * (1.0 + xi * sx) * (1.0 + eta * sy) * sz * (2.0 / h);
            B[0][3 * a + 0] = dx;
            B[1][3 * a + 1] = dy;
            B[2][3 * a + 2] = dz;
            B[3][3 * a + 0] = dy;
            B[3][3 * a + 1] = dx;
            B[4][3 * a + 1] = dz;
            B[4][3 * a + 2] = dy;
            B[5][3 * a + 0] = dz;
            B[5][3 * a + 2] = dx;
        }
        for (int r = 0; r < 24; ++r)
            for (int c = 0; c < 24; ++c) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k)
                    for (int l = 0; l < 6; ++l) s += B[k][r] * D[k][l] * B[l][c];
                Ke[r * 24 + c] += s * detJ;
            }
    }
}

/* A box of Nx x Ny x Nz hexahedral elements of side h (the unit cube of N^3
 * elements is Nx = Ny = Nz = N, h = 1/N). Nodes (x, y, z), 0 <= x <= Nx,
 * 0 <= y <= Ny, 0 <= z <= Nz, are numbered x fastest, then y, then z.
 * Free nodes are those with z >= z0 (z0 = 1 when the z = 0 face is clamped
 * and its dofs eliminated, z0 = 0 for the free-floating body). */
typedef struct {
    int nx, ny, nz, z0;
} Box;

static int64_t node_id(const Box *B, int x, int y, int z)
{
    return (int64_t)x + (int64_t)(B->nx + 1) * ((int64_t)y + (int64_t)(B->ny + 1) * (z - B->z0));
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Neighbour free nodes of free node (x,y,z): the free nodes of every element
 * that contains it, sorted and deduplicated. Returns the count (<= 27). */
static int node_neighbours(const Box *B, int x, int y, int z, int64_t *out)
{
    int64_t tmp[64];
    int cnt = 0;
    for (int ez = z - 1; ez <= z; ++ez)
        for (int ey = y - 1; ey <= y; ++ey)
            for (int ex = x - 1; ex <= x; ++ex) {
                if (ex < 0 || ey < 0 || ez < 0 || ex >= B->nx || ey >= B->ny || ez >= B->nz) continue;
                for (int a = 0; a < 8; ++a) {
                    int nx = ex + (a & 1), ny = ey + ((a >> 1) & 1), nz = ez + ((a >> 2) & 1);
                    if (nz < B->z0) continue;
                    tmp[cnt++] = node_id(B, nx, ny, nz);
                }
            }
    qsort(tmp, (size_t)cnt, sizeof(int64_t), cmp_i64);
    int m = 0;
    for (int i = 0; i < cnt; ++i)
        if (m == 0 || tmp[i] != out[m - 1]) out[m++] = tmp[i];
    return m;
}

/* Sizes of the assembled box system: n = 3 * #free nodes, nnz of the CSR. */
int or_fem_box_sizes(int Nx, int Ny, int Nz, int clamp, int64_t *n, int64_t *nnz)
{
    if (Nx < 1 || Ny < 1 || Nz < 1) return -1;
    Box B = {Nx, Ny, Nz, clamp ? 1 : 0};
    int64_t nn = 0, nzc = 0;
    int64_t nb[27];
    for (int z = B.z0; z <= Nz; ++z)
        for (int y = 0; y <= Ny; ++y)
            for (int x = 0; x <= Nx; ++x) {
                nn += 1;
                nzc += 9 * (int64_t)node_neighbours(&B, x, y, z, nb);
            }
    *n = 3 * nn;
    *nnz = nzc;
    return 0;
}

int or_fem_hex_sizes(int N, int clamp, int64_t *n, int64_t *nnz)
{
    return or_fem_box_sizes(N, N, N, clamp, n, nnz);
}

/* Assemble A = sum_e E_e K_e over the box's elements (element id
 * ex + Nx*(ey + Ny*ez)), element side h, keeping only free dofs (dof =
 * 3*node + component). Columns are sorted in each row. The value of every
 * entry is accumulated element by element in ascending element order. */
int or_fem_box_assemble(int Nx, int Ny, int Nz, double h, int clamp, double nu, const double *E,
                        int32_t *rowptr, int32_t *col, double *val)
{
    if (Nx < 1 || Ny < 1 || Nz < 1 || !(h > 0.0)) return -1;
    Box B = {Nx, Ny, Nz, clamp ? 1 : 0};
    double Ke[576];
    or_hex_element_stiffness(nu, h, Ke);
    int64_t nb[27];
    int64_t pos = 0;
    rowptr[0] = 0;
    for (int z = B.z0; z <= Nz; ++z)
        for (int y = 0; y <= Ny; ++y)
            for (int x = 0; x <= Nx; ++x) {
                int m = node_neighbours(&B, x, y, z, nb);
                for (int c = 0; c < 3; ++c) {
                    for (int k = 0; k < m; ++k)
                        for (int d = 0; d < 3; ++d) {
                            col[pos] = (int32_t)(3 * nb[k] + d);
                            val[pos] = 0.0;
                            pos++;
                        }
                    int64_t row = 3 * node_id(&B, x, y, z) + c;
                    rowptr[row + 1] = (int32_t)pos;
                }
            }
    for (int ez = 0; ez < Nz; ++ez)
        for (int ey = 0; ey < Ny; ++ey)
            for (int ex = 0; ex < Nx; ++ex) {
                double Ee = E[(int64_t)ex + (int64_t)Nx * (ey + (int64_t)Ny * ez)];
                for (int a = 0; a < 8; ++a) {
                    int az = ez + ((a >> 2) & 1);
                    if (az < B.z0) continue;
                    int64_t pa = node_id(&B, ex + (a & 1), ey + ((a >> 1) & 1), az);
                    for (int b = 0; b < 8; ++b) {
                        int bz = ez + ((b >> 2) & 1);
                        if (bz < B.z0) continue;
                        int64_t pb = node_id(&B, ex + (b & 1), ey + ((b >> 1) & 1), bz);
                        for (int c = 0; c < 3; ++c) {
                            int64_t i = 3 * pa + c;
                            for (int d = 0; d < 3; ++d) {
                                int32_t j = (int32_t)(3 * pb + d);
                                int32_t lo = rowptr[i], hi = rowptr[i + 1] - 1;
                                while (lo < hi) {
                                    int32_t mid = (lo + hi) / 2;
                                    if (col[mid] < j) lo = mid + 1; else hi = mid;
                                }
                                if (col[lo] != j) return -2;
                                val[lo] += Ee * Ke[(3 * a + c) * 24 + 3 * b + d];
                            }
                        }
                    }
                }
            }
    return 0;
}

/* The unit cube of N^3 elements (element id ex + N*(ey + N*ez)). */
int or_fem_hex_assemble(int N, int clamp, double nu, const double *E,
                        int32_t *rowptr, int32_t *col, double *val)
{
    if (N < 1) return -1;
    return or_fem_box_assemble(N, N, N, 1.0 / N, clamp, nu, E, rowptr, col, val);
}

/* ======================================================================
 * A2. Lower-triangular pattern (the pattern of L in IC(0): "the sparsity
 * pattern of L typically mirrors that of A", Introduction; Model
 * Architecture uses only the lower triangle) and its level sets.
 * ====================================================================== */

int64_t or_lower_nnz(int64_t n, const int32_t *rowptr, const int32_t *col)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] <= i) c++;
    return c;
}

/* tril(A): Lrowptr/Lcol (and Lval if both val and Lval are non-NULL). */
void or_lower_pattern(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                      int32_t *Lrowptr, int32_t *Lcol, double *Lval)
{
    int64_t q = 0;
    Lrowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] <= i) {
                Lcol[q] = col[p];
                if (val && Lval) Lval[q] = val[p];
                q++;
            }
        Lrowptr[i + 1] = (int32_t)q;
    }
}

/* level(i) = 0 if row i has no strictly-lower entry, else
 * 1 + max level(j) over its strictly-lower entries j. Returns #levels. */
int32_t or_levels(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, int32_t *level)
{
    int32_t nlev = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t lv = 0;
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
            int32_t j = Lcol[p];
            if (j < i && level[j] + 1 > lv) lv = level[j] + 1;
        }
        level[i] = lv;
        if (lv + 1 > nlev) nlev = lv + 1;
    }
    return nlev;
}

/* ======================================================================
 * A3. IC(0): L on the pattern of tril(A) with (L L^T)_ij = a_ij for every
 * (i,j) in that pattern (Introduction; Baseline Methods; Supplementary 2).
 *   L_ij = (a_ij - sum_{k<j} L_ik L_jk) / L_jj     (j < i, (i,j) in pattern)
 *   L_ii = sqrt(a_ii - sum_{k<i} L_ik^2)
 * with k over the pattern intersection, summed in ascending k. The diagonal
 * used is a_ii + alpha*a_ii (alpha = 0: plain IC(0); alpha > 0: shifted).
 * Lval must hold tril(A)'s values on entry; it is overwritten with L.
 * Returns -1 on success or the first row whose pivot is <= 0 or non-finite.
 * ====================================================================== */
int64_t or_ic0(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, double *Lval, double alpha)
{
    for (int64_t i = 0; i < n; ++i) {
        int32_t rs = Lrowptr[i], re = Lrowptr[i + 1];
        if (re <= rs || Lcol[re - 1] != i) return i; /* missing diagonal */
        for (int32_t p = rs; p < re - 1; ++p) {
            int32_t j = Lcol[p];
            double s = Lval[p];
            int32_t q = rs, r = Lrowptr[j], rend = Lrowptr[j + 1] - 1;
            while (q < p && r < rend) {
                if (Lcol[q] == Lcol[r]) {
                    s = s - Lval[q] * Lval[r];
                    q++;
                    r++;
                } else if (Lcol[q] < Lcol[r]) {
                    q++;
                } else {
                    r++;
                }
            }
            Lval[p] = s / Lval[Lrowptr[j + 1] - 1];
        }
        double a = Lval[re - 1];
        double s = a + alpha * a;
        for (int32_t q = rs; q < re - 1; ++q) s = s - Lval[q] * Lval[q];
        if (!(s > 0.0) || !isfinite(s)) return i;
        Lval[re - 1] = sqrt(s);
    }
    return -1;
}

/* IC(0) with the diagonal-shift restart: on breakdown retry with
 * alpha = 1e-3, 2e-3, 4e-3, ... (at most max_tries shifted tries).
 * Atril: tril(A) values; Lval receives L. Returns -1 on success (alpha_out =
 * the shift used, 0 if none) or the failing row of the last try. */
int64_t or_ic0_auto(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *Atril,
                    double *Lval, int max_tries, double *alpha_out)
{
    int64_t nnz = Lrowptr[n];
    double alpha = 0.0;
    int64_t bad = -1;
    for (int t = 0; t <= max_tries; ++t) {
        memcpy(Lval, Atril, sizeof(double) * (size_t)nnz);
        bad = or_ic0(n, Lrowptr, Lcol, Lval, alpha);
        if (bad < 0) {
            *alpha_out = alpha;
            return -1;
        }
        alpha = (t == 0) ? 1e-3 : 2.0 * alpha;
    }
    *alpha_out = alpha;
    return bad;
}

/* ======================================================================
 * A7. Sparse kernels of the PCG loop.
 * ====================================================================== */

/* y = A x, CSR, summed in stored order. */
void or_spmv(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
             const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s = s + val[p] * x[col[p]];
        y[i] = s;
    }
}

/* The same product with the rows split over the host's cores (OpenMP), for
 * the all-core CPU timing; every row is summed exactly as in or_spmv, so the
 * result is identical. The triangular solves have no such variant: they are
 * sequential by definition. */
void or_spmv_threads(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                     const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s = s + val[p] * x[col[p]];
        y[i] = s;
    }
}

int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Forward substitution L y = r (Supplementary 5, Eq.(11) read as
 * y_i = (r_i - sum_{j<i} L_ij y_j) / L_ii). The diagonal is the last entry. */
void or_lsolve(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval,
               const double *r, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = r[i];
        int32_t re = Lrowptr[i + 1];
        for (int32_t p = Lrowptr[i]; p < re - 1; ++p) s = s - Lval[p] * y[Lcol[p]];
        y[i] = s / Lval[re - 1];
    }
}

/* Back substitution L^T z = y, column-oriented on L itself:
 * z_i = (y_i - sum_{j>i} L_ji z_j) / L_ii for i = n-1 .. 0. */
void or_ltsolve(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval,
                const double *y, double *z)
{
    memcpy(z, y, sizeof(double) * (size_t)n);
    for (int64_t i = n - 1; i >= 0; --i) {
        int32_t re = Lrowptr[i + 1];
        z[i] = z[i] / Lval[re - 1];
        for (int32_t p = Lrowptr[i]; p < re - 1; ++p) z[Lcol[p]] = z[Lcol[p]] - Lval[p] * z[i];
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

/* IC-PCG exactly as Algorithm 1 of the supplementary material, with the stop
 * rule read as ||r_k||_2 / ||b||_2 <= tol on the recurrence residual. If
 * Lval is NULL the preconditioner is the identity (plain CG, "None").
 * x holds x0 on entry and the solution on exit. iters counts x updates.
 * If ||r_0|| already satisfies the rule, no iteration is taken.
 * hist (nullable): x after every iteration (iters*n doubles).
 * rhist (nullable): ||r_k||_2 for k = 0..iters.
 * Returns 0 on convergence, 1 if maxit was reached, 2 on breakdown
 * (non-positive or non-finite p^T A p or r^T z). */
int or_pcg(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
           const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval,
           const double *b, double *x, double tol, int maxit, int *iters, double *relres,
           double *hist, double *rhist)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    int status = 1;
    int k = 0;
    double bnorm = sqrt(dot(n, b, b));
    /* line 1: r0 = b - A x0 */
    or_spmv(n, rowptr, col, val, x, w);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    double rnorm = sqrt(dot(n, r, r));
    if (rhist) rhist[0] = rnorm;
    if (bnorm == 0.0 || rnorm <= tol * bnorm) {
        status = 0;
        goto done;
    }
    double rz_old = 0.0;
    while (k < maxit) {
        /* lines 2-3 / 11-12: L y = r, L^T z = y */
        if (Lval) {
            or_lsolve(n, Lrowptr, Lcol, Lval, r, y);
            or_ltsolve(n, Lrowptr, Lcol, Lval, y, z);
        } else {
            memcpy(z, r, sizeof(double) * (size_t)n);
        }
        double rz = dot(n, r, z);
        if (!(isfinite(rz)) || rz <= 0.0) { status = 2; break; }
        if (k == 0) {
            memcpy(p, z, sizeof(double) * (size_t)n); /* line 4 */
        } else {
            double beta = rz / rz_old; /* line 13 */
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i]; /* line 14 */
        }
        rz_old = rz;
        or_spmv(n, rowptr, col, val, p, w); /* line 5 / 15 */
        double pw = dot(n, p, w);
        if (!(isfinite(pw)) || pw <= 0.0) { status = 2; break; }
        double alpha = rz / pw; /* line 6 / 16 */
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i]; /* line 7 / 17 */
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * w[i]; /* line 8 / 18 */
        k++;
        rnorm = sqrt(dot(n, r, r));
        if (hist) memcpy(hist + (size_t)(k - 1) * (size_t)n, x, sizeof(double) * (size_t)n);
        if (rhist) rhist[k] = rnorm;
        if (rnorm <= tol * bnorm) { status = 0; break; } /* line 10 */
    }
done:
    *iters = k;
    *relres = (bnorm > 0.0) ? rnorm / bnorm : 0.0;
    free(r); free(y); free(z); free(p); free(w);
    return status;
}

/* ======================================================================
 * A4. Graph inputs (Model Architecture; Supplementary 4, Table 2).
 *   edge feature e_ij = a_ij / s on tril(A)'s pattern, s = population
 *   standard deviation of tril(A)'s stored values (diagonal included);
 *   node features x_v (9): deg(v), max/min/mean/var deg over neighbours,
 *   dominance |a_vv| / sum_{j!=v}|a_vj|, decay |a_vv| / max_{j!=v}|a_vj|,
 *   sin(v), cos(v). deg(v) = number of off-diagonal entries in row v of A;
 *   neighbours = the off-diagonal columns of row v. Empty neighbour sets and
 *   zero denominators give 0.
 * ====================================================================== */
void or_features(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                 double *x9, const int32_t *Lrowptr, double *e, double *scale)
{
    int64_t nnzL = Lrowptr[n];
    /* tril values in row order */
    double *tv = (double *)malloc(sizeof(double) * (size_t)(nnzL > 0 ? nnzL : 1));
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] <= i) tv[q++] = val[p];
    double mean = 0.0;
    for (int64_t k = 0; k < nnzL; ++k) mean += tv[k];
    mean /= (double)nnzL;
    double var = 0.0;
    for (int64_t k = 0; k < nnzL; ++k) var += (tv[k] - mean) * (tv[k] - mean);
    var /= (double)nnzL;
    double s = sqrt(var);
    *scale = s;
    for (int64_t k = 0; k < nnzL; ++k) e[k] = tv[k] / s;
    free(tv);

    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int32_t d = 0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] != i) d++;
        deg[i] = d;
    }
    for (int64_t i = 0; i < n; ++i) {
        double dmax = 0, dmin = 0, dsum = 0, dsq = 0, diag = 0, offsum = 0, offmax = 0;
        int cnt = 0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j == i) { diag = fabs(val[p]); continue; }
            double dj = (double)deg[j];
            if (cnt == 0 || dj > dmax) dmax = dj;
            if (cnt == 0 || dj < dmin) dmin = dj;
            dsum += dj;
            cnt++;
            offsum += fabs(val[p]);
            if (fabs(val[p]) > offmax) offmax = fabs(val[p]);
        }
        double dmean = cnt ? dsum / cnt : 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j == i) continue;
            double t = (double)deg[j] - dmean;
            dsq += t * t;
        }
        double *xv = x9 + 9 * i;
        xv[0] = (double)deg[i];
        xv[1] = dmax;
        xv[2] = dmin;
        xv[3] = dmean;
        xv[4] = cnt ? dsq / cnt : 0.0;
        xv[5] = offsum > 0 ? diag / offsum : 0.0;
        xv[6] = offmax > 0 ? diag / offmax : 0.0;
        xv[7] = sin((double)i);
        xv[8] = cos((double)i);
    }
    free(deg);
}

/* ======================================================================
 * A5/A6. The GNN correction (Eq.(2), Eq.(7)-(9), Model Architecture).
 *
 * Flat parameter layout (H = 32 hidden units, 3504 values):
 *   GraphNorm gamma[9], beta[9], alpha[9]
 *   for block l = 0,1,2:
 *     edge MLP  W1[32][20], b1[32], W2[32], b2[1]
 *     if l < 2: node MLP W3[32][11], b3[32], W4[9][32], b4[9]
 * Edge input  = [e_cur, e0, x_i(9), x_j(9)] for the edge (i,j) of tril(A),
 *               i = row >= j = column; e_cur = e0 in block 0.
 * Edge MLP    = W2 tanh(W1 h + b1) + b2  -> new edge value.
 * Aggregation = sum and mean of the new edge values over the edges incident
 *               to each node (an off-diagonal edge reaches both ends, a
 *               self-loop counts once).
 * Node MLP    = W4 tanh(W3 [x_v, sum_v, mean_v] + b3) + b4 -> new x_v.
 * Block 2 has no node update; its edge values are g.
 * Correction  (in units scaled by s): off-diagonal Lhat_ij = LhatIC_ij + g_ij,
 *             diagonal Lhat_ii = LhatIC_ii * exp(g_ii / 2), i.e. the exp then
 *             sqrt positivity map applied multiplicatively to L_IC.
 * bf16 is a bit set of the operands rounded to bfloat16 (round to nearest
 * even) before an exact FP64 product, which is what BF16 weights with FP32
 * accumulation compute: bit 0 (value 1) the edge MLP's first layer (W1 and
 * its input h); bit 1 (value 2) both layers of the node MLP (W3 and its input
 * [x, S, M]; W4 and the tanh output). The backward pass honours bit 0 only
 * (the node-MLP rounding is an inference mode).
 * ====================================================================== */
#define GH 32
#define GPAR_GN 27
#define GPAR_EDGE (GH * 20 + GH + GH + 1)
#define GPAR_NODE (GH * 11 + GH + 9 * GH + 9)
#define GPAR_TOTAL (GPAR_GN + 3 * GPAR_EDGE + 2 * GPAR_NODE)

int or_gnn_param_count(void) { return GPAR_TOTAL; }

static int64_t off_edge(int l) { return GPAR_GN + (int64_t)l * (GPAR_EDGE + GPAR_NODE); }
static int64_t off_node(int l) { return off_edge(l) + GPAR_EDGE; }

/* Round to bfloat16 (8 significant bits), ties to even, straight from FP64. */
double or_round_bf16(double v)
{
    if (!isfinite(v) || v == 0.0) return v;
    int ex;
    double m = frexp(v, &ex);   /* v = m * 2^ex, 0.5 <= |m| < 1 */
    double r = nearbyint(ldexp(m, 8)); /* default rounding mode: ties to even */
    return ldexp(r, ex - 8);
}

/* Activations saved by the forward pass for the backward pass. */
typedef struct {
    double *x[3];     /* node input of block l, n*9 (x[0] = GraphNorm output) */
    double *ecur[3];  /* edge input of block l, E */
    double *a1[3];    /* tanh hidden of edge MLP, E*H */
    double *h[3];     /* edge MLP input (as used, possibly bf16-rounded), E*20 */
    double *enew[3];  /* edge MLP output, E */
    double *S[2], *M[2]; /* aggregation, n */
    double *a3[2];    /* tanh hidden of node MLP, n*H */
    double *gn_c;     /* GraphNorm centred input, n*9 */
    double gn_sig[9], gn_mu[9];
} or_gnn_tape;

static void tape_alloc(or_gnn_tape *t, int64_t n, int64_t E)
{
    memset(t, 0, sizeof *t);
    for (int l = 0; l < 3; ++l) {
        t->x[l] = (double *)calloc((size_t)(n * 9), sizeof(double));
        t->ecur[l] = (double *)calloc((size_t)E, sizeof(double));
        t->a1[l] = (double *)calloc((size_t)(E * GH), sizeof(double));
        t->h[l] = (double *)calloc((size_t)(E * 20), sizeof(double));
        t->enew[l] = (double *)calloc((size_t)E, sizeof(double));
    }
    for (int l = 0; l < 2; ++l) {
        t->S[l] = (double *)calloc((size_t)n, sizeof(double));
        t->M[l] = (double *)calloc((size_t)n, sizeof(double));
        t->a3[l] = (double *)calloc((size_t)(n * GH), sizeof(double));
    }
    t->gn_c = (double *)calloc((size_t)(n * 9), sizeof(double));
}

static void tape_free(or_gnn_tape *t)
{
    for (int l = 0; l < 3; ++l) {
        free(t->x[l]); free(t->ecur[l]); free(t->a1[l]); free(t->h[l]); free(t->enew[l]);
    }
    for (int l = 0; l < 2; ++l) { free(t->S[l]); free(t->M[l]); free(t->a3[l]); }
    free(t->gn_c);
}

/* incident-edge count per node on the tril graph (self-loop once) */
static void node_degree(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, double *deg)
{
    for (int64_t v = 0; v < n; ++v) deg[v] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
            int32_t j = Lcol[p];
            deg[i] += 1.0;
            if (j != i) deg[j] += 1.0;
        }
}

static void gnn_forward_tape(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol,
                             const double *x9, const double *e0, const double *theta, int bf16,
                             double *g, or_gnn_tape *t)
{
    int64_t E = Lrowptr[n];
    /* GraphNorm on the input node features */
    const double *gam = theta, *bet = theta + 9, *alp = theta + 18;
    for (int f = 0; f < 9; ++f) {
        double mu = 0.0;
        for (int64_t v = 0; v < n; ++v) mu += x9[9 * v + f];
        mu /= (double)n;
        double var = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double c = x9[9 * v + f] - alp[f] * mu;
            t->gn_c[9 * v + f] = c;
            var += c * c;
        }
        var /= (double)n;
        double sig = sqrt(var + 1e-5);
        t->gn_mu[f] = mu;
        t->gn_sig[f] = sig;
        for (int64_t v = 0; v < n; ++v) t->x[0][9 * v + f] = gam[f] * t->gn_c[9 * v + f] / sig + bet[f];
    }
    double *deg = (double *)malloc(sizeof(double) * (size_t)n);
    node_degree(n, Lrowptr, Lcol, deg);
    memcpy(t->ecur[0], e0, sizeof(double) * (size_t)E);
    for (int l = 0; l < 3; ++l) {
        const double *W1 = theta + off_edge(l);
        const double *b1 = W1 + GH * 20;
        const double *W2 = b1 + GH;
        const double *b2 = W2 + GH;
        const double *xl = t->x[l];
        for (int64_t i = 0; i < n; ++i)
            for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
                int32_t j = Lcol[p];
                double *h = t->h[l] + 20 * (int64_t)p;
                h[0] = t->ecur[l][p];
                h[1] = e0[p];
                for (int f = 0; f < 9; ++f) h[2 + f] = xl[9 * i + f];
                for (int f = 0; f < 9; ++f) h[11 + f] = xl[9 * (int64_t)j + f];
                if (bf16 & 1)
                    for (int f = 0; f < 20; ++f) h[f] = or_round_bf16(h[f]);
                double out = b2[0];
                for (int u = 0; u < GH; ++u) {
                    double z = b1[u];
                    for (int f = 0; f < 20; ++f) {
                        double w = (bf16 & 1) ? or_round_bf16(W1[u * 20 + f]) : W1[u * 20 + f];
                        z += w * h[f];
                    }
                    double a = tanh(z);
                    t->a1[l][(int64_t)p * GH + u] = a;
                    out += W2[u] * a;
                }
                t->enew[l][p] = out;
            }
        if (l == 2) break;
        memcpy(t->ecur[l + 1], t->enew[l], sizeof(double) * (size_t)E);
        double *S = t->S[l], *M = t->M[l];
        for (int64_t v = 0; v < n; ++v) S[v] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
                int32_t j = Lcol[p];
                S[i] += t->enew[l][p];
                if (j != i) S[j] += t->enew[l][p];
            }
        for (int64_t v = 0; v < n; ++v) M[v] = deg[v] > 0 ? S[v] / deg[v] : 0.0;
        const double *W3 = theta + off_node(l);
        const double *b3 = W3 + GH * 11;
        const double *W4 = b3 + GH;
        const double *b4 = W4 + 9 * GH;
        for (int64_t v = 0; v < n; ++v) {
            double u_in[11];
            for (int f = 0; f < 9; ++f) u_in[f] = xl[9 * v + f];
            u_in[9] = S[v];
            u_in[10] = M[v];
            double *a3 = t->a3[l] + v * GH;
            const int rn = (bf16 & 2) != 0;
            if (rn)
                for (int f = 0; f < 11; ++f) u_in[f] = or_round_bf16(u_in[f]);
            for (int u = 0; u < GH; ++u) {
                double z = b3[u];
                for (int f = 0; f < 11; ++f) z += (rn ? or_round_bf16(W3[u * 11 + f]) : W3[u * 11 + f]) * u_in[f];
                a3[u] = tanh(z);
            }
            for (int f = 0; f < 9; ++f) {
                double o = b4[f];
                for (int u = 0; u < GH; ++u)
                    o += rn ? or_round_bf16(W4[f * GH + u]) * or_round_bf16(a3[u]) : W4[f * GH + u] * a3[u];
                t->x[l + 1][9 * v + f] = o;
            }
        }
    }
    memcpy(g, t->enew[2], sizeof(double) * (size_t)E);
    free(deg);
}

/* g = GNN(A) on tril(A)'s pattern: x9 raw node features (n*9), e0 scaled edge
 * values (E), theta the flat parameters. */
void or_gnn_forward(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *x9,
                    const double *e0, const double *theta, int bf16, double *g)
{
    or_gnn_tape t;
    tape_alloc(&t, n, Lrowptr[n]);
    gnn_forward_tape(n, Lrowptr, Lcol, x9, e0, theta, bf16, g, &t);
    tape_free(&t);
}

/* The same forward, also returning intermediates that tests pin to closed
 * forms: x0 (n x 9, the GraphNorm output), block 0's node sums S0 and means
 * M0 (n each) and its node update x1 (n x 9). */
void or_gnn_forward_parts(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *x9,
                          const double *e0, const double *theta, int bf16, double *g, double *x0,
                          double *S0, double *M0, double *x1)
{
    or_gnn_tape t;
    tape_alloc(&t, n, Lrowptr[n]);
    gnn_forward_tape(n, Lrowptr, Lcol, x9, e0, theta, bf16, g, &t);
    memcpy(x0, t.x[0], sizeof(double) * (size_t)(9 * n));
    memcpy(S0, t.S[0], sizeof(double) * (size_t)n);
    memcpy(M0, t.M[0], sizeof(double) * (size_t)n);
    memcpy(x1, t.x[1], sizeof(double) * (size_t)(9 * n));
    tape_free(&t);
}

/* Eq.(2) with the positivity map: Lout = LIC + g off the diagonal and
 * LIC * exp(g/2) on it. Both in the same units (the caller scales). */
void or_correct(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *LIC,
                const double *g, double *Lout)
{
    for (int64_t i = 0; i < n; ++i)
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p)
            Lout[p] = (Lcol[p] == i) ? LIC[p] * exp(g[p] / 2.0) : LIC[p] + g[p];
}

/* Backward of or_correct: dg = dLout off the diagonal and
 * dLout * LIC * exp(g/2) / 2 on it (the derivative of each output entry). */
void or_correct_backward(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *LIC,
                         const double *g, const double *dLout, double *dg)
{
    for (int64_t i = 0; i < n; ++i)
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p)
            dg[p] = (Lcol[p] == i) ? dLout[p] * LIC[p] * exp(g[p] / 2.0) / 2.0 : dLout[p];
}

/* Backward of the GNN for the gradient dg of the edge output g.
 * dtheta (GPAR_TOTAL) is overwritten with d(loss)/d(theta). */
void or_gnn_backward(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *x9,
                     const double *e0, const double *theta, int bf16, const double *dg,
                     double *dtheta)
{
    int64_t E = Lrowptr[n];
    or_gnn_tape t;
    tape_alloc(&t, n, E);
    double *g = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    bf16 &= 1; /* the node-MLP rounding is an inference mode */
    gnn_forward_tape(n, Lrowptr, Lcol, x9, e0, theta, bf16, g, &t);
    free(g);
    memset(dtheta, 0, sizeof(double) * GPAR_TOTAL);
    double *deg = (double *)malloc(sizeof(double) * (size_t)n);
    node_degree(n, Lrowptr, Lcol, deg);

    double *de = (double *)calloc((size_t)E, sizeof(double));   /* d enew of current block */
    double *dx = (double *)calloc((size_t)(n * 9), sizeof(double)); /* d x[l+1] */
    double *dxl = (double *)calloc((size_t)(n * 9), sizeof(double));
    double *dS = (double *)calloc((size_t)n, sizeof(double));
    double *dM = (double *)calloc((size_t)n, sizeof(double));
    memcpy(de, dg, sizeof(double) * (size_t)E);

    for (int l = 2; l >= 0; --l) {
        if (l < 2) {
            /* node MLP backward: x[l+1] = W4 a3 + b4, a3 = tanh(W3 u + b3) */
            const double *W3 = theta + off_node(l);
            const double *b3 = W3 + GH * 11;
            const double *W4 = b3 + GH;
            double *dW3 = dtheta + off_node(l);
            double *db3 = dW3 + GH * 11;
            double *dW4 = db3 + GH;
            double *db4 = dW4 + 9 * GH;
            (void)b3;
            for (int64_t v = 0; v < n; ++v) { dS[v] = 0.0; dM[v] = 0.0; }
            for (int64_t v = 0; v < n; ++v) {
                const double *a3 = t.a3[l] + v * GH;
                const double *dxo = dx + 9 * v;
                double u_in[11];
                for (int f = 0; f < 9; ++f) u_in[f] = t.x[l][9 * v + f];
                u_in[9] = t.S[l][v];
                u_in[10] = t.M[l][v];
                for (int f = 0; f < 9; ++f) {
                    db4[f] += dxo[f];
                    for (int u = 0; u < GH; ++u) dW4[f * GH + u] += dxo[f] * a3[u];
                }
                for (int u = 0; u < GH; ++u) {
                    double da = 0.0;
                    for (int f = 0; f < 9; ++f) da += W4[f * GH + u] * dxo[f];
                    double dz = da * (1.0 - a3[u] * a3[u]);
                    db3[u] += dz;
                    for (int f = 0; f < 11; ++f) dW3[u * 11 + f] += dz * u_in[f];
                    for (int f = 0; f < 9; ++f) dxl[9 * v + f] += W3[u * 11 + f] * dz;
                    dS[v] += W3[u * 11 + 9] * dz;
                    dM[v] += W3[u * 11 + 10] * dz;
                }
            }
            /* aggregation backward into the block's edge output */
            for (int64_t i = 0; i < n; ++i)
                for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
                    int32_t j = Lcol[p];
                    de[p] += dS[i] + dM[i] / deg[i];
                    if (j != i) de[p] += dS[j] + dM[j] / deg[j];
                }
        }
        /* edge MLP backward: enew = W2 a1 + b2, a1 = tanh(W1 h + b1) */
        const double *W1 = theta + off_edge(l);
        const double *W2 = W1 + GH * 20 + GH;
        double *dW1 = dtheta + off_edge(l);
        double *db1 = dW1 + GH * 20;
        double *dW2 = db1 + GH;
        double *db2 = dW2 + GH;
        double *dec = (double *)calloc((size_t)E, sizeof(double)); /* d ecur[l] */
        for (int64_t i = 0; i < n; ++i)
            for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
                int32_t j = Lcol[p];
                const double *a1 = t.a1[l] + (int64_t)p * GH;
                const double *h = t.h[l] + 20 * (int64_t)p;
                double d = de[p];
                db2[0] += d;
                double dh[20] = {0};
                for (int u = 0; u < GH; ++u) {
                    dW2[u] += d * a1[u];
                    double dz = d * W2[u] * (1.0 - a1[u] * a1[u]);
                    db1[u] += dz;
                    for (int f = 0; f < 20; ++f) {
                        double w = (bf16 & 1) ? or_round_bf16(W1[u * 20 + f]) : W1[u * 20 + f];
                        dW1[u * 20 + f] += dz * h[f];
                        dh[f] += w * dz;
                    }
                }
                dec[p] = dh[0];
                for (int f = 0; f < 9; ++f) dxl[9 * i + f] += dh[2 + f];
                for (int f = 0; f < 9; ++f) dxl[9 * (int64_t)j + f] += dh[11 + f];
            }
        /* move to block l-1: its output feeds ecur[l] and x[l] */
        memcpy(de, dec, sizeof(double) * (size_t)E);
        free(dec);
        memcpy(dx, dxl, sizeof(double) * (size_t)(n * 9));
        memset(dxl, 0, sizeof(double) * (size_t)(n * 9));
    }
    /* GraphNorm backward; dx now holds d x[0] */
    double *dgam = dtheta, *dbet = dtheta + 9, *dalp = dtheta + 18;
    const double *gam = theta;
    for (int f = 0; f < 9; ++f) {
        double sig = t.gn_sig[f], mu = t.gn_mu[f];
        double sb = 0.0, sg = 0.0, sdsig = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double d = dx[9 * v + f], c = t.gn_c[9 * v + f];
            sb += d;
            sg += d * c / sig;
            sdsig += d * gam[f] * c * (-1.0 / (sig * sig));
        }
        dbet[f] = sb;
        dgam[f] = sg;
        double sdc = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double c = t.gn_c[9 * v + f];
            double dc = dx[9 * v + f] * gam[f] / sig + sdsig * c / ((double)n * sig);
            sdc += dc;
        }
        dalp[f] = -mu * sdc;
    }
    free(de); free(dx); free(dxl); free(dS); free(dM); free(deg);
    tape_free(&t);
}

/* ======================================================================
 * A8/A9. The probe (Hutchinson) loss of Eq.(4)-(5) with the COO products of
 * Algorithms 1-2, for m probes z_k (m*n, probe k at z + k*n):
 *   loss = (1/m) sum_k || L (L^T z_k) - A z_k ||_2^2
 * L in its own CSR (tril pattern), A in full CSR. With dL non-NULL also
 *   d loss / d L_ij = (2/m) sum_k (v_i u_j + z_i w_j)   on the pattern,
 * with u = L^T z, v = L u - A z, w = L^T v.
 * ====================================================================== */
double or_probe_loss(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                     const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval,
                     const double *Z, int m, double *dL)
{
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *az = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t E = Lrowptr[n];
    if (dL) memset(dL, 0, sizeof(double) * (size_t)E);
    double loss = 0.0;
    for (int k = 0; k < m; ++k) {
        const double *z = Z + (int64_t)k * n;
        /* Algorithm 2, first gather/scatter: u = L^T z */
        for (int64_t i = 0; i < n; ++i) u[i] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) u[Lcol[p]] += Lval[p] * z[i];
        /* Algorithm 2, second round: v = L u ; Algorithm 1: A z */
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) s += Lval[p] * u[Lcol[p]];
            v[i] = s;
        }
        or_spmv(n, rowptr, col, val, z, az);
        double q = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            v[i] -= az[i];
            q += v[i] * v[i];
        }
        loss += q;
        if (dL) {
            for (int64_t i = 0; i < n; ++i) w[i] = 0.0;
            for (int64_t i = 0; i < n; ++i)
                for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) w[Lcol[p]] += Lval[p] * v[i];
            for (int64_t i = 0; i < n; ++i)
                for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
                    int32_t j = Lcol[p];
                    dL[p] += (2.0 / m) * (v[i] * u[j] + z[i] * w[j]);
                }
        }
    }
    free(u); free(v); free(w); free(az);
    return loss / m;
}

/* ======================================================================
 * A10. Adam (Training and Inference: Adam, learning rate 0.005 with
 * warm-up). beta1 0.9, beta2 0.999, eps 1e-8; t is the 1-based step.
 * ====================================================================== */
void or_adam_step(int64_t np, double *theta, const double *grad, double *m1, double *m2,
                  int t, double lr)
{
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t k = 0; k < np; ++k) {
        m1[k] = b1 * m1[k] + (1.0 - b1) * grad[k];
        m2[k] = b2 * m2[k] + (1.0 - b2) * grad[k] * grad[k];
        double mh = m1[k] / c1, vh = m2[k] / c2;
        theta[k] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Learning-rate schedule: linear warm-up over the first warm steps to
 * lr_max, then constant (the paper names a warm-up strategy only). */
double or_lr_at(int t, int warm, double lr_max)
{
    if (warm <= 0 || t >= warm) return lr_max;
    return lr_max * (double)t / (double)warm;
}

/* ======================================================================
 * Fill-in dropout (Supplementary 5, Eq. (10)): an off-diagonal entry of the
 * factor whose absolute value is at most thr is set to zero and removed from
 * the pattern; the diagonal always stays. Writes the kept factor as CSR
 * (out_rowptr n+1, out_col/out_val capacity nnz(L)); returns its nnz.
 * ====================================================================== */
int64_t or_dropout(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval, double thr,
                   int32_t *out_rowptr, int32_t *out_col, double *out_val)
{
    int64_t k = 0;
    out_rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
            int keep = (Lcol[p] == i) || (fabs(Lval[p]) > thr);
            if (keep) {
                out_col[k] = Lcol[p];
                out_val[k] = Lval[p];
                ++k;
            }
        }
        out_rowptr[i + 1] = (int32_t)k;
    }
    return k;
}

/* ======================================================================
 * Deviation of a factor from the IC(0) factor (the diagnostic of the
 * paper's Figure 5): r = |Lpred - LIC| / |LIC| over the entries with
 * LIC != 0. out: mean and max of r on the diagonal, mean and max off the
 * diagonal, the diagonal and off-diagonal entry counts.
 * ====================================================================== */
void or_factor_deviation(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *LIC,
                         const double *Lpred, double *out)
{
    double sd = 0.0, md = 0.0, so = 0.0, mo = 0.0, cd = 0.0, co = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
            if (LIC[p] == 0.0) continue;
            double r = fabs(Lpred[p] - LIC[p]) / fabs(LIC[p]);
            if (Lcol[p] == i) {
                sd += r;
                if (r > md) md = r;
                cd += 1.0;
            } else {
                so += r;
                if (r > mo) mo = r;
                co += 1.0;
            }
        }
    }
    out[0] = cd > 0.0 ? sd / cd : 0.0;
    out[1] = md;
    out[2] = co > 0.0 ? so / co : 0.0;
    out[3] = mo;
    out[4] = cd;
    out[5] = co;
}

/* Row groups: runs of consecutive rows with identical column sets in A, cut
 * every c rows, c being the greatest common divisor of the run lengths when
 * it lies in 2..gmax and gmax otherwise (a hex node's three dofs form one
 * group even where two nodes have identical rows). Writes the start rows and
 * n at the end; returns the group count. */
static int same_row(const int32_t *rowptr, const int32_t *col, int64_t a, int64_t b)
{
    if (rowptr[a + 1] - rowptr[a] != rowptr[b + 1] - rowptr[b]) return 0;
    for (int32_t k = 0; k < rowptr[a + 1] - rowptr[a]; ++k)
        if (col[rowptr[a] + k] != col[rowptr[b] + k]) return 0;
    return 1;
}

int64_t or_row_groups(int64_t n, const int32_t *rowptr, const int32_t *col, int gmax, int32_t *starts)
{
    int64_t g = 0, run = 0;
    for (int64_t i = 1; i <= n; ++i) {
        if (i == n || !same_row(rowptr, col, i - 1, i)) {
            int64_t a = g, b = i - run;
            while (b) {
                int64_t t = a % b;
                a = b;
                b = t;
            }
            g = a;
            run = i;
        }
    }
    int64_t cut = (g >= 2 && g <= gmax) ? g : gmax;
    int64_t ng = 0;
    run = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (i > 0 && !same_row(rowptr, col, i - 1, i)) run = i;
        if ((i - run) % cut == 0) starts[ng++] = (int32_t)i;
    }
    starts[ng] = (int32_t)n;
    return ng;
}

/* Node-granular fill-in dropout: the factor is cut into blocks by the row
 * groups (rows of one group against the columns of one group); an external
 * block -- rows of group g, columns of an earlier group h -- is removed as a
 * whole when every one of its entries is at most thr in absolute value, and
 * group g's own lower block (in-group entries and diagonals) always stays.
 * Output as or_dropout. */
int64_t or_dropout_grouped(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval,
                           double thr, int64_t ngroups, const int32_t *starts, int32_t *out_rowptr,
                           int32_t *out_col, double *out_val)
{
    int64_t *gof = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t g = 0; g < ngroups; ++g)
        for (int32_t i = starts[g]; i < starts[g + 1]; ++i) gof[i] = g;
    int64_t k = 0;
    out_rowptr[0] = 0;
    for (int64_t g = 0; g < ngroups; ++g) {
        int32_t s = starts[g], e = starts[g + 1];
        for (int32_t i = s; i < e; ++i) {
            for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
                int32_t c = Lcol[p];
                int keep = 1;
                if (c < s) { /* external column, in group h */
                    int64_t h = gof[c];
                    keep = 0;
                    for (int32_t r = s; r < e; ++r)
                        for (int32_t q = Lrowptr[r]; q < Lrowptr[r + 1] && Lcol[q] < s; ++q)
                            if (gof[Lcol[q]] == h && fabs(Lval[q]) > thr) keep = 1;
                }
                if (keep) {
                    out_col[k] = c;
                    out_val[k] = Lval[p];
                    ++k;
                }
            }
            out_rowptr[i + 1] = (int32_t)k;
        }
    }
    free(gof);
    return k;
}
