/*
 * gicpcg.h -- C-ABI of the GB300 library for GNN-corrected IC(0)-preconditioned
 * conjugate gradient (arxiv 2412.07127, "Deep Learning-Enhanced Preconditioning
 * for Efficient Conjugate Gradient Solvers in Large-Scale PDE Systems").
 *
 * The calls follow the paper's statement of the problem: a sparse SPD matrix A
 * and a vector b go in, x comes out (Supplementary 2, the "black box" view of
 * PCG); in between the library factors IC(0), corrects L with the GNN
 * (Eq.(2)) and runs PCG (Supplementary Algorithm 1).
 *
 * Conventions (every entry point):
 *  - Return an int status: GIC_OK (0) or a negative GIC_ERR_* code. No call
 *    aborts the process and no call waits without bound: device-side waits
 *    are bounded and report GIC_ERR_TIMEOUT.
 *  - Pointers documented "device" are caller-owned CUDA device memory of the
 *    handle's device (for example torch tensors); pointers documented "host"
 *    are ordinary host memory. The library never frees caller memory.
 *  - Work is enqueued on the handle's stream. Calls that return a value
 *    through a host pointer synchronise that stream before returning.
 *  - Index arrays are int32 and must describe fewer than 2^31 entries
 *    (else GIC_ERR_TOO_LARGE). Values of A, b, x are float64.
 *  - A CSR matrix has sorted, duplicate-free column indices in every row, a
 *    stored diagonal in every row and a structurally symmetric pattern.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef GICPCG_H
#define GICPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define GIC_OK 0
#define GIC_ERR_INVALID_ARG (-1)    /* bad pointer, size or pattern */
#define GIC_ERR_NOT_SPD (-2)        /* IC(0) met a pivot <= 0 or non-finite */
#define GIC_ERR_NO_CONVERGENCE (-3) /* PCG reached maxit */
#define GIC_ERR_TIMEOUT (-4)        /* a bounded device wait ran out */
#define GIC_ERR_CUDA (-5)           /* a CUDA runtime call failed */
#define GIC_ERR_TOO_LARGE (-6)      /* sizes beyond int32 indexing */
#define GIC_ERR_UNSUPPORTED (-7)    /* pattern outside the kernels' limits */
#define GIC_ERR_BREAKDOWN (-8)      /* PCG met r^T z <= 0 or p^T A p <= 0 */
#define GIC_ERR_WORKSPACE (-9)      /* workspace smaller than required */

/* value types of L */
#define GIC_F64 0
#define GIC_F32 1
#define GIC_IDENTITY 2 /* no preconditioner: plain CG (the paper's "None") */

typedef struct gic_handle gic_handle;
typedef struct gic_pattern gic_pattern;

/* ---------------------------------------------------------------- handle */
/* Create a handle on CUDA device `device` that enqueues work on `stream`
 * (a cudaStream_t, borrowed; NULL = the legacy default stream). */
int gic_create(gic_handle **h, int device, void *stream);
int gic_set_stream(gic_handle *h, void *stream);
int gic_destroy(gic_handle *h);
/* Static English text of a status code. */
const char *gic_status_string(int status);
/* Text of the last CUDA failure seen by any handle of this process. */
const char *gic_last_cuda_error(void);

/* ------------------------------------------------- A1: FE assembly
 * The paper's systems come from 3-D static structural FE analysis
 * (Experiments, Datasets; Supplementary 1). This synthetic stand-in is 3-D
 * linear elasticity on the unit cube cut into N^3 trilinear hex elements
 * (2x2x2 Gauss rule, Poisson ratio nu, element e = ex + N*(ey + N*ez) with
 * Young modulus E[e]); the z = 0 face is clamped and its dofs eliminated.
 * Free node (x,y,z), z >= 1, has id x + (N+1)*(y + (N+1)*(z-1)); its dofs
 * are 3*id + c, c = 0,1,2.
 */
/* n = 3N(N+1)^2 and nnz = 9(3N+1)^2(3N-2). Host outputs. */
int gic_fem_hex_sizes(int N, int64_t *n, int64_t *nnz);
/* Assemble nb independent systems into one block-diagonal CSR: system k uses
 * E + k*N^3 (device, float64) and occupies rows/columns [k*n, (k+1)*n).
 * rowptr (nb*n+1), col (nb*nnz) int32 and val (nb*nnz) float64 are device
 * outputs sized by the caller. nb = 1 assembles one system. */
int gic_fem_hex_assemble(gic_handle *h, int N, double nu, int nb, const double *E,
                         int32_t *rowptr, int32_t *col, double *val);

/* ------------------------------------------------- A2: pattern analysis
 * Builds, on the device, the pattern of L = tril(A) (IC(0) keeps A's lower
 * pattern: Introduction; Model Architecture), its transpose, groups of
 * consecutive rows with identical patterns (solved together by one warp) and
 * the level of every row (level 0: no strictly-lower entry; else 1 + the
 * largest level among its strictly-lower columns). rowptr/col (device) are
 * borrowed and must stay valid and unchanged while *P lives. The pattern is
 * library-owned: release it with gic_pattern_destroy. Synchronous.
 * Errors: GIC_ERR_INVALID_ARG for unsorted/duplicate columns, a missing
 * diagonal or an asymmetric pattern; GIC_ERR_TOO_LARGE for nnz >= 2^31. */
int gic_analyze(gic_handle *h, int64_t n, int64_t nnz, const int32_t *rowptr,
                const int32_t *col, gic_pattern **P);
int gic_pattern_destroy(gic_pattern *P);
/* Host outputs (any may be NULL). */
int gic_pattern_info(const gic_pattern *P, int64_t *n, int64_t *nnzA, int64_t *nnzL,
                     int32_t *nlevels, int32_t *ngroups);
/* Copies of the analysis (device outputs, any may be NULL): Lrowptr (n+1),
 * Lcol (nnzL), level (n), group start rows (ngroups+1). */
int gic_pattern_export(gic_handle *h, const gic_pattern *P, int32_t *Lrowptr, int32_t *Lcol,
                       int32_t *level, int32_t *group_start);

/* ------------------------------------------------- A3: IC(0)
 * L on tril(A)'s pattern with (L L^T)_ij = a_ij on that pattern
 * (Introduction; Baseline Methods; Supplementary 2):
 *   L_ij = (a_ij - sum_{k<j} L_ik L_jk) / L_jj,  L_ii = sqrt(a_ii' - sum L_ik^2)
 * with a_ii' = a_ii + alpha*a_ii (alpha = 0: plain IC(0)).
 * valA: device float64, A's values (nnzA, CSR order). valL: device float64
 * output, nnzL values in L's CSR order (tril(A) order).
 * On a pivot <= 0 or non-finite: GIC_ERR_NOT_SPD and *bad_row (host) = the
 * smallest failing row; valL is then undefined. Synchronous. */
int gic_ic0(gic_handle *h, const gic_pattern *P, const double *valA, double *valL,
            double alpha, int64_t *bad_row);
/* IC(0) with the shift restart: alpha = 0, then 1e-3, 2e-3, 4e-3, ... for at
 * most max_tries shifted attempts. *alpha_out (host) = the shift that
 * succeeded (0: none). *bad_row (host, nullable) = failing row of the last try. */
int gic_ic0_auto(gic_handle *h, const gic_pattern *P, const double *valA, double *valL,
                 int max_tries, double *alpha_out, int64_t *bad_row);
/* Copy valL (float64) into float32 (device), the FP32 factor of the mixed
 * precision solve. */
int gic_convert_f64_f32(gic_handle *h, int64_t count, const double *src, float *dst);

/* ------------------------------------------------- A7: PCG building blocks
 * y = A x (CSR SpMV). valA, x, y: device float64. xdoty (nullable, device
 * float64 scalar) receives x^T y. */
int gic_spmv(gic_handle *h, const gic_pattern *P, const double *valA, const double *x,
             double *y, double *xdoty);
/* Forward substitution L y = r, read from Supplementary 5 Eq.(11) as
 * y_i = (r_i - sum_{j<i} L_ij y_j) / L_ii. valL: device, nnzL values of type
 * l_dtype (GIC_F64 or GIC_F32) in L's CSR order; r, y: device float64.
 * ws: device workspace of at least gic_workspace_size(GIC_WS_SOLVE) bytes. */
int gic_lsolve(gic_handle *h, const gic_pattern *P, const void *valL, int l_dtype,
               const double *r, double *y, void *ws, size_t ws_bytes);
/* Back substitution L^T z = y: z_i = (y_i - sum_{j>i} L_ji z_j) / L_ii.
 * Arguments as gic_lsolve (valL is L's values; the transpose is built in ws). */
int gic_ltsolve(gic_handle *h, const gic_pattern *P, const void *valL, int l_dtype,
                const double *y, double *z, void *ws, size_t ws_bytes);

/* Preconditioned CG exactly as Supplementary Algorithm 1 with P = L L^T,
 * stopping when ||r_k||_2 <= rtol * ||b||_2 on the recurrence residual
 * (no iteration is taken if x0 already satisfies it).
 * valA: device float64; valL: device, type l_dtype (GIC_F64, GIC_F32, or
 * GIC_IDENTITY with valL = NULL for plain CG); b: device float64;
 * x: device float64, x0 on entry, solution on exit.
 * Host outputs: *iters = number of x updates, *relres = ||r||/||b|| at exit.
 * CG scalars, dot products and vectors are float64.
 * Returns GIC_OK, GIC_ERR_NO_CONVERGENCE (maxit reached, x is the last
 * iterate), GIC_ERR_BREAKDOWN or GIC_ERR_TIMEOUT. Synchronous. */
int gic_pcg(gic_handle *h, const gic_pattern *P, const double *valA, const void *valL,
            int l_dtype, const double *b, double *x, double rtol, int maxit, int32_t *iters,
            double *relres, void *ws, size_t ws_bytes);

/* Per-kernel-class device time of the solve calls, measured with CUDA
 * events on the handle's stream around every launch while enabled (the PCG
 * loop then synchronises after each launch, so enable it only to profile).
 * Classes: GIC_PROF_LSOLVE, GIC_PROF_LTSOLVE, GIC_PROF_SPMV, GIC_PROF_VECTOR.
 * gic_profile_enable clears the counters; gic_profile_read copies them to
 * host arrays of GIC_PROF_CLASSES entries (milliseconds, launch counts). */
#define GIC_PROF_LSOLVE 0
#define GIC_PROF_LTSOLVE 1
#define GIC_PROF_SPMV 2
#define GIC_PROF_VECTOR 3
#define GIC_PROF_CLASSES 4
int gic_profile_enable(gic_handle *h, int on);
int gic_profile_read(gic_handle *h, double *ms, int64_t *launches);
/* Reads and clears the device error flags of the handle (host output;
 * bit 0: a bounded wait ran out). Synchronous. */
int gic_solve_error_flags(gic_handle *h, unsigned *flags);

/* Workspace sizes (host output, bytes) of the calls that take one. */
#define GIC_WS_SOLVE 0 /* gic_lsolve / gic_ltsolve */
#define GIC_WS_PCG 1   /* gic_pcg */
int gic_workspace_size(gic_handle *h, const gic_pattern *P, int op, int l_dtype, size_t *bytes);

#ifdef __cplusplus
}
#endif
#endif /* GICPCG_H */
