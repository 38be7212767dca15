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
 * consecutive rows with identical patterns (solved together; runs of such
 * rows are cut at their common length when it is 2..8, else every 8 rows) and
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
/* Schedule of the sync-free kernels (host outputs, any may be NULL): number
 * of chunks (runs of row groups one warp processes in order), how they are
 * ordered -- 0: single groups in level order; 1: multi-group runs in order of
 * their first (forward) or last (backward) level; 2: multi-group runs in a
 * topological order of their dependencies, taken when the level order would
 * start a run before one it reads (as thinning a factor can make) -- and the
 * padded entry count of the SELL-32 copy of A the PCG SpMV uses for patterns
 * not made of 3x3 node blocks (0 for those that are: they run the block
 * SpMV, see gic_pattern_spmv_layout). */
int gic_pattern_schedule(const gic_pattern *P, int32_t *nchunks, int32_t *chunked, int64_t *sell_nnz);
/* SpMV layout the PCG uses for this pattern (host outputs, any may be NULL):
 * node_blocks = 1 if A is made of 3x3 node blocks (runs of 3 rows from a
 * multiple of 3 with identical columns in aligned triples: the hex systems),
 * which then run the block SpMV, else 0 (SELL-32 CSR); entries = values in
 * that layout, padding included. */
int gic_pattern_spmv_layout(const gic_pattern *P, int32_t *node_blocks, int64_t *entries);
/* The triangular-solve kernels gic_pcg / gic_lsolve / gic_ltsolve will run on
 * this pattern for a factor of l_dtype (GIC_F64 or GIC_F32) under the
 * handle's current tuning (host output): 3 level-sliced, 2 warp-specialised,
 * 1 staged one-warp, 0 generic. */
int gic_solve_kernels_chosen(gic_handle *h, const gic_pattern *P, int l_dtype, int32_t *pipeline);
/* Which triangular-solve kernels the pattern admits (host outputs, any may be
 * NULL): warp-specialised (1/0), level-sliced (1/0; one lane per row, slices
 * of whole row groups of one level) and the forward sweep's slice count. */
int gic_pattern_solve_kernels(const gic_pattern *P, int32_t *warp_specialised, int32_t *level_sliced,
                              int32_t *slices);
/* Pair-sliced schedule of an analysed pattern (outputs host, any may be
 * NULL): *mode = 1 paired levels, 2 one level per step, 0 or negative: not
 * built (-bits: 1 a group substitutes more than 3 groups, 2 a column outside
 * the earlier pairs, 4/8/16/32 a far / near / right-hand-side / early list
 * beyond the kernels' register budget, 128 groups of more than 3 rows, 256
 * not asked for: built when GIC_TUNE_PIPELINE is 5 at analysis time, or
 * automatic and the system in the band where the automatic choice takes
 * these kernels);
 * *slices = forward slices; *glevels = group levels (longest chain of
 * dependent row groups). */
int gic_pattern_pair_schedule(const gic_pattern *P, int32_t *mode, int32_t *slices, int32_t *glevels);
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
/* PCG as gic_pcg with the factor on a pattern of its own: the SpMV runs on
 * PA (the matrix), the triangular solves on the lower triangle of PL (same n),
 * for instance a factor thinned by gic_dropout. ws: device workspace of
 * gic_workspace_size_split bytes. Same outputs and status codes as gic_pcg. */
int gic_workspace_size_split(gic_handle *h, const gic_pattern *PA, const gic_pattern *PL,
                             int l_dtype, size_t *bytes);
int gic_pcg_split(gic_handle *h, const gic_pattern *PA, const double *valA, const gic_pattern *PL,
                  const void *valL, int l_dtype, const double *b, double *x, double rtol, int maxit,
                  int32_t *iters, double *relres, void *ws, size_t ws_bytes);

/* --------------------------- fill-in dropout, deviation, direct prediction
 * Fill-in dropout (Supplementary 5, Eq. (10)): off-diagonal factor entries
 * with |L_ij| <= threshold become zero and leave the pattern; the diagonal is
 * always kept. Eq. (10)'s epsilon applies to the scaled factor L/sqrt(s), so
 * threshold = epsilon * sqrt(s). valL: device float64, nnzL values on P.
 * Outputs (caller-owned device memory): the symmetric pattern S = L' + L'^T
 * of the kept factor, Srowptr (n+1) and Scol (capacity nnzA), ready for
 * gic_analyze; Lval_out (capacity nnzL) = the kept values in the CSR order
 * of tril(S). Host outputs: *nnzS, *nnzL_out. */
int gic_dropout(gic_handle *h, const gic_pattern *P, const double *valL, double threshold,
                int32_t *Srowptr, int32_t *Scol, double *Lval_out, int64_t *nnzS, int64_t *nnzL_out);
/* Node-granular variant (no counterpart in the paper; it keeps the row-group
 * structure the fast solve kernels need): the factor is cut into blocks by
 * the row groups of P (rows with identical patterns, a hex node's three
 * dofs); an external block (rows of group g, columns of an earlier group h)
 * is dropped whole when every entry in it is at most threshold and kept
 * whole otherwise; each group's own lower block always stays. The rows of a
 * group then keep identical patterns in S, so gic_analyze of S finds the
 * same groups. Arguments and outputs as gic_dropout. */
int gic_dropout_grouped(gic_handle *h, const gic_pattern *P, const double *valL, double threshold,
                        int32_t *Srowptr, int32_t *Scol, double *Lval_out, int64_t *nnzS, int64_t *nnzL_out);
/* Deviation of a factor from the IC(0) factor (the diagnostic of the paper's
 * Figure 5): |Lpred_ij - LIC_ij| / |LIC_ij| over entries with LIC_ij != 0.
 * LIC, Lpred: device float64 on P. out (host, 6 values): mean and maximum on
 * the diagonal, mean and maximum off the diagonal, the two entry counts. */
int gic_factor_deviation(gic_handle *h, const gic_pattern *P, const double *LIC, const double *Lpred,
                         double *out);
/* Base factor of the direct prediction L = GNN(A) (Eq. (1), the paper's
 * "NIC" ablation): correcting it with gic_gnn_correct (or, scaled, with
 * gic_gnn_correct_scaled) gives off-diagonal g and diagonal exp(g/2).
 * Writes (device, nnzL values, either may be NULL): L = sqrt(s_k) on the
 * diagonal of graph k and 0 elsewhere (scale: device float64 [ngraphs] from
 * gic_features), Lhat = 1 on the diagonal and 0 elsewhere (float32). */
int gic_identity_factor(gic_handle *h, const gic_pattern *P, int ngraphs, const double *scale, double *L,
                        float *Lhat);

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

/* ------------------------------------------------- A4-A6: the GNN correction
 * A batch is a block-diagonal pattern of `ngraphs` graphs of equal size
 * (n divisible by ngraphs; ngraphs = 1 for one matrix). Per-graph statistics
 * (the scale s, GraphNorm) are computed per graph.
 * Parameters (theta, float32, gic_gnn_param_count() = 3504 values):
 *   GraphNorm gamma[9], beta[9], alpha[9]; then for block l = 0,1,2 the edge
 *   MLP W1[32][20], b1[32], W2[32], b2[1], and for l = 0,1 the node MLP
 *   W3[32][11], b3[32], W4[9][32], b4[9]. */
int gic_gnn_param_count(void);
/* Graph inputs (Model Architecture; Supplementary 4, Table 2): per graph
 * s = population standard deviation of tril(A)'s stored values; edge feature
 * e0 = a_ij / s on L's pattern (nnzL float32, device); node features x9
 * (n x 9 float32, device): degree, max/min/mean/variance of the neighbours'
 * degrees, dominance |a_ii| / sum_{j!=i} |a_ij|, decay |a_ii| / max_{j!=i}
 * |a_ij|, sin(i) and cos(i) of the row index within its graph (0 where a
 * denominator or the neighbour set is empty). Ahat (nullable, nnzA float32)
 * receives A / s. scale_dev (device, ngraphs float64) receives s;
 * scale_host (nullable, host) too, then the call synchronises. */
int gic_features(gic_handle *h, const gic_pattern *P, int ngraphs, const double *valA, float *x9,
                 float *e0, float *Ahat, double *scale_dev, double *scale_host);
/* Workspace (bytes, host output) of gic_gnn_forward (training = 0) or of
 * gic_gnn_forward_train + gic_gnn_backward (training = 1). */
int gic_gnn_workspace_size(gic_handle *h, const gic_pattern *P, int ngraphs, int training,
                           size_t *bytes);
/* g = GNN(A) on L's pattern (Eq.(7)-(9); Model Architecture): GraphNorm of
 * x9, then 3 blocks of edge MLP 20->32->1 (tanh) on [e_cur, e0, x_i, x_j],
 * sum and mean of the new edge values over each node's incident edges (a
 * self-loop once), node MLP 11->32->9 (tanh) on [x, sum, mean] (none in the
 * last block). theta, x9, e0: device float32; g: device float32 (nnzL).
 * FP32 arithmetic. */
int gic_gnn_forward(gic_handle *h, const gic_pattern *P, int ngraphs, const float *theta,
                    const float *x9, const float *e0, float *g, void *ws, size_t ws_bytes);
/* Same forward, keeping every layer's activations in ws for gic_gnn_backward. */
int gic_gnn_forward_train(gic_handle *h, const gic_pattern *P, int ngraphs, const float *theta,
                          const float *x9, const float *e0, float *g, void *ws, size_t ws_bytes);
/* dtheta (device float32, 3504) = d(loss)/d(theta) given dg = d(loss)/dg,
 * after gic_gnn_forward_train with the same inputs and ws. Deterministic. */
int gic_gnn_backward(gic_handle *h, const gic_pattern *P, int ngraphs, const float *theta,
                     const float *x9, const float *e0, const float *dg, float *dtheta, void *ws,
                     size_t ws_bytes);
/* Eq.(2) with the exp-then-sqrt diagonal map, original units, float64:
 * Lout_ij = LIC_ij + sqrt(s) g_ij (i > j), Lout_ii = LIC_ii exp(g_ii / 2).
 * *diag_ok (host, nullable; the call then synchronises) = 1 if every
 * diagonal is positive and finite (else the caller keeps LIC). */
int gic_gnn_correct(gic_handle *h, const gic_pattern *P, int ngraphs, const double *LIC,
                    const float *g, const double *scale_dev, double *Lout, int *diag_ok);
/* LIChat = LIC / sqrt(s) per graph (float32): the factor in units scaled by s. */
int gic_scale_factor(gic_handle *h, const gic_pattern *P, int ngraphs, const double *LIC,
                     const double *scale_dev, float *LIChat);
/* Correction in scaled units, float32: Lhat = LIChat + g, diagonal
 * LIChat exp(g / 2); and its backward dg = dLhat (off-diagonal),
 * dLhat * Lhat / 2 (diagonal). */
int gic_gnn_correct_scaled(gic_handle *h, const gic_pattern *P, const float *LIChat, const float *g,
                           float *Lhat);
int gic_gnn_correct_backward(gic_handle *h, const gic_pattern *P, const float *Lhat,
                             const float *dLhat, float *dg);

/* ------------------------------------------------- A8-A10: training
 * Probe (Hutchinson) loss of Eq.(4)-(5) with the index/value products of
 * Algorithms 1-2, in scaled units: per graph
 *   loss_g = (1/m) sum_k || Lhat (Lhat^T z_k) - Ahat z_k ||_2^2
 * and loss[ngraphs] = their mean. Ahat: nnzA float32 (A / s); Lhat: nnzL
 * float32; Z: m x n float32 probes (probe k at Z + k*n), 1 <= m <= 16;
 * loss: device float32, ngraphs + 1 values. dLhat (nullable, nnzL float32)
 * receives d loss[ngraphs] / d Lhat on the pattern:
 *   (2 / (m ngraphs)) sum_k (v_k,i u_k,j + z_k,i w_k,j),
 * u = Lhat^T z, v = Lhat u - Ahat z, w = Lhat^T v. */
int gic_probe_workspace_size(gic_handle *h, const gic_pattern *P, int ngraphs, int m, size_t *bytes);
int gic_probe_loss(gic_handle *h, const gic_pattern *P, int ngraphs, const float *Ahat,
                   const float *Lhat, const float *Z, int m, float *loss, float *dLhat, void *ws,
                   size_t ws_bytes);
/* One Adam step (Training and Inference: Adam with warm-up; beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected, t = 1-based step) on np float32
 * values in place (theta, first and second moments m1, m2). */
int gic_adam_step(gic_handle *h, int64_t np, float *theta, const float *grad, float *m1,
                  float *m2, int t, double lr);

/* Tuning of the sync-free kernels (IC(0), triangular solves); results agree
 * to round-off across settings: GIC_TUNE_SOLVE_WARPS_PER_SM = cap on resident
 * solve warps (teams of three warps for the warp-specialised solves) per SM
 * (0 = automatic: 4, 8 or 16 teams by chunks per SM; 32 warps for the
 * level-sliced solves); GIC_TUNE_POLL =
 * polling: low 16 bits = nanoseconds slept between polls, bit 16 set = one
 * polling lane per warp (default 1<<16);
 * GIC_TUNE_PIPELINE = triangular-solve kernels: 4 (default) = automatic
 * (below 48 chunks per SM warp-specialised, up to 120 pair-sliced, above
 * level-sliced, each where the pattern admits them, else staged one-warp),
 * 5 = pair-sliced solves (two
 * lanes per row; the group levels taken two at a time, the second level's
 * reads of the first substituted by their own solve, so one cross-SM
 * hand-off serves two levels) where the analysis built them, else as 3;
 * 3 = level-sliced solves (one
 * lane per row; slices of whole row groups of one level, premultiplied
 * blocks) where the pattern admits them, else 2 = warp-specialised solves on
 * premultiplied row-group blocks (groups of <= 3 rows, <= 61 external
 * columns), else 1 = staged one-warp solves (<= 3 rows, <= 48 columns),
 * else 0 = generic; a lower value caps the
 * choice; GIC_TUNE_QDELTA = level
 * window of the dependencies the warp-specialised solves treat as "late"
 * (read by gic_analyze; default 6); GIC_TUNE_GNN_BF16 = 1 (default): the
 * inference forward (gic_gnn_forward, gic_solve_host) runs the edge MLP's
 * first layer on the tensor cores with BF16 inputs and weights and FP32
 * accumulation, 0: FP32 on the CUDA cores; GIC_TUNE_TRAIN_BF16 = 0 (default):
 * the training forward (gic_gnn_forward_train) and backward (gic_gnn_backward)
 * compute the edge MLP in FP32, 1: in BF16 as inference does (tensor cores,
 * BF16 inputs and W1, FP32 accumulation; FP32 master weights), the backward
 * recomputing the hidden layer from the same BF16-rounded inputs and W1 and
 * passing the gradient straight through the rounding (both calls must see
 * the same setting); GIC_TUNE_PAIR_LEVELS (read by gic_analyze) = 0
 * (default): the pair-sliced schedule pairs the levels, 1: one level per
 * step (the same two-lanes-per-row kernels without substitution). */
#define GIC_TUNE_SOLVE_WARPS_PER_SM 1
#define GIC_TUNE_POLL 2
#define GIC_TUNE_PIPELINE 3
#define GIC_TUNE_QDELTA 4
#define GIC_TUNE_GNN_BF16 5
#define GIC_TUNE_TRAIN_BF16 6
#define GIC_TUNE_PAIR_LEVELS 7
int gic_set_tuning(gic_handle *h, int key, int value);

/* Failure-path self-test of the bounded device waits: one warp waits on a
 * word that nothing writes, giving up after `polls` polls (1..2^21). Returns
 * GIC_ERR_TIMEOUT (the expected outcome: the wait ran out, was reported and
 * the handle stays usable) or GIC_OK if the wait unexpectedly ended. */
int gic_selftest_wait_timeout(gic_handle *h, int64_t polls);

/* y = A x and *xdoty = x^T y for callers that cannot allocate device memory
 * (inside another allocator, under a fixed memory budget, or where a
 * synchronous allocation is not allowed). No paper counterpart: same
 * arithmetic as gic_spmv, but it needs no handle, no pattern and no
 * workspace, and allocates nothing. Its scratch (partial sums and a
 * counter) is a file-scope device array of about 8 MiB that every GPU
 * loading this library holds until exit. The first call in a CUDA context
 * (a device's primary context, another driver context, or the primary context
 * again after cudaDeviceReset) looks up that array's device address in that
 * context, so make it before any stream capture: a first call whose stream
 * is being captured returns GIC_ERR_UNSUPPORTED.
 * Calls share the scratch: calls that overlap on the GPU (other streams)
 * race; calls in one stream are ordered. rowptr (n+1), col, val, x, y,
 * xdoty: device memory of the current device; stream: a cudaStream_t
 * (NULL = legacy default). n is limited to 8,388,608 rows (larger:
 * GIC_ERR_TOO_LARGE). Asynchronous. */
int gic_spmv_dot_noalloc(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                         const double *x, double *y, double *xdoty, void *stream);

/* Number of kernels this handle has launched so far (host output). */
int gic_launch_count(gic_handle *h, int64_t *count);

/* ------------------------------------------------- end to end
 * The paper's black-box use of PCG (Supplementary 2): A and b in host memory
 * in, x in host memory out. Copies A (CSR: rowptr n+1, col nnz int32; val
 * nnz float64) and b (n float64) to the device, analyses the pattern,
 * factors IC(0) with the shift restart, corrects L with the GNN when theta
 * (host float32, gic_gnn_param_count() values) is non-NULL, runs PCG from
 * x0 = 0 with the factor in l_dtype precision (GIC_F64 or GIC_F32) and copies
 * x (n float64) back. Host buffers may be pageable or pinned. ws: device
 * workspace of gic_solve_host_workspace_size() bytes. Host outputs: iters,
 * relres, and (nullable) alpha = the IC(0) shift used and used_gnn = 1 if the
 * corrected factor was kept (0 if it fell back to plain IC(0) because its
 * diagonal was not positive and finite). Synchronous. */
int gic_solve_host(gic_handle *h, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                   const double *val, const double *b, double *x, const float *theta, int l_dtype,
                   double rtol, int maxit, int32_t *iters, double *relres, double *alpha,
                   int *used_gnn, void *ws, size_t ws_bytes);
int gic_solve_host_workspace_size(gic_handle *h, int64_t n, int64_t nnz, int with_gnn, int l_dtype,
                                  size_t *bytes);

/* Workspace sizes (host output, bytes) of the calls that take one. */
#define GIC_WS_SOLVE 0 /* gic_lsolve / gic_ltsolve */
#define GIC_WS_PCG 1   /* gic_pcg */
int gic_workspace_size(gic_handle *h, const gic_pattern *P, int op, int l_dtype, size_t *bytes);

#ifdef __cplusplus
}
#endif
#endif /* GICPCG_H */
