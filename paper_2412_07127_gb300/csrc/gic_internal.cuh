// gic_internal.cuh -- shared device/host helpers of the CUDA library.
// Nothing here is visible through the C-ABI; include/gicpcg.h is the boundary.
#pragma once
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/gicpcg.h"

namespace gic {

// ---------------------------------------------------------------- errors
#define GIC_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            gic::set_last_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return GIC_ERR_CUDA;                             \
        }                                                    \
    } while (0)

#define GIC_TRY(expr)                  \
    do {                               \
        int s_ = (expr);               \
        if (s_ != GIC_OK) return s_;   \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Device error flags (bit set in handle->dev_err).
enum : unsigned { ERR_TIMEOUT = 1u, ERR_BOUNDS = 2u };

// Spin-wait limit: polls of one word before a waiting warp gives up, sets
// ERR_TIMEOUT and writes NaN so that everything downstream drains (about a
// second: a poll is an L2 round trip, then sleeps after the first 2^16).
constexpr long long SPIN_LIMIT = 1ll << 21;

// A quiet-NaN bit pattern that arithmetic never produces (the GPU's
// canonical NaN differs), used as "not written yet" in solve outputs.
constexpr unsigned long long SENTINEL_BITS = 0x7ff4dead0000beefull;

__device__ __forceinline__ double sentinel_d() { return __longlong_as_double((long long)SENTINEL_BITS); }
__device__ __forceinline__ bool is_sentinel(double v)
{
    return (unsigned long long)__double_as_longlong(v) == SENTINEL_BITS;
}

// Relaxed load of a value that is its own ready flag (no other data is read
// on the strength of it; code that reads other data after a wait puts a
// fence in between). The FP64 flavour keeps a "memory" clobber, the FP32 one
// does not: without it the compiler may move shared-memory reads ahead of the
// load (a volatile asm is still never merged, hoisted out of a polling loop
// or reordered with another volatile asm). Measured on the triangular
// solves: the FP32 sweeps are 10-25% faster without the clobber, the FP64
// ones 4-16% slower (their FMA chains are scheduled worse).
__device__ __forceinline__ double ld_relaxed(const double *p)
{
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_acquire(const double *p)
{
    unsigned long long u;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(u) : "l"(p) : "memory");
    return __longlong_as_double((long long)u);
}
__device__ __forceinline__ void st_relaxed(double *p, double v)
{
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_release(double *p, double v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"((unsigned long long)__double_as_longlong(v))
                 : "memory");
}
__device__ __forceinline__ int ld_acquire_i32(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *p is no longer the sentinel; bounded. Polls with relaxed
// loads (each poll is one L2 round trip), sleeping sleep_ns between polls
// (0: none), and after 2^16 polls at least 128 ns. After `limit` polls it
// gives up, sets ERR_TIMEOUT and returns NaN.
__device__ __forceinline__ double wait_value(const double *p, unsigned *err, long long limit = SPIN_LIMIT,
                                             unsigned sleep_ns = 0)
{
    double v = ld_relaxed(p);
    if (!is_sentinel(v)) return v;
    for (long long it = 0; it < limit; ++it) {
        if (it > 65536) __nanosleep(128);
        else if (sleep_ns) __nanosleep(sleep_ns);
        v = ld_relaxed(p);
        if (!is_sentinel(v)) return v;
        if ((it & 255) == 255 && *((volatile unsigned *)err) != 0u) return __longlong_as_double(0x7ff8000000000000ll);
    }
    atomicOr(err, ERR_TIMEOUT);
    return __longlong_as_double(0x7ff8000000000000ll);
}

// Polling configuration of the sync-free kernels: low 16 bits = sleep
// between polls in ns, POLL_ONE_LANE = only the lane holding the outstanding
// dependency produced last polls, the others reload once it lands.
constexpr int POLL_ONE_LANE = 1 << 16;

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// float flavour of the sentinel machinery (FP32 preconditioner vectors)
constexpr unsigned SENTINEL_BITS_F = 0x7fa0beefu; // signalling-NaN payload
__device__ __forceinline__ float sentinel_f() { return __uint_as_float(SENTINEL_BITS_F); }
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == SENTINEL_BITS_F; }
__device__ __forceinline__ float ld_relaxed(const float *p)
{
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_relaxed(float *p, float v)
{
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
template <typename T> __device__ __forceinline__ T sentinel_of();
template <> __device__ __forceinline__ double sentinel_of<double>() { return sentinel_d(); }
template <> __device__ __forceinline__ float sentinel_of<float>() { return sentinel_f(); }
template <typename T> __device__ __forceinline__ T qnan_of();
template <> __device__ __forceinline__ double qnan_of<double>() { return __longlong_as_double(0x7ff8000000000000ll); }
template <> __device__ __forceinline__ float qnan_of<float>() { return __uint_as_float(0x7fc00000u); }

// generic bounded wait (same policy as wait_value)
template <typename T>
__device__ __forceinline__ T wait_word(const T *p, unsigned *err, unsigned sleep_ns)
{
    T v = ld_relaxed(p);
    if (!is_sentinel(v)) return v;
    for (long long it = 0; it < SPIN_LIMIT; ++it) {
        if (it > 65536) __nanosleep(128);
        else if (sleep_ns) __nanosleep(sleep_ns);
        v = ld_relaxed(p);
        if (!is_sentinel(v)) return v;
        if ((it & 255) == 255 && *((volatile unsigned *)err) != 0u) return qnan_of<T>();
    }
    atomicOr(err, ERR_TIMEOUT);
    return qnan_of<T>();
}

// outstanding dependencies of a lane (at most two words): one polling lane
// at a time (the one holding the dependency produced last), or all lanes
template <bool LAST_IS_MAX, typename T>
__device__ __forceinline__ void wait_pair(const T *y, int32_t j0, int32_t j1, T &y0, T &y1, unsigned *err, int poll)
{
    const unsigned sl = (unsigned)(poll & 0xffff);
    bool p0 = j0 >= 0 && is_sentinel(y0), p1 = j1 >= 0 && is_sentinel(y1);
    if (!(poll & POLL_ONE_LANE)) {
        if (p0) y0 = wait_word(y + j0, err, sl);
        if (p1) y1 = wait_word(y + j1, err, sl);
        return;
    }
    unsigned pend = __ballot_sync(0xffffffffu, p0 || p1);
    for (int round = 0; pend && round < 130; ++round) {
        int32_t mine, jm;
        if (LAST_IS_MAX) {
            mine = max(p0 ? j0 : -1, p1 ? j1 : -1);
            jm = __reduce_max_sync(0xffffffffu, mine);
        } else {
            mine = min(p0 ? j0 : INT_MAX, p1 ? j1 : INT_MAX);
            jm = __reduce_min_sync(0xffffffffu, mine);
        }
        if (mine == jm) wait_word(y + jm, err, sl);
        __syncwarp();
        if (p0) { y0 = ld_relaxed(y + j0); p0 = is_sentinel(y0); }
        if (p1) { y1 = ld_relaxed(y + j1); p1 = is_sentinel(y1); }
        pend = __ballot_sync(0xffffffffu, p0 || p1);
        if (pend && *((volatile unsigned *)err) != 0u) break;
    }
    if (p0) y0 = qnan_of<T>();
    if (p1) y1 = qnan_of<T>();
}

// Asynchronous global -> shared copies (no register staging); a thread's
// copies complete in commit-group order.
__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_t(T *smem, const T *gmem)
{
    if (sizeof(T) == 8) cp_async_8(smem, gmem);
    else cp_async_4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Wait until neither of a lane's two dependency values is the sentinel.
// With POLL_ONE_LANE one lane at a time polls, the one holding the
// outstanding dependency produced last (the largest column in the forward
// sweep, LAST_IS_MAX; the smallest in the backward one); otherwise every lane
// polls its own words concurrently.
template <bool LAST_IS_MAX>
__device__ __forceinline__ void wait_deps(const double *y, int32_t j0, int32_t j1, double &y0, double &y1,
                                          unsigned *err, int poll)
{
    const unsigned sl = (unsigned)(poll & 0xffff);
    bool p0 = j0 >= 0 && is_sentinel(y0), p1 = j1 >= 0 && is_sentinel(y1);
    if (!(poll & POLL_ONE_LANE)) {
        if (p0) y0 = wait_value(y + j0, err, SPIN_LIMIT, sl);
        if (p1) y1 = wait_value(y + j1, err, SPIN_LIMIT, sl);
        return;
    }
    unsigned pend = __ballot_sync(0xffffffffu, p0 || p1);
    for (int round = 0; pend && round < 130; ++round) {
        int32_t mine, jm;
        if (LAST_IS_MAX) {
            mine = max(p0 ? j0 : -1, p1 ? j1 : -1);
            jm = __reduce_max_sync(0xffffffffu, mine);
        } else {
            mine = min(p0 ? j0 : INT_MAX, p1 ? j1 : INT_MAX);
            jm = __reduce_min_sync(0xffffffffu, mine);
        }
        if (mine == jm) wait_value(y + jm, err, SPIN_LIMIT, sl);
        __syncwarp();
        if (p0) { y0 = ld_relaxed(y + j0); p0 = is_sentinel(y0); }
        if (p1) { y1 = ld_relaxed(y + j1); p1 = is_sentinel(y1); }
        pend = __ballot_sync(0xffffffffu, p0 || p1);
        if (pend && *((volatile unsigned *)err) != 0u) break;
    }
    if (p0) y0 = __longlong_as_double(0x7ff8000000000000ll);
    if (p1) y1 = __longlong_as_double(0x7ff8000000000000ll);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- pattern
// Analysis of one symmetric CSR pattern (device arrays, library owned).
// One sweep's level-sliced schedule: per slice its width w (column steps),
// the early part's width we (steps [0, we): early columns; [we, w): late and
// previous-group ones, each part front-padded per group), its group count
// ng, the offset of its first step in the coefficient arrays (kv, in steps
// of 32 values) and in the column array (kc); per slice 32 lane descriptors
// (row or -1, slot | t << 8 | G << 16 | ne << 24: the group's slot in the
// slice, the row's index in its group, the group's size, its early column
// count); the columns of slot i at step k at col[kc + k ng + i] (-1: padding).
struct SliceSched {
    int32_t nsl = 0;
    int64_t steps = 0, ncol = 0;
    int32_t *w = nullptr, *we = nullptr, *ng = nullptr;
    int64_t *kv = nullptr, *kc = nullptr;
    int2 *lane = nullptr;
    int32_t *col = nullptr;
};

// Pair-sliced schedule of one sweep (gic_psolve.cu): slices of whole groups
// with at most 16 rows, two lanes per row (lane 2i + h: row i of the slice,
// half h), each half taking every other column of each part of the group's
// list. Per slice: w steps per lane, of which we early and wf far (the rest
// near), wr right-hand-side steps, ng groups; kv / kr = first coefficient
// step (32 values each), kc / krc = first column word (2 per group and step).
struct PairSched {
    int32_t nsl = 0;
    int64_t steps = 0, ncol = 0, rsteps = 0, nrcol = 0;
    int32_t *w = nullptr, *we = nullptr, *wf = nullptr, *wr = nullptr, *ng = nullptr;
    int64_t *kv = nullptr, *kc = nullptr, *kr = nullptr, *krc = nullptr;
    int2 *lane = nullptr;
    int32_t *col = nullptr, *rcol = nullptr;
};

struct Pattern {
    int64_t n = 0, nnzA = 0, nnzL = 0;
    int32_t ngroups = 0, nlevels = 0;
    int32_t block_rows = 8; // rows at which runs of identical rows are cut into groups
    int32_t max_ext_lower = 0, max_ext_upper = 0, max_group = 0;
    // A (borrowed, caller owned; must outlive the pattern)
    const int32_t *rowptr = nullptr, *col = nullptr;
    // L = tril(A) CSR; L entry p of row i is A entry rowptr[i] + (p - Lrowptr[i])
    int32_t *Lrowptr = nullptr, *Lcol = nullptr;
    // U = L^T CSR (the diagonal first in each row); tperm[q] = L position
    int32_t *Urowptr = nullptr, *Ucol = nullptr, *tperm = nullptr;
    // groups of consecutive rows with identical A patterns (<= GMAX rows)
    int32_t *grp = nullptr;   // ngroups+1 start rows
    int32_t *rowgrp = nullptr; // n: the first row of each row's group
    int32_t *level = nullptr; // n row levels
    int32_t *Lrow = nullptr;  // nnzL: row of every L entry (edge -> its row node)
    // Solve schedule: chunks = runs of consecutive groups with increasing
    // levels (for hex elasticity the x-pencils), ordered by start level for
    // the forward sweep and by end level (descending) for the backward one.
    // Every cross-chunk dependency points to an earlier chunk in that order
    // (checked; otherwise every group is its own chunk, in level order).
    int32_t nchunks = 0;
    int chunked = 0; // 0 single groups, 1 runs in level order, 2 runs in key order
    int32_t *chunk_grp = nullptr;     // nchunks+1 start groups
    int32_t *ord_f = nullptr, *ord_b = nullptr;
    // SELL-32 layout of A's pattern for SpMV: slices of 32 rows, column-major
    // inside a slice, padded to the slice's longest row with the row itself.
    int64_t nslices = 0, sell_nnz = 0;
    int64_t *sell_ptr = nullptr;      // nslices+1 entry offsets
    int32_t *sell_w = nullptr;        // nslices widths
    int32_t *sell_col = nullptr;      // sell_nnz column indices
    // 3x3 node-block copy of A's pattern for the PCG SpMV (gic_bsr.cu), where
    // A is made of them: slices of 32 nodes, bsr_ptr[s] = first block step
    // of slice s, bsr_w[s] = its width, bsr_col = node column per (step, lane)
    int bsr_ready = 0;
    int64_t bsr_nsl = 0, bsr_steps = 0;
    int64_t *bsr_ptr = nullptr;
    int32_t *bsr_w = nullptr, *bsr_col = nullptr;
    // Schedule of the warp-specialised solves (groups of <= 3 rows with at
    // most QCOL - 3 external columns): every group's external columns in the
    // order [early | late | prev] -- prev: rows of the group solved just
    // before it in its chunk; late: columns within qdelta levels of the
    // group (finished shortly before it); early: the rest -- with the
    // original position of each column in the group's rows. Forward data
    // sit at the group's first L offset (Lrowptr[s]), backward data at its
    // first U offset (Urowptr[s]); qf_cnt / qb_cnt pack the counts as
    // ne | nl << 8 | np << 16 | G << 24.
    int qready = 0, qdelta = 0;
    int32_t *qf_col = nullptr, *qb_col = nullptr;
    uint8_t *qf_pos = nullptr, *qb_pos = nullptr;
    int32_t *qf_cnt = nullptr, *qb_cnt = nullptr;
    // Level-sliced schedule (one lane per row, gic_ssolve.cu), per sweep:
    // the groups sorted by level (forward: first row's, ascending; backward:
    // last row's, descending), then by external column count and index, cut
    // into slices of whole groups with at most 32 rows that never span two
    // levels. Needs the warp-specialised schedule (its column orders).
    int sready = 0;
    SliceSched sf, sb;
    // Pair-sliced schedule (gic_psolve.cu): group levels (glev, per row: the
    // longest dependency chain of groups ending at the row's group), and per
    // sweep the groups taken two levels at a time; a group at the second
    // level of a pair has the rows it reads at the first substituted by
    // their own solve, so that both levels of a pair only read earlier
    // pairs. Needs groups of at most 3 rows.
    int32_t nglev = 0;
    int32_t *glev = nullptr;
    int32_t *ic_ord = nullptr; // the groups in group-level order (IC(0)'s schedule)
    int pready = 0, pwhy = 0; // pwhy: why not built (bits, see gic_psolve.cu)
    PairSched pf, pb;
    int device = 0;
};

constexpr int QCOL = 64;   // external columns of a group in the warp-specialised solves
constexpr int QLATE = 16;  // at most this many late columns per group

constexpr int GMAX = 8;    // rows per group
constexpr int MAXDIM = 48; // max lower entries of a row handled by IC(0)

}  // namespace gic

namespace gic {
// Node v's aggregation of the edge values e of the lower pattern with its
// diagonal (Section "Model Architecture"): every edge sends its value to both
// endpoints, a self-loop once; S = the sum, M = the mean over the incident
// edges (v's L row, then the strictly upper part of its U row).
__device__ __forceinline__ void gnn_aggregate(int64_t v, const int32_t *Lrowptr, const int32_t *Urowptr,
                                              const int32_t *tperm, const float *e, float &S, float &M)
{
    float s = 0.f;
    const int32_t la = Lrowptr[v], lb = Lrowptr[v + 1];
    for (int32_t p = la; p < lb; ++p) s += e[p];
    const int32_t ua = Urowptr[v], ub = Urowptr[v + 1];
    for (int32_t q = ua + 1; q < ub; ++q) s += e[tperm[q]];
    S = s;
    M = s / (float)((lb - la) + (ub - ua) - 1);
}

// level-sliced schedule of a pattern (gic_ssolve.cu)
int build_ssched(gic_handle *h, Pattern &P);
void free_ssched(SliceSched &S);
// pair-sliced schedule of a pattern (gic_psolve.cu)
int build_psched(gic_handle *h, Pattern &P);
void free_psched(PairSched &S);
// 3x3 node-block SpMV layout of a pattern (gic_bsr.cu)
int build_bsr(gic_handle *h, Pattern &P);
void free_bsr(Pattern &P);
}  // namespace gic

struct gic_pattern {
    gic::Pattern p;
};

struct gic_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    unsigned *dev_err = nullptr;   // device error flags
    void *dev_small = nullptr;     // 64 KiB of library scratch (scalars, Ke)
    void *host_pinned = nullptr;   // 4 KiB pinned readback area
    long long launches = 0;        // kernels this handle has launched
    int tune_solve_warps_per_sm = 0; // cap on resident solve warps per SM (0: none)
    int tune_poll = gic::POLL_ONE_LANE; // polling configuration of the sync-free kernels
    int tune_pipeline = 4;              // 4: automatic, 3: SM-local, 2: warp-specialised, 1: staged, 0: generic
    int tune_qdelta = 6;                // level window of the "late" columns (pattern analysis)
    int tune_gnn_bf16 = 1;              // GNN inference: edge MLP on the tensor cores in BF16 (0: FP32)
    int tune_train_bf16 = 0;            // GNN training forward/backward: BF16 edge MLP (1) or FP32 (0)
    int tune_pair_levels = 0;           // pair-sliced schedule: 0 paired levels, 1 one level per step
};

namespace gic {
size_t pcg_ws_bytes(int64_t n, int64_t nnzL, int64_t sell_nnz, int l_dtype);
size_t gnn_infer_ws_bytes(int64_t n, int64_t nnzL);
int gnn_correct_inplace(gic_handle *h, const gic_pattern *P, const double *valA, const float *theta_host,
                        double *L, void *ws, size_t ws_bytes, int *kept);
int check_handle(gic_handle *h);
// exclusive prefix sum of n int32 counts into out[0..n] (out[n] = total)
int scan_excl_i32(gic_handle *h, const int32_t *in, int64_t n, int32_t *out, long long *total);
int read_and_clear_dev_err(gic_handle *h, unsigned *flags);
}
