// gic_solve.cu -- A7: the PCG loop of Supplementary Algorithm 1 on the GPU.
//
// Kernels:
//   k_lsolve / k_ltsolve  sync-free triangular solves (Supplementary 5,
//       Eq.(11) read as plain forward/back substitution). One warp owns a
//       group of consecutive rows with identical patterns; it gathers the
//       group's off-block columns once, waits (bounded) on each needed
//       solution entry, and finishes the dense diagonal block in registers.
//       "Not yet computed" is a sentinel NaN stored in the solution vector,
//       so the wait and the data are one 8-byte word. Groups are dealt
//       round-robin to a co-resident (cooperative) grid in dependency order,
//       so the first unfinished group can always run.
//   k_spmv                CSR SpMV, one warp per row, with the dot product the
//       PCG step needs fused in (p^T A p) or the initial residual b - A x0.
//   k_update_p / k_update_xr   the vector updates of Algorithm 1, lines
//       13-14 and 17-18, with r^T r fused into the second.
// Every dot product is reduced deterministically: per-block (or per-warp)
// partials in a fixed layout, summed in index order by the last block to
// finish, which also computes alpha / beta and the stop test on the device.
#include <limits.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include <cuda.h>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int SPMV_BLOCK = 256;
constexpr int VEC_BLOCK = 256;

// ------------------------------------------------------------ SpTRSV
// Schedule: the pattern's chunks (runs of consecutive row groups with
// increasing levels; for hex elasticity the x-pencils) are dealt round-robin
// to a co-resident grid in an order where every cross-chunk dependency
// points to an earlier chunk, so the first unfinished chunk can always
// progress. One warp solves a chunk group by group; the last 64 rows it
// produced stay in a shared-memory ring, so the dependency on the previous
// group (the neighbour along x) never leaves the SM. Every index and factor
// value a group needs is loaded before it waits; then one lane polls the
// outstanding dependency with the largest column (the last one produced)
// and the others reload once it lands. "Not yet computed" is a sentinel NaN
// stored in the solution vector, so the flag and the datum are one word.
constexpr int RING = 64;

// value of dependency j: from the ring if this warp produced it recently,
// else one relaxed load from global memory (may still be the sentinel)
__device__ __forceinline__ double dep_first(const double *y, const double *ring, int32_t j, int32_t lo, int32_t hi)
{
    if (j >= lo && j < hi) return ring[j & (RING - 1)];
    return ld_relaxed(y + j);
}

// Per-warp shared staging of a window of WIN consecutive groups: their start
// rows, sizes, row-pointer bases and external column lists. Loading a window
// costs one dependent chain of global loads; inside it every address a group
// needs comes from shared memory, so the loads for the next group really are
// issued ahead (a warp stalls only when it uses a value).
constexpr int WIN = 32;  // groups per window
constexpr int WCOL = 48; // external columns per group kept in shared memory

struct WarpStage {
    int32_t s[WIN], G[WIN], b[WIN], m[WIN];
    int32_t cols[WIN][WCOL];
    double ring[RING];
};

// Everything a group needs before it can wait, in registers. The sweep keeps
// two of these: the group being solved and the next one, whose loads are in
// flight while the current group waits and computes.
template <int GM>
struct GroupRegs {
    int32_t s, G, m, b, j0, j1;
    double d0, d1;                  // dependency values loaded early (may be the sentinel)
    double rr[GM], iv[GM], aux[GM]; // aux: y (backward sweep)
    double v0[GM], v1[GM];
    double lin[GM * (GM - 1) / 2 + 1];
};

// Forward window: group starts, L row-pointer bases, external counts and the
// external columns of each group's first row (shared by the whole group).
__device__ __forceinline__ void stage_window_L(WarpStage &W, int32_t w0, int32_t cnt, const int32_t *grp,
                                               const int32_t *Lrowptr, const int32_t *Lcol, int lane)
{
    if (lane < cnt) {
        const int32_t s = grp[w0 + lane];
        const int32_t G = grp[w0 + lane + 1] - s;
        const int32_t b0 = Lrowptr[s];
        W.s[lane] = s;
        W.G[lane] = G;
        W.b[lane] = b0;
        W.m[lane] = Lrowptr[s + 1] - b0 - 1;
    }
    __syncwarp();
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
        const int32_t m = W.m[k], b0 = W.b[k];
        if (lane < m && lane < WCOL) W.cols[k][lane] = Lcol[b0 + lane];
        if (lane + 32 < m && lane + 32 < WCOL) W.cols[k][lane + 32] = Lcol[b0 + lane + 32];
    }
    __syncwarp();
}

template <typename TL, int GM>
__device__ __forceinline__ void load_group_L(GroupRegs<GM> &q, const WarpStage &W, int k, int cnt,
                                             const int32_t *Lcol, const TL *Lval, const double *invd,
                                             const double *r, const double *y, int lane)
{
    q.G = 0;
    q.j0 = q.j1 = -1;
    if (k >= cnt) return;
    const int32_t s = W.s[k], G = W.G[k], b0 = W.b[k], m = W.m[k];
    q.s = s;
    q.G = G;
    q.m = m;
    q.b = b0;
    q.j0 = (lane < m) ? ((lane < WCOL) ? W.cols[k][lane] : Lcol[b0 + lane]) : -1;
    q.j1 = (lane + 32 < m) ? ((lane + 32 < WCOL) ? W.cols[k][lane + 32] : Lcol[b0 + lane + 32]) : -1;
    // early look at the dependencies (the previous group's rows are not
    // written yet; those are taken from the ring when this group runs)
    q.d0 = (q.j0 >= 0) ? ld_relaxed(y + q.j0) : 0.0;
    q.d1 = (q.j1 >= 0) ? ld_relaxed(y + q.j1) : 0.0;
#pragma unroll
    for (int t = 0; t < GM; ++t) {
        const int32_t base = b0 + t * (m + 1) + (t * (t - 1)) / 2;
        q.rr[t] = (t < G) ? r[s + t] : 0.0;
        q.iv[t] = (t < G) ? invd[s + t] : 0.0;
        q.v0[t] = (t < G && lane < m) ? (double)Lval[base + lane] : 0.0;
        q.v1[t] = (t < G && lane + 32 < m) ? (double)Lval[base + lane + 32] : 0.0;
#pragma unroll
        for (int u = 0; u < t; ++u) q.lin[t * (t - 1) / 2 + u] = (t < G) ? (double)Lval[base + m + u] : 0.0;
    }
}

// Forward: y_i = (r_i - sum_{j<i} L_ij y_j) / L_ii. y must hold the sentinel.
template <typename TL, int GM>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_lsolve(int32_t nchunks, const int32_t *__restrict__ ord,
                                                        const int32_t *__restrict__ chunk_grp,
                                                        const int32_t *__restrict__ grp,
                                                        const int32_t *__restrict__ Lrowptr,
                                                        const int32_t *__restrict__ Lcol, const TL *__restrict__ Lval,
                                                        const double *__restrict__ invd, const double *__restrict__ r,
                                                        double *y, unsigned *err, int poll, const Scalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) unsigned char stage_raw[];
    const int lane = threadIdx.x & 31;
    WarpStage &W = reinterpret_cast<WarpStage *>(stage_raw)[threadIdx.x >> 5];
    double *ring = W.ring;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    GroupRegs<GM> cur, nxt;
    for (int64_t pos = w; pos < nchunks; pos += nw) {
        const int32_t c = ord[pos];
        const int32_t g0 = chunk_grp[c], g1 = chunk_grp[c + 1];
        const int32_t row0 = grp[g0];
        for (int32_t w0 = g0; w0 < g1; w0 += WIN) {
            const int cnt = min(WIN, g1 - w0);
            stage_window_L(W, w0, cnt, grp, Lrowptr, Lcol, lane);
            load_group_L<TL, GM>(cur, W, 0, cnt, Lcol, Lval, invd, r, y, lane);
            for (int k = 0; k < cnt; ++k) {
                load_group_L<TL, GM>(nxt, W, k + 1, cnt, Lcol, Lval, invd, r, y, lane);
                const int32_t s = cur.s, m = cur.m;
                const int G = cur.G;
                const int32_t lo = max(row0, s - RING);
                double y0 = (cur.j0 >= lo && cur.j0 < s) ? ring[cur.j0 & (RING - 1)] : cur.d0;
                double y1 = (cur.j1 >= lo && cur.j1 < s) ? ring[cur.j1 & (RING - 1)] : cur.d1;
                wait_deps<true>(y, cur.j0, cur.j1, y0, y1, err, poll);
                double acc[GM];
#pragma unroll
                for (int t = 0; t < GM; ++t) acc[t] = fma(cur.v1[t], y1, cur.v0[t] * y0);
                if (m > 64) { // rows with more than 64 external columns
                    const int32_t b0 = cur.b;
                    for (int32_t kk = lane + 64; kk < m; kk += 32) {
                        const int32_t j = Lcol[b0 + kk];
                        double yj = (j >= lo && j < s) ? ring[j & (RING - 1)] : ld_relaxed(y + j), dummy = 0.0;
                        wait_deps<true>(y, j, -1, yj, dummy, err, poll);
#pragma unroll
                        for (int t = 0; t < GM; ++t)
                            if (t < G) acc[t] = fma((double)Lval[b0 + t * (m + 1) + (t * (t - 1)) / 2 + kk], yj, acc[t]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int t = 0; t < GM; ++t)
                        if (t < G) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
                if (lane == 0) {
                    double yl[GM];
#pragma unroll
                    for (int t = 0; t < GM; ++t) {
                        if (t < G) {
                            double v = cur.rr[t] - acc[t];
#pragma unroll
                            for (int u = 0; u < t; ++u) v = fma(-cur.lin[t * (t - 1) / 2 + u], yl[u], v);
                            yl[t] = v * cur.iv[t];
                            st_relaxed(y + s + t, yl[t]);
                            ring[(s + t) & (RING - 1)] = yl[t];
                        }
                    }
                }
                __syncwarp();
                cur = nxt;
            }
        }
    }
}

// Backward window (groups w1-cnt+1 .. w1, staged in descending order): U row
// bases, external counts and the external columns of each group's last row.
__device__ __forceinline__ void stage_window_U(WarpStage &W, int32_t w1, int32_t cnt, const int32_t *grp,
                                               const int32_t *Urowptr, const int32_t *Ucol, int lane)
{
    if (lane < cnt) {
        const int32_t g = w1 - lane;
        const int32_t s = grp[g];
        const int32_t G = grp[g + 1] - s;
        const int32_t be = Urowptr[s + G - 1];
        W.s[lane] = s;
        W.G[lane] = G;
        W.b[lane] = be;
        W.m[lane] = Urowptr[s + G] - be - 1;
    }
    __syncwarp();
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
        const int32_t m = W.m[k], be = W.b[k];
        if (lane < m && lane < WCOL) W.cols[k][lane] = Ucol[be + 1 + lane];
        if (lane + 32 < m && lane + 32 < WCOL) W.cols[k][lane + 32] = Ucol[be + 1 + lane + 32];
    }
    __syncwarp();
}

// backward: row s+t of U holds G-t in-group entries (diagonal first), then
// the mu external ones shared by the group (those of row e = s+G-1)
template <typename TL, bool PCG, int GM>
__device__ __forceinline__ void load_group_U(GroupRegs<GM> &q, const WarpStage &W, int k, int cnt,
                                             const int32_t *Ucol, const TL *Uval, const double *invd,
                                             const double *y, const double *r, const double *z, int lane)
{
    q.G = 0;
    q.j0 = q.j1 = -1;
    if (k >= cnt) return;
    const int32_t s = W.s[k], G = W.G[k], be = W.b[k], mu = W.m[k];
    q.s = s;
    q.G = G;
    q.m = mu;
    q.b = be;
    q.j0 = (lane < mu) ? ((lane < WCOL) ? W.cols[k][lane] : Ucol[be + 1 + lane]) : -1;
    q.j1 = (lane + 32 < mu) ? ((lane + 32 < WCOL) ? W.cols[k][lane + 32] : Ucol[be + 1 + lane + 32]) : -1;
    q.d0 = (q.j0 >= 0) ? ld_relaxed(z + q.j0) : 0.0;
    q.d1 = (q.j1 >= 0) ? ld_relaxed(z + q.j1) : 0.0;
    int32_t base[GM];
#pragma unroll
    for (int t = 0; t < GM; ++t) base[t] = be - (G - 1 - t) * (mu + 1) - ((G - 1 - t) * (G - t)) / 2;
#pragma unroll
    for (int t = 0; t < GM; ++t) {
        const int32_t ext = base[t] + (G - t);
        q.aux[t] = (t < G) ? y[s + t] : 0.0;
        q.rr[t] = (PCG && t < G) ? r[s + t] : 0.0;
        q.iv[t] = (t < G) ? invd[s + t] : 0.0;
        q.v0[t] = (t < G && lane < mu) ? (double)Uval[ext + lane] : 0.0;
        q.v1[t] = (t < G && lane + 32 < mu) ? (double)Uval[ext + lane + 32] : 0.0;
    }
#pragma unroll
    for (int u = 1; u < GM; ++u)
#pragma unroll
        for (int t = 0; t < u; ++t)
            q.lin[u * (u - 1) / 2 + t] = (u < G) ? (double)Uval[base[t] + (u - t)] : 0.0;
}

// Backward: z_i = (y_i - sum_{j>i} L_ji z_j) / L_ii on U = L^T. z must hold
// the sentinel. Chunks run in the backward order and each one from its last
// group down. With PCG the kernel also resets y to the sentinel (for the
// next forward solve) and forms r^T z, then beta = r_k^T z_k /
// r_{k-1}^T z_{k-1} (Algorithm 1 line 13) in the last warp to finish.
template <typename TL, bool PCG, int GM>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_ltsolve(int32_t nchunks, const int32_t *__restrict__ ord,
                                                         const int32_t *__restrict__ chunk_grp,
                                                         const int32_t *__restrict__ grp,
                                                         const int32_t *__restrict__ Urowptr,
                                                         const int32_t *__restrict__ Ucol, const TL *__restrict__ Uval,
                                                         const double *__restrict__ invd, double *y, double *z,
                                                         const double *__restrict__ r, double *partials,
                                                         unsigned *err, int poll, Scalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) unsigned char stage_raw[];
    const int lane = threadIdx.x & 31;
    WarpStage &W = reinterpret_cast<WarpStage *>(stage_raw)[threadIdx.x >> 5];
    double *ring = W.ring;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dot = 0.0;
    GroupRegs<GM> cur, nxt;
    for (int64_t pos = w; pos < nchunks; pos += nw) {
        const int32_t c = ord[pos];
        const int32_t g0 = chunk_grp[c], g1 = chunk_grp[c + 1];
        const int32_t rowEnd = grp[g1];
        for (int32_t w1 = g1 - 1; w1 >= g0; w1 -= WIN) {
            const int cnt = min(WIN, w1 - g0 + 1);
            stage_window_U(W, w1, cnt, grp, Urowptr, Ucol, lane);
            load_group_U<TL, PCG, GM>(cur, W, 0, cnt, Ucol, Uval, invd, y, r, z, lane);
            for (int k = 0; k < cnt; ++k) {
                load_group_U<TL, PCG, GM>(nxt, W, k + 1, cnt, Ucol, Uval, invd, y, r, z, lane);
                const int32_t s = cur.s, mu = cur.m;
                const int G = cur.G;
                const int32_t e = s + G - 1;
                const int32_t hi = min(rowEnd, e + 1 + RING);
                double z0 = (cur.j0 > e && cur.j0 < hi) ? ring[cur.j0 & (RING - 1)] : cur.d0;
                double z1 = (cur.j1 > e && cur.j1 < hi) ? ring[cur.j1 & (RING - 1)] : cur.d1;
                wait_deps<false>(z, cur.j0, cur.j1, z0, z1, err, poll);
                double acc[GM];
#pragma unroll
                for (int t = 0; t < GM; ++t) acc[t] = fma(cur.v1[t], z1, cur.v0[t] * z0);
                if (mu > 64) {
                    const int32_t be = cur.b;
                    for (int32_t kk = lane + 64; kk < mu; kk += 32) {
                        const int32_t j = Ucol[be + 1 + kk];
                        double zj = (j > e && j < hi) ? ring[j & (RING - 1)] : ld_relaxed(z + j), dummy = 0.0;
                        wait_deps<false>(z, j, -1, zj, dummy, err, poll);
#pragma unroll
                        for (int t = 0; t < GM; ++t)
                            if (t < G) acc[t] = fma((double)Uval[Urowptr[s + t] + (G - t) + kk], zj, acc[t]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int t = 0; t < GM; ++t)
                        if (t < G) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
                if (lane == 0) {
                    double zl[GM];
#pragma unroll
                    for (int t = GM - 1; t >= 0; --t) {
                        if (t < G) {
                            double v = cur.aux[t] - acc[t];
#pragma unroll
                            for (int u = t + 1; u < GM; ++u)
                                if (u < G) v = fma(-cur.lin[u * (u - 1) / 2 + t], zl[u], v);
                            zl[t] = v * cur.iv[t];
                            st_relaxed(z + s + t, zl[t]);
                            ring[(s + t) & (RING - 1)] = zl[t];
                            if (PCG) {
                                y[s + t] = sentinel_d();
                                dot = fma(cur.rr[t], zl[t], dot);
                            }
                        }
                    }
                }
                __syncwarp();
                cur = nxt;
            }
        }
    }
    if (PCG) {
        // per-warp partial, then the last warp of the grid reduces
        if (lane == 0) partials[w] = dot;
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence();
            last = (atomicAdd(&sc->counter, 1u) == (unsigned)nw - 1u);
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            double rz = warp_sum_partials(partials, (int)nw);
            if (lane == 0) {
                sc->counter = 0;
                if (!(rz > 0.0) || !isfinite(rz)) {
                    sc->status = GIC_ERR_BREAKDOWN;
                    sc->done = 1;
                } else {
                    sc->beta = (sc->iter == 0) ? 0.0 : rz / sc->rz;
                    sc->rz = rz;
                }
            }
        }
    }
}

// ------------------------------------------------------------ pipelined SpTRSV
// Same schedule as k_lsolve / k_ltsolve, for patterns whose row groups have
// at most 3 rows and at most WCOL external columns, in arithmetic type T
// (double: the FP64 solve; float: the FP32 preconditioner apply, factor,
// vectors and sums all in FP32). Per chunk a warp:
//  * stages the metadata of the chunk (segments of CHMAX groups) once;
//  * keeps NST groups in flight: columns, factor values, right-hand side and
//    reciprocal diagonal copied global -> shared by cp.async NST-1 groups
//    before the group runs;
//  * splits each group's sum: the part over dependencies not produced by
//    the previous group of the chunk is reduced one group early, as soon as
//    those values are there (read two groups early, polled only if still
//    the sentinel); when the previous group finishes, every lane adds its
//    at most 3x3 contribution from registers and solves the dense in-group
//    block. The in-chunk step (the x-neighbour for hex elasticity) then
//    costs a few dependent FMAs instead of a warp reduction.
// Arithmetic on this part: a dependent FP64 FMA is ~65 cycles and FP64
// issue is ~1.6 lanes/clock/SM, so the reduction also keeps FP64
// instructions few (three rows reduced in 6 adds, not 15).
constexpr int CHMAX = 160;
constexpr int NST = 4;

template <typename T, int GM>
struct PStage {
    double rd[GM];                 // r in FP64 (PCG dot of the backward sweep)
    T v[GM][WCOL];                 // external values of each row of the group
    T lin[GM * (GM - 1) / 2 + 1];  // in-group entries
    T rr[GM], iv[GM], aux[GM];     // right-hand side (forward), 1/L_ii, y (backward)
    int32_t cols[WCOL];
};

template <typename T, int GM>
struct PWarp {
    int32_t s[CHMAX], G[CHMAX], b[CHMAX], m[CHMAX];
    PStage<T, GM> st[NST];
};

// (t,u) of the q-th entry of a strictly lower triangle stored row by row
__device__ __forceinline__ void tri_index(int q, int &t, int &u)
{
    t = 1;
    while (q >= t) { q -= t; ++t; }
    u = q;
}

template <typename T, int GM>
__device__ __forceinline__ void fill_stage_L(PStage<T, GM> &st, const PWarp<T, GM> &W, int k, const int32_t *Lcol,
                                             const T *Lval, const T *r, const T *invd, int lane)
{
    const int32_t s = W.s[k], G = W.G[k], b0 = W.b[k], m = W.m[k];
    if (lane < m) cp_async_4(&st.cols[lane], Lcol + b0 + lane);
    if (lane + 32 < m) cp_async_4(&st.cols[lane + 32], Lcol + b0 + lane + 32);
#pragma unroll
    for (int t = 0; t < GM; ++t) {
        if (t < G) {
            const int32_t base = b0 + t * (m + 1) + (t * (t - 1)) / 2;
            if (lane < m) cp_async_t(&st.v[t][lane], Lval + base + lane);
            if (lane + 32 < m) cp_async_t(&st.v[t][lane + 32], Lval + base + lane + 32);
        }
    }
    if (lane < G * (G - 1) / 2) {
        int t, u;
        tri_index(lane, t, u);
        cp_async_t(&st.lin[lane], Lval + b0 + t * (m + 1) + (t * (t - 1)) / 2 + m + u);
    }
    if (lane < G) {
        cp_async_t(&st.rr[lane], r + s + lane);
        cp_async_t(&st.iv[lane], invd + s + lane);
    }
}

// early read of the dependencies of stage-resident group k that lie below
// `ps` (everything not produced by the group before it)
template <typename T, int GM>
__device__ __forceinline__ void early_L(const PStage<T, GM> &st, int32_t m, int32_t ps, const T *y, int lane, T &d0, T &d1)
{
    const int32_t j0 = (lane < m) ? st.cols[lane] : -1, j1 = (lane + 32 < m) ? st.cols[lane + 32] : -1;
    d0 = (j0 >= 0 && j0 < ps) ? ld_relaxed(y + j0) : (T)0;
    d1 = (j1 >= 0 && j1 < ps) ? ld_relaxed(y + j1) : (T)0;
}

// the part of group k's sums over dependencies below ps
template <typename T, int GM>
__device__ __forceinline__ void ext_sum_L(T (&S)[GM], const PStage<T, GM> &st, int32_t m, int G, int32_t ps,
                                          const T *y, T d0, T d1, unsigned *err, int poll, int lane)
{
    int32_t j0 = (lane < m) ? st.cols[lane] : -1, j1 = (lane + 32 < m) ? st.cols[lane + 32] : -1;
    if (j0 >= ps) j0 = -1;
    if (j1 >= ps) j1 = -1;
    wait_pair<true, T>(y, j0, j1, d0, d1, err, poll);
    if (j0 < 0) d0 = (T)0;
    if (j1 < 0) d1 = (T)0;
#pragma unroll
    for (int t = 0; t < GM; ++t) {
        const T a0 = (t < G && j0 >= 0) ? st.v[t][lane] : (T)0;
        const T a1 = (t < G && j1 >= 0) ? st.v[t][lane + 32] : (T)0;
        S[t] = fma(a1, d1, a0 * d0);
    }
    warp_sum_n<T, GM>(S, lane);
}

// Forward: y_i = (r_i - sum_{j<i} L_ij y_j) / L_ii. y must hold the sentinel.
template <typename T, int GM>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_lsolve_p(int32_t nchunks, const int32_t *__restrict__ ord,
                                                          const int32_t *__restrict__ chunk_grp,
                                                          const int32_t *__restrict__ grp,
                                                          const int32_t *__restrict__ Lrowptr,
                                                          const int32_t *__restrict__ Lcol,
                                                          const T *__restrict__ Lval, const T *__restrict__ invd,
                                                          const T *__restrict__ r, T *y, unsigned *err, int poll,
                                                          const Scalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) unsigned char pw_raw[];
    const int lane = threadIdx.x & 31;
    PWarp<T, GM> &W = reinterpret_cast<PWarp<T, GM> *>(pw_raw)[threadIdx.x >> 5];
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pos = w; pos < nchunks; pos += nw) {
        const int32_t c = ord[pos];
        const int32_t g0 = chunk_grp[c], g1 = chunk_grp[c + 1];
        T yprev[GM];
#pragma unroll
        for (int t = 0; t < GM; ++t) yprev[t] = (T)0;
        int32_t prev_s = INT_MAX; // rows of the previous group: [prev_s, prev_s + G)
        for (int32_t seg = g0; seg < g1; seg += CHMAX) {
            const int cnt = min(CHMAX, g1 - seg);
            for (int k = lane; k < cnt; k += 32) {
                const int32_t s = grp[seg + k];
                const int32_t b0 = Lrowptr[s];
                W.s[k] = s;
                W.G[k] = grp[seg + k + 1] - s;
                W.b[k] = b0;
                W.m[k] = Lrowptr[s + 1] - b0 - 1;
            }
            __syncwarp();
#pragma unroll
            for (int d = 0; d < NST; ++d) {
                if (d < cnt) fill_stage_L<T, GM>(W.st[d], W, d, Lcol, Lval, r, invd, lane);
                cp_async_commit();
            }
            cp_async_wait<NST - 2>();
            __syncwarp();
            T Sx[GM], dB0 = 0, dB1 = 0;
            {
                T d0, d1;
                early_L<T, GM>(W.st[0], W.m[0], prev_s, y, lane, d0, d1);
                ext_sum_L<T, GM>(Sx, W.st[0], W.m[0], W.G[0], prev_s, y, d0, d1, err, poll, lane);
                if (cnt > 1) early_L<T, GM>(W.st[1], W.m[1], W.s[0], y, lane, dB0, dB1);
            }
            for (int k = 0; k < cnt; ++k) {
                const PStage<T, GM> &st = W.st[k % NST];
                const int32_t s = W.s[k], m = W.m[k];
                const int G = W.G[k];
                // contribution of the previous group (its rows are the
                // largest external columns) and the dense in-group solve
                T tot[GM];
#pragma unroll
                for (int t = 0; t < GM; ++t) tot[t] = Sx[t];
                for (int e = m - 1; e >= 0 && e >= m - GM; --e) {
                    const int32_t j = st.cols[e];
                    if (j < prev_s) break;
                    const T yp = pick3<T>(j - prev_s, yprev[0], yprev[GM > 1 ? 1 : 0], yprev[GM > 2 ? 2 : 0]);
#pragma unroll
                    for (int t = 0; t < GM; ++t)
                        if (t < G) tot[t] = fma(st.v[t][e], yp, tot[t]);
                }
                T yl[GM];
#pragma unroll
                for (int t = 0; t < GM; ++t) {
                    T v = st.rr[t] - tot[t];
#pragma unroll
                    for (int u = 0; u < t; ++u) v = fma(-st.lin[t * (t - 1) / 2 + u], yl[u], v);
                    yl[t] = (t < G) ? v * st.iv[t] : (T)0;
                }
                if (lane < G) st_relaxed(y + s + lane, pick3<T>(lane, yl[0], yl[GM > 1 ? 1 : 0], yl[GM > 2 ? 2 : 0]));
#pragma unroll
                for (int t = 0; t < GM; ++t) yprev[t] = yl[t];
                prev_s = s;
                // the part of the next group's sums not involving this group
                if (k + 1 < cnt) {
                    const int kn = k + 1;
                    ext_sum_L<T, GM>(Sx, W.st[kn % NST], W.m[kn], W.G[kn], s, y, dB0, dB1, err, poll, lane);
                }
                __syncwarp();
                if (k + NST < cnt) fill_stage_L<T, GM>(W.st[k % NST], W, k + NST, Lcol, Lval, r, invd, lane);
                cp_async_commit();
                cp_async_wait<NST - 2>();
                __syncwarp();
                if (k + 2 < cnt) early_L<T, GM>(W.st[(k + 2) % NST], W.m[k + 2], W.s[k + 1], y, lane, dB0, dB1);
            }
            cp_async_wait<0>();
            __syncwarp();
        }
    }
}

template <typename T, bool PCG, int GM>
__device__ __forceinline__ void fill_stage_U(PStage<T, GM> &st, const PWarp<T, GM> &W, int k, const int32_t *Ucol,
                                             const T *Uval, const double *rd, const T *invd, const T *y, int lane)
{
    const int32_t s = W.s[k], G = W.G[k], be = W.b[k], mu = W.m[k];
    if (lane < mu) cp_async_4(&st.cols[lane], Ucol + be + 1 + lane);
    if (lane + 32 < mu) cp_async_4(&st.cols[lane + 32], Ucol + be + 1 + lane + 32);
#pragma unroll
    for (int t = 0; t < GM; ++t) {
        if (t < G) {
            const int32_t base = be - (G - 1 - t) * (mu + 1) - ((G - 1 - t) * (G - t)) / 2;
            const int32_t ext = base + (G - t);
            if (lane < mu) cp_async_t(&st.v[t][lane], Uval + ext + lane);
            if (lane + 32 < mu) cp_async_t(&st.v[t][lane + 32], Uval + ext + lane + 32);
        }
    }
    if (lane < G * (G - 1) / 2) { // lin[u(u-1)/2 + t] = U[s+t][s+u], t < u
        int uu, t;
        tri_index(lane, uu, t);
        const int32_t base = be - (G - 1 - t) * (mu + 1) - ((G - 1 - t) * (G - t)) / 2;
        cp_async_t(&st.lin[lane], Uval + base + (uu - t));
    }
    if (lane < G) {
        if (PCG) cp_async_8(&st.rd[lane], rd + s + lane);
        cp_async_t(&st.iv[lane], invd + s + lane);
        cp_async_t(&st.aux[lane], y + s + lane);
    }
}

// dependencies of group k above `pe` (everything not produced by the group
// processed before it, which sits just above)
template <typename T, int GM>
__device__ __forceinline__ void early_U(const PStage<T, GM> &st, int32_t mu, int32_t pe, const T *z, int lane, T &d0, T &d1)
{
    const int32_t j0 = (lane < mu) ? st.cols[lane] : -1, j1 = (lane + 32 < mu) ? st.cols[lane + 32] : -1;
    d0 = (j0 >= 0 && j0 > pe) ? ld_relaxed(z + j0) : (T)0;
    d1 = (j1 >= 0 && j1 > pe) ? ld_relaxed(z + j1) : (T)0;
}

template <typename T, int GM>
__device__ __forceinline__ void ext_sum_U(T (&S)[GM], const PStage<T, GM> &st, int32_t mu, int G, int32_t pe,
                                          const T *z, T d0, T d1, unsigned *err, int poll, int lane)
{
    int32_t j0 = (lane < mu) ? st.cols[lane] : -1, j1 = (lane + 32 < mu) ? st.cols[lane + 32] : -1;
    if (j0 >= 0 && j0 <= pe) j0 = -1;
    if (j1 >= 0 && j1 <= pe) j1 = -1;
    wait_pair<false, T>(z, j0, j1, d0, d1, err, poll);
    if (j0 < 0) d0 = (T)0;
    if (j1 < 0) d1 = (T)0;
#pragma unroll
    for (int t = 0; t < GM; ++t) {
        const T a0 = (t < G && j0 >= 0) ? st.v[t][lane] : (T)0;
        const T a1 = (t < G && j1 >= 0) ? st.v[t][lane + 32] : (T)0;
        S[t] = fma(a1, d1, a0 * d0);
    }
    warp_sum_n<T, GM>(S, lane);
}

// Backward: z_i = (y_i - sum_{j>i} L_ji z_j) / L_ii on U = L^T. z must hold
// the sentinel. Chunks run in the backward order and each one from its last
// group down. With PCG the kernel also resets y to the sentinel (for the
// next forward solve) and forms r^T z in FP64, then beta = r_k^T z_k /
// r_{k-1}^T z_{k-1} (Algorithm 1 line 13) in the last warp to finish.
template <typename T, bool PCG, int GM>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_ltsolve_p(int32_t nchunks, const int32_t *__restrict__ ord,
                                                           const int32_t *__restrict__ chunk_grp,
                                                           const int32_t *__restrict__ grp,
                                                           const int32_t *__restrict__ Urowptr,
                                                           const int32_t *__restrict__ Ucol,
                                                           const T *__restrict__ Uval, const T *__restrict__ invd,
                                                           T *y, T *z, const double *__restrict__ rd,
                                                           double *partials, unsigned *err, int poll, Scalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) unsigned char pw_raw[];
    const int lane = threadIdx.x & 31;
    PWarp<T, GM> &W = reinterpret_cast<PWarp<T, GM> *>(pw_raw)[threadIdx.x >> 5];
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dot = 0.0;
    for (int64_t pos = w; pos < nchunks; pos += nw) {
        const int32_t c = ord[pos];
        const int32_t g0 = chunk_grp[c], g1 = chunk_grp[c + 1];
        T zprev[GM];
#pragma unroll
        for (int t = 0; t < GM; ++t) zprev[t] = (T)0;
        int32_t prev_s = INT_MIN, prev_e = INT_MIN; // rows of the group processed before
        for (int32_t segEnd = g1 - 1; segEnd >= g0; segEnd -= CHMAX) {
            const int cnt = min(CHMAX, segEnd - g0 + 1);
            for (int k = lane; k < cnt; k += 32) { // k-th group of the segment, from its end
                const int32_t g = segEnd - k;
                const int32_t s = grp[g];
                const int32_t G = grp[g + 1] - s;
                const int32_t be = Urowptr[s + G - 1];
                W.s[k] = s;
                W.G[k] = G;
                W.b[k] = be;
                W.m[k] = Urowptr[s + G] - be - 1;
            }
            __syncwarp();
#pragma unroll
            for (int d = 0; d < NST; ++d) {
                if (d < cnt) fill_stage_U<T, PCG, GM>(W.st[d], W, d, Ucol, Uval, rd, invd, y, lane);
                cp_async_commit();
            }
            cp_async_wait<NST - 2>();
            __syncwarp();
            T Sx[GM], dB0 = 0, dB1 = 0;
            {
                T d0, d1;
                early_U<T, GM>(W.st[0], W.m[0], prev_e, z, lane, d0, d1);
                ext_sum_U<T, GM>(Sx, W.st[0], W.m[0], W.G[0], prev_e, z, d0, d1, err, poll, lane);
                if (cnt > 1) early_U<T, GM>(W.st[1], W.m[1], W.s[0] + W.G[0] - 1, z, lane, dB0, dB1);
            }
            for (int k = 0; k < cnt; ++k) {
                const PStage<T, GM> &st = W.st[k % NST];
                const int32_t s = W.s[k], mu = W.m[k];
                const int G = W.G[k];
                const int32_t e = s + G - 1;
                T tot[GM];
#pragma unroll
                for (int t = 0; t < GM; ++t) tot[t] = Sx[t];
                // the previous group's rows are the smallest external columns
                for (int q = 0; q < mu && q < GM; ++q) {
                    const int32_t j = st.cols[q];
                    if (j > prev_e) break;
                    const T zp = pick3<T>(j - prev_s, zprev[0], zprev[GM > 1 ? 1 : 0], zprev[GM > 2 ? 2 : 0]);
#pragma unroll
                    for (int t = 0; t < GM; ++t)
                        if (t < G) tot[t] = fma(st.v[t][q], zp, tot[t]);
                }
                T zl[GM];
#pragma unroll
                for (int t = GM - 1; t >= 0; --t) {
                    T v = st.aux[t] - tot[t];
#pragma unroll
                    for (int u = t + 1; u < GM; ++u)
                        if (u < G) v = fma(-st.lin[u * (u - 1) / 2 + t], zl[u], v);
                    zl[t] = (t < G) ? v * st.iv[t] : (T)0;
                }
                if (lane < G) {
                    const T zv = pick3<T>(lane, zl[0], zl[GM > 1 ? 1 : 0], zl[GM > 2 ? 2 : 0]);
                    st_relaxed(z + s + lane, zv);
                    if (PCG) {
                        y[s + lane] = sentinel_of<T>();
                        dot = fma(st.rd[lane], (double)zv, dot);
                    }
                }
#pragma unroll
                for (int t = 0; t < GM; ++t) zprev[t] = zl[t];
                prev_s = s;
                prev_e = e;
                if (k + 1 < cnt) {
                    const int kn = k + 1;
                    ext_sum_U<T, GM>(Sx, W.st[kn % NST], W.m[kn], W.G[kn], e, z, dB0, dB1, err, poll, lane);
                }
                __syncwarp();
                if (k + NST < cnt) fill_stage_U<T, PCG, GM>(W.st[k % NST], W, k + NST, Ucol, Uval, rd, invd, y, lane);
                cp_async_commit();
                cp_async_wait<NST - 2>();
                __syncwarp();
                if (k + 2 < cnt)
                    early_U<T, GM>(W.st[(k + 2) % NST], W.m[k + 2], W.s[k + 1] + W.G[k + 1] - 1, z, lane, dB0, dB1);
            }
            cp_async_wait<0>();
            __syncwarp();
        }
    }
    if (PCG) {
        dot = warp_sum(dot); // lanes < G held the products
        if (lane == 0) partials[w] = dot;
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence();
            last = (atomicAdd(&sc->counter, 1u) == (unsigned)nw - 1u);
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            double rz = warp_sum_partials(partials, (int)nw);
            if (lane == 0) {
                sc->counter = 0;
                if (!(rz > 0.0) || !isfinite(rz)) {
                    sc->status = GIC_ERR_BREAKDOWN;
                    sc->done = 1;
                } else {
                    sc->beta = (sc->iter == 0) ? 0.0 : rz / sc->rz;
                    sc->rz = rz;
                }
            }
        }
    }
}

// ------------------------------------------------------------ SpMV
// MODE 0: y = A x (optional x^T y into *out_dot)
// MODE 1: y = A p, pw = p^T y, alpha = rz / pw          (Algorithm 1 lines 15-16)
// MODE 2: r = b - A x, rr = r^T r, bb = b^T b, stop test (Algorithm 1 line 1)
template <int MODE>
__global__ void __launch_bounds__(SPMV_BLOCK) k_spmv(int64_t n, const int32_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col, const double *__restrict__ val,
                                                     const double *__restrict__ x, double *__restrict__ y,
                                                     const double *__restrict__ b, double *partials, double *out_dot,
                                                     Scalars *sc)
{
    if (MODE != 0 && sc->done) return;
    __shared__ double sh[SPMV_BLOCK / 32];
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double d1 = 0.0, d2 = 0.0;
    for (int64_t i = w; i < n; i += nw) {
        const int32_t a = rowptr[i], e = rowptr[i + 1];
        // all loads of up to 128 entries in flight before the first use
        int32_t c[4];
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int32_t p = a + lane + 32 * k;
            c[k] = (p < e) ? __ldg(col + p) : -1;
            v[k] = (p < e) ? __ldg(val + p) : 0.0;
        }
        double xv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = (c[k] >= 0) ? __ldg(x + c[k]) : 0.0;
        double s = fma(v[3], xv[3], fma(v[2], xv[2], fma(v[1], xv[1], v[0] * xv[0])));
        for (int32_t p = a + lane + 128; p < e; p += 32) s = fma(val[p], __ldg(x + col[p]), s);
        s = warp_sum(s);
        if (lane == 0) {
            if (MODE == 2) {
                double bi = b[i];
                double ri = bi - s;
                y[i] = ri;
                d1 = fma(ri, ri, d1);
                d2 = fma(bi, bi, d2);
            } else {
                y[i] = s;
                d1 = fma(x[i], s, d1);
            }
        }
    }
    if (MODE == 0 && !out_dot) return;
    double s1 = block_sum(d1, sh);
    double s2 = (MODE == 2) ? block_sum(d2, sh) : 0.0;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s1;
        if (MODE == 2) partials[gridDim.x + blockIdx.x] = s2;
    }
    __shared__ bool is_last;
    if (threadIdx.x == 0) is_last = last_block(&sc->counter, gridDim.x);
    __syncthreads();
    if (!is_last || threadIdx.x >= 32) return;
    __threadfence();
    double t1 = warp_sum_partials(partials, gridDim.x);
    double t2 = (MODE == 2) ? warp_sum_partials(partials + gridDim.x, gridDim.x) : 0.0;
    if (lane != 0) return;
    sc->counter = 0;
    if (MODE == 0) {
        *out_dot = t1;
    } else if (MODE == 1) {
        sc->pw = t1;
        if (!(t1 > 0.0) || !isfinite(t1)) {
            sc->status = GIC_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->alpha = sc->rz / t1;
        }
    } else {
        sc->rr = t1;
        sc->bb = t2;
        if (t2 == 0.0 || sqrt(t1) <= sc->tol * sqrt(t2)) {
            sc->done = 1;
            sc->status = GIC_OK;
        }
        if (!isfinite(t1)) {
            sc->done = 1;
            sc->status = GIC_ERR_BREAKDOWN;
        }
    }
}

// SELL-32 SpMV: one warp per slice of 32 rows, one row per lane, column-
// major entries inside the slice, so every load is a coalesced 256-byte
// (values) or 128-byte (columns) line and every FP64 instruction does up to
// 32 useful multiply-adds with no cross-lane reduction (FP64 issue slots are
// the scarce resource next to HBM on this part). Modes as k_spmv.
__global__ void k_sell_vals(int64_t n, int64_t nslices, const int32_t *rowptr, const double *val, const int64_t *sptr,
                            const int32_t *w, double *sval)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslices * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i >> 5;
        const int t = (int)(i & 31);
        const int32_t a = (i < n) ? rowptr[i] : 0, len = (i < n) ? rowptr[i + 1] - a : 0;
        for (int32_t k = 0; k < w[sl]; ++k) sval[sptr[sl] + (int64_t)k * 32 + t] = (k < len) ? val[a + k] : 0.0;
    }
}

template <int MODE>
__global__ void __launch_bounds__(SPMV_BLOCK) k_spmv_sell(int64_t n, int64_t nslices, const int64_t *__restrict__ sptr,
                                                          const int32_t *__restrict__ sw,
                                                          const int32_t *__restrict__ scol,
                                                          const double *__restrict__ sval,
                                                          const double *__restrict__ x, double *__restrict__ y,
                                                          const double *__restrict__ b, double *partials,
                                                          Scalars *sc)
{
    if (sc->done) return;
    __shared__ double sh[SPMV_BLOCK / 32];
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double d1 = 0.0, d2 = 0.0;
    for (int64_t sl = w; sl < nslices; sl += nw) {
        const int64_t i = sl * 32 + lane;
        const int32_t width = (i < n) ? sw[sl] : 0; // lanes past the last row load nothing
        const int64_t o = sptr[sl] + lane;
        double s0 = 0.0, s1 = 0.0;
        int32_t k = 0;
        for (; k + 4 <= width; k += 4) {
            int32_t c[4];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = __ldg(scol + o + 32 * (int64_t)(k + u));
                v[u] = __ldg(sval + o + 32 * (int64_t)(k + u));
            }
            double xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = __ldg(x + c[u]);
            s0 = fma(v[0], xv[0], s0);
            s1 = fma(v[1], xv[1], s1);
            s0 = fma(v[2], xv[2], s0);
            s1 = fma(v[3], xv[3], s1);
        }
        for (; k < width; ++k) s0 = fma(__ldg(sval + o + 32 * (int64_t)k), __ldg(x + __ldg(scol + o + 32 * (int64_t)k)), s0);
        const double s = s0 + s1;
        if (i < n) {
            if (MODE == 2) {
                const double bi = b[i];
                const double ri = bi - s;
                y[i] = ri;
                d1 = fma(ri, ri, d1);
                d2 = fma(bi, bi, d2);
            } else {
                y[i] = s;
                d1 = fma(x[i], s, d1);
            }
        }
    }
    double s1 = block_sum(d1, sh);
    double s2 = (MODE == 2) ? block_sum(d2, sh) : 0.0;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s1;
        if (MODE == 2) partials[gridDim.x + blockIdx.x] = s2;
    }
    __shared__ bool is_last;
    if (threadIdx.x == 0) is_last = last_block(&sc->counter, gridDim.x);
    __syncthreads();
    if (!is_last || threadIdx.x >= 32) return;
    __threadfence();
    double t1 = warp_sum_partials(partials, gridDim.x);
    double t2 = (MODE == 2) ? warp_sum_partials(partials + gridDim.x, gridDim.x) : 0.0;
    if (lane != 0) return;
    sc->counter = 0;
    if (MODE == 1) {
        sc->pw = t1;
        if (!(t1 > 0.0) || !isfinite(t1)) {
            sc->status = GIC_ERR_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->alpha = sc->rz / t1;
        }
    } else {
        sc->rr = t1;
        sc->bb = t2;
        if (t2 == 0.0 || sqrt(t1) <= sc->tol * sqrt(t2)) {
            sc->done = 1;
            sc->status = GIC_OK;
        }
        if (!isfinite(t1)) {
            sc->done = 1;
            sc->status = GIC_ERR_BREAKDOWN;
        }
    }
}

// p = z + beta p (p = z on the first step); z back to the sentinel (ZT:
// float for the FP32 preconditioner vectors), and y too when yr is given
// (the pair-sliced backward sweep reads y without resetting it). With IDENT
// the preconditioner is the identity and z is r itself.
template <bool IDENT, typename ZT>
__global__ void __launch_bounds__(VEC_BLOCK) k_update_p(int64_t n, ZT *z, double *p, const double *r, ZT *yr,
                                                        Scalars *sc)
{
    if (sc->done) return;
    const int first = (sc->iter == 0);
    const double beta = sc->beta;
    // two independent elements per iteration (twice the loads in flight)
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + st < n; i += 2 * st) {
        const int64_t j = i + st;
        if (IDENT) {
            const double zi = r[i], zj = r[j], pi = first ? 0.0 : p[i], pj = first ? 0.0 : p[j];
            p[i] = first ? zi : fma(beta, pi, zi);
            p[j] = first ? zj : fma(beta, pj, zj);
        } else {
            const double zi = (double)z[i], zj = (double)z[j], pi = first ? 0.0 : p[i], pj = first ? 0.0 : p[j];
            p[i] = first ? zi : fma(beta, pi, zi);
            p[j] = first ? zj : fma(beta, pj, zj);
            z[i] = sentinel_of<ZT>();
            z[j] = sentinel_of<ZT>();
            if (yr) {
                yr[i] = sentinel_of<ZT>();
                yr[j] = sentinel_of<ZT>();
            }
        }
    }
    if (i < n) {
        if (IDENT) {
            const double zi = r[i];
            p[i] = first ? zi : fma(beta, p[i], zi);
        } else {
            const double zi = (double)z[i];
            p[i] = first ? zi : fma(beta, p[i], zi);
            z[i] = sentinel_of<ZT>();
            if (yr) yr[i] = sentinel_of<ZT>();
        }
    }
}

// r^T r for the identity preconditioner (r^T z with z = r): computes beta.
__global__ void __launch_bounds__(VEC_BLOCK) k_ident_rz(int64_t n, const double *r, double *partials, Scalars *sc)
{
    if (sc->done) return;
    __shared__ double sh[VEC_BLOCK / 32];
    double d = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d = fma(r[i], r[i], d);
    double s = block_sum(d, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    __shared__ bool is_last;
    if (threadIdx.x == 0) is_last = last_block(&sc->counter, gridDim.x);
    __syncthreads();
    if (!is_last || threadIdx.x >= 32) return;
    __threadfence();
    double rz = warp_sum_partials(partials, gridDim.x);
    if ((threadIdx.x & 31) != 0) return;
    sc->counter = 0;
    if (!(rz > 0.0) || !isfinite(rz)) {
        sc->status = GIC_ERR_BREAKDOWN;
        sc->done = 1;
    } else {
        sc->beta = (sc->iter == 0) ? 0.0 : rz / sc->rz;
        sc->rz = rz;
    }
}

// x += alpha p, r -= alpha w, rr = r^T r; iteration count and stop test.
// r32 (nullable) receives float(r) for the FP32 preconditioner.
__global__ void __launch_bounds__(VEC_BLOCK) k_update_xr(int64_t n, double *x, double *r, const double *p,
                                                         const double *w, float *r32, double *partials, Scalars *sc)
{
    if (sc->done) return;
    __shared__ double sh[VEC_BLOCK / 32];
    const double alpha = sc->alpha;
    double d = 0.0;
    // two independent elements per iteration (twice the loads in flight)
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + st < n; i += 2 * st) {
        const int64_t j = i + st;
        const double pi = p[i], pj = p[j], wi = w[i], wj = w[j], xi = x[i], xj = x[j], r0 = r[i], r1 = r[j];
        x[i] = fma(alpha, pi, xi);
        x[j] = fma(alpha, pj, xj);
        const double ri = fma(-alpha, wi, r0), rj = fma(-alpha, wj, r1);
        r[i] = ri;
        r[j] = rj;
        if (r32) {
            r32[i] = (float)ri;
            r32[j] = (float)rj;
        }
        d = fma(ri, ri, d);
        d = fma(rj, rj, d);
    }
    if (i < n) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, w[i], r[i]);
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        d = fma(ri, ri, d);
    }
    double s = block_sum(d, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    __shared__ bool is_last;
    if (threadIdx.x == 0) is_last = last_block(&sc->counter, gridDim.x);
    __syncthreads();
    if (!is_last || threadIdx.x >= 32) return;
    __threadfence();
    double rr = warp_sum_partials(partials, gridDim.x);
    if ((threadIdx.x & 31) != 0) return;
    sc->counter = 0;
    sc->rr = rr;
    sc->iter += 1;
    if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) {
        sc->done = 1;
        sc->status = GIC_OK;
    } else if (!isfinite(rr)) {
        sc->done = 1;
        sc->status = GIC_ERR_BREAKDOWN;
    } else if (sc->iter >= sc->maxit) {
        sc->done = 1;
        sc->status = GIC_ERR_NO_CONVERGENCE;
    }
}

__global__ void k_init_scalars(Scalars *sc, double tol, int maxit)
{
    Scalars s = {};
    s.tol = tol;
    s.maxit = maxit;
    s.status = GIC_OK;
    *sc = s;
}

__global__ void k_convert_f64_f32(int64_t cnt, const double *src, float *dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_convert_f32_f64(int64_t cnt, const float *src, double *dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_fill_sentinel_t(int64_t n, T *a, T *b)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a[i] = sentinel_of<T>();
        if (b) b[i] = sentinel_of<T>();
    }
}

// U values (transpose of L in U's CSR order) and reciprocal diagonal (TI).
template <typename TL, typename TI>
__global__ void k_factor_setup(int64_t n, int64_t nnzL, const int32_t *tperm, const int32_t *Lrowptr, const TL *Lval,
                               TL *Uval, TI *invd)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnzL; q += stride) Uval[q] = Lval[tperm[q]];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        invd[i] = (TI)(1.0 / (double)Lval[Lrowptr[i + 1] - 1]);
}

// ------------------------------------------------------------ host side

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// How the solves of one factor run: generic (any pattern, FP64 vectors and
// sums), pipelined (groups of <= 3 rows, <= WCOL external columns) or
// warp-specialised on premultiplied group blocks (gic_qsolve.cu; groups of
// <= 3 rows, <= QCOL external columns), each with an FP64 or an FP32
// factor. The pipelined and warp-specialised FP32 modes keep their vectors
// and sums in FP32 too.
// SM-local (gic_bsolve.cu) on the same blocks where the pattern's chunk
// blocks allow it.
enum SolveMode {
    MODE_GEN64, MODE_GEN32, MODE_P64, MODE_P32, MODE_Q64, MODE_Q32, MODE_S64, MODE_S32, MODE_D64, MODE_D32, MODE_IDENT
};

static bool f32_vectors(SolveMode m) { return m == MODE_P32 || m == MODE_Q32 || m == MODE_S32 || m == MODE_D32; }
static bool premultiplied(SolveMode m) { return m == MODE_Q64 || m == MODE_Q32; }
static bool sliced(SolveMode m) { return m == MODE_S64 || m == MODE_S32; }
static bool paired(SolveMode m) { return m == MODE_D64 || m == MODE_D32; }

struct SolveWs {
    void *Uval;                   // U values (generic, pipelined), backward blocks (warp-specialised) or
                                  // backward slice coefficients (level-sliced)
    void *Qf;                     // forward premultiplied blocks or forward slice coefficients
    double *invd;                 // generic modes and P64
    float *invd32, *r32, *y32, *z32; // P32
    double *r, *y, *z, *p, *w;
    double *partials;
    double *sval; // A's values in the pattern's SELL-32 layout
    Scalars *sc;
    size_t bytes;
};

static bool pipelined_fits(const Pattern &P)
{
    return P.max_group <= 3 && P.max_ext_lower <= WCOL && P.max_ext_upper <= WCOL;
}

static SolveMode solve_mode(const gic_handle *h, const Pattern &P, int l_dtype)
{
    if (l_dtype == GIC_IDENTITY) return MODE_IDENT;
    // automatic choice (measured on the hex systems from 40^3 to 148^3): the
    // level-sliced kernels (one lane per row) where many independent groups
    // are ready at once, i.e. many chunks per SM; the pair-sliced ones (half
    // the hand-offs, 1.7x the arithmetic) in a middle band; else the
    // warp-specialised kernels (three warps per chunk, most arithmetic off
    // the dependency chain) where the pattern admits them, else the staged
    // one-warp kernels
    int pipeline = h->tune_pipeline;
    if (pipeline == 4 || pipeline > 5) {
        const int64_t c = P.nchunks, sms = h->num_sms;
        pipeline = (c < (int64_t)SLICED_CHUNKS_PER_SM * sms) ? 2
                   : (P.pready == 1 && c < (int64_t)PAIRED_CHUNKS_PER_SM * sms) ? 5 : 3;
    }
    if (pipeline == 5 && P.pready) return (l_dtype == GIC_F32) ? MODE_D32 : MODE_D64;
    if (pipeline >= 3 && P.sready) return (l_dtype == GIC_F32) ? MODE_S32 : MODE_S64;
    if (pipeline >= 2 && P.qready) return (l_dtype == GIC_F32) ? MODE_Q32 : MODE_Q64;
    const bool pipe = pipeline && pipelined_fits(P);
    if (l_dtype == GIC_F32) return pipe ? MODE_P32 : MODE_GEN32;
    return pipe ? MODE_P64 : MODE_GEN64;
}

// Workspace layout for a PCG whose SpMV runs on pattern PA and whose solves
// run on the factor pattern PL (the same object unless the factor's pattern
// was thinned, e.g. by fill-in dropout).
static SolveWs carve(const Pattern &PA, const Pattern &PL, int l_dtype, SolveMode mode, void *ws)
{
    Pattern P;
    P.n = PA.n;
    P.nnzL = PL.nnzL;
    P.sell_nnz = PA.sell_nnz;
    const bool p32 = f32_vectors(mode);
    SolveWs o = {};
    char *c = (char *)ws;
    size_t off = 0;
    size_t es = (l_dtype == GIC_F32) ? 4 : 8;
    const size_t fb = sliced(mode) ? s_values_bytes(PL.sf, es)
                      : paired(mode) ? p_values_bytes(PL.pf, es) : es * (size_t)P.nnzL;
    const size_t bb = sliced(mode) ? s_values_bytes(PL.sb, es)
                      : paired(mode) ? p_values_bytes(PL.pb, es) : es * (size_t)P.nnzL;
    o.sc = (Scalars *)(c + off); off += align_up(sizeof(Scalars));
    o.partials = (double *)(c + off); off += align_up(sizeof(double) * 2 * MAX_PARTIALS);
    o.Uval = c + off; off += (l_dtype == GIC_IDENTITY) ? 0 : align_up(bb);
    o.Qf = c + off; off += (l_dtype == GIC_IDENTITY) ? 0 : align_up(fb);
    o.invd = (double *)(c + off); off += (l_dtype == GIC_IDENTITY) ? 0 : align_up(8 * (size_t)P.n);
    if (p32) {
        float **fv[4] = {&o.invd32, &o.r32, &o.y32, &o.z32};
        for (int k = 0; k < 4; ++k) { *fv[k] = (float *)(c + off); off += align_up(4 * (size_t)P.n); }
    }
    o.sval = (double *)(c + off); off += align_up(8 * (size_t)(PA.bsr_ready ? 288 * PA.bsr_steps : P.sell_nnz));
    double **vecs[5] = {&o.r, &o.y, &o.z, &o.p, &o.w};
    for (int k = 0; k < 5; ++k) { *vecs[k] = (double *)(c + off); off += align_up(8 * (size_t)P.n); }
    o.bytes = off;
    return o;
}

// Workspace bound for a PCG on a pattern not analysed yet (the end-to-end
// call): the warp-specialised layout plus room for the level-sliced and
// pair-sliced ones on patterns like the hex systems' (level-sliced: one
// slice per 10 groups of 3 rows, a few padded steps; pair-sliced: ≈ 2x the
// factor's entries per sweep for the substituted groups' longer lists); a
// pattern that needs more runs the warp-specialised solves.
size_t pcg_ws_bytes(int64_t n, int64_t nnzL, int64_t sell_nnz, int l_dtype)
{
    Pattern P;
    P.n = n;
    P.nnzL = nnzL;
    P.sell_nnz = sell_nnz;
    const size_t es = (l_dtype == GIC_F32) ? 4 : 8;
    const SolveMode m = (l_dtype == GIC_F32) ? MODE_Q32 : MODE_Q64;
    return carve(P, P, l_dtype, m, nullptr).bytes + es * (size_t)(nnzL / 4 * 9 + 16 * n) + 4096;
}

static unsigned vec_grid(gic_handle *h, int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    int64_t cap = (int64_t)h->num_sms * 8; // 64 warps per SM: enough loads in flight for HBM
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

static unsigned spmv_grid(gic_handle *h, int64_t n)
{
    int64_t warps = SPMV_BLOCK / 32;
    int64_t b = (n + warps - 1) / warps;
    int64_t cap = (int64_t)h->num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

static int64_t solve_warps(gic_handle *h, const Pattern &P)
{
    int64_t need = P.nchunks;
    if (h->tune_solve_warps_per_sm > 0) {
        int64_t cap = (int64_t)h->tune_solve_warps_per_sm * h->num_sms;
        if (need > cap) need = cap;
    }
    return need;
}

// ---- generic kernels (FP64 vectors)
template <typename TL, int GM>
static int launch_lsolve_g(gic_handle *h, const Pattern &P, const TL *Lval, const double *invd, const double *r,
                           double *y, Scalars *sc)
{
    int32_t nc = P.nchunks;
    const int32_t *ord = P.ord_f, *cg = P.chunk_grp, *g = P.grp, *lr = P.Lrowptr, *lc = P.Lcol;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&nc, &ord, &cg, &g, &lr, &lc, &Lval, &invd, &r, &y, &er, &poll, &sc};
    const size_t smem = sizeof(WarpStage) * (SOLVE_BLOCK / 32);
    static bool ad[64] = {};
    if (!ad[h->device & 63]) {
        GIC_CUDA_TRY(cudaFuncSetAttribute(k_lsolve<TL, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ad[h->device & 63] = true;
    }
    return launch_persistent(h, (const void *)k_lsolve<TL, GM>, SOLVE_BLOCK, smem, solve_warps(h, P), args);
}

template <typename TL>
static int launch_lsolve_gen(gic_handle *h, const Pattern &P, const TL *Lval, const double *invd, const double *r,
                             double *y, Scalars *sc)
{
    if (P.max_group <= 1) return launch_lsolve_g<TL, 1>(h, P, Lval, invd, r, y, sc);
    if (P.max_group <= 3) return launch_lsolve_g<TL, 3>(h, P, Lval, invd, r, y, sc);
    return launch_lsolve_g<TL, GMAX>(h, P, Lval, invd, r, y, sc);
}

template <typename TL, bool PCG, int GM>
static int launch_ltsolve_g(gic_handle *h, const Pattern &P, const TL *Uval, const double *invd, double *y, double *z,
                            const double *r, double *partials, Scalars *sc)
{
    int32_t nc = P.nchunks;
    const int32_t *ord = P.ord_b, *cg = P.chunk_grp, *g = P.grp, *ur = P.Urowptr, *uc = P.Ucol;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&nc, &ord, &cg, &g, &ur, &uc, &Uval, &invd, &y, &z, &r, &partials, &er, &poll, &sc};
    int64_t need = solve_warps(h, P);
    if (PCG && need > MAX_PARTIALS) need = MAX_PARTIALS; // grid warps <= partial slots
    const size_t smem = sizeof(WarpStage) * (SOLVE_BLOCK / 32);
    static bool ad[64] = {};
    if (!ad[h->device & 63]) {
        GIC_CUDA_TRY(cudaFuncSetAttribute(k_ltsolve<TL, PCG, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        ad[h->device & 63] = true;
    }
    return launch_persistent(h, (const void *)k_ltsolve<TL, PCG, GM>, SOLVE_BLOCK, smem, need, args);
}

template <typename TL, bool PCG>
static int launch_ltsolve_gen(gic_handle *h, const Pattern &P, const TL *Uval, const double *invd, double *y,
                              double *z, const double *r, double *partials, Scalars *sc)
{
    if (P.max_group <= 1) return launch_ltsolve_g<TL, PCG, 1>(h, P, Uval, invd, y, z, r, partials, sc);
    if (P.max_group <= 3) return launch_ltsolve_g<TL, PCG, 3>(h, P, Uval, invd, y, z, r, partials, sc);
    return launch_ltsolve_g<TL, PCG, GMAX>(h, P, Uval, invd, y, z, r, partials, sc);
}

// ---- pipelined kernels (vectors and sums in T)
template <typename T, int GM>
static int launch_lsolve_pg(gic_handle *h, const Pattern &P, const T *Lval, const T *invd, const T *r, T *y,
                            Scalars *sc)
{
    int32_t nc = P.nchunks;
    const int32_t *ord = P.ord_f, *cg = P.chunk_grp, *g = P.grp, *lr = P.Lrowptr, *lc = P.Lcol;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&nc, &ord, &cg, &g, &lr, &lc, &Lval, &invd, &r, &y, &er, &poll, &sc};
    const size_t smem = sizeof(PWarp<T, GM>) * (SOLVE_BLOCK / 32);
    static bool ad[64] = {};
    if (!ad[h->device & 63]) {
        GIC_CUDA_TRY(cudaFuncSetAttribute(k_lsolve_p<T, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ad[h->device & 63] = true;
    }
    return launch_persistent(h, (const void *)k_lsolve_p<T, GM>, SOLVE_BLOCK, smem, solve_warps(h, P), args);
}

template <typename T>
static int launch_lsolve_p(gic_handle *h, const Pattern &P, const T *Lval, const T *invd, const T *r, T *y, Scalars *sc)
{
    if (P.max_group <= 1) return launch_lsolve_pg<T, 1>(h, P, Lval, invd, r, y, sc);
    return launch_lsolve_pg<T, 3>(h, P, Lval, invd, r, y, sc);
}

template <typename T, bool PCG, int GM>
static int launch_ltsolve_pg(gic_handle *h, const Pattern &P, const T *Uval, const T *invd, T *y, T *z,
                             const double *rd, double *partials, Scalars *sc)
{
    int32_t nc = P.nchunks;
    const int32_t *ord = P.ord_b, *cg = P.chunk_grp, *g = P.grp, *ur = P.Urowptr, *uc = P.Ucol;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&nc, &ord, &cg, &g, &ur, &uc, &Uval, &invd, &y, &z, &rd, &partials, &er, &poll, &sc};
    int64_t need = solve_warps(h, P);
    if (PCG && need > MAX_PARTIALS) need = MAX_PARTIALS;
    const size_t smem = sizeof(PWarp<T, GM>) * (SOLVE_BLOCK / 32);
    static bool ad[64] = {};
    if (!ad[h->device & 63]) {
        GIC_CUDA_TRY(cudaFuncSetAttribute(k_ltsolve_p<T, PCG, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        ad[h->device & 63] = true;
    }
    return launch_persistent(h, (const void *)k_ltsolve_p<T, PCG, GM>, SOLVE_BLOCK, smem, need, args);
}

template <typename T, bool PCG>
static int launch_ltsolve_p(gic_handle *h, const Pattern &P, const T *Uval, const T *invd, T *y, T *z,
                            const double *rd, double *partials, Scalars *sc)
{
    if (P.max_group <= 1) return launch_ltsolve_pg<T, PCG, 1>(h, P, Uval, invd, y, z, rd, partials, sc);
    return launch_ltsolve_pg<T, PCG, 3>(h, P, Uval, invd, y, z, rd, partials, sc);
}

// Transposed values and reciprocal diagonal for the mode.
static int setup_factor(gic_handle *h, const Pattern &P, SolveMode mode, const void *Lval, const SolveWs &W)
{
    if (premultiplied(mode)) return q_setup(h, P, f32_vectors(mode), Lval, W.Qf, W.Uval);
    if (sliced(mode)) return s_setup(h, P, f32_vectors(mode), Lval, W.Qf, W.Uval);
    if (paired(mode)) return p_setup(h, P, f32_vectors(mode), Lval, W.Qf, W.Uval);
    int64_t cnt = P.nnzL > P.n ? P.nnzL : P.n;
    unsigned gr = vec_grid(h, cnt, 256);
    ++h->launches;
    if (mode == MODE_GEN64 || mode == MODE_P64)
        k_factor_setup<double, double><<<gr, 256, 0, h->stream>>>(P.n, P.nnzL, P.tperm, P.Lrowptr,
                                                                   (const double *)Lval, (double *)W.Uval, W.invd);
    else if (mode == MODE_GEN32)
        k_factor_setup<float, double><<<gr, 256, 0, h->stream>>>(P.n, P.nnzL, P.tperm, P.Lrowptr,
                                                                  (const float *)Lval, (float *)W.Uval, W.invd);
    else if (mode == MODE_P32)
        k_factor_setup<float, float><<<gr, 256, 0, h->stream>>>(P.n, P.nnzL, P.tperm, P.Lrowptr, (const float *)Lval,
                                                                 (float *)W.Uval, W.invd32);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

// Optional per-kernel-class timing: while enabled, a pair of CUDA events is
// recorded on the handle's stream around every solve-path launch (no host
// synchronisation), and the elapsed times are summed into the classes when a
// call finishes (or the event pool fills).
struct Prof {
    int on = 0;
    int used = 0;
    static constexpr int CAP = 8192;
    cudaEvent_t ev[CAP] = {};
    int cls[CAP / 2] = {};
    double ms[GIC_PROF_CLASSES] = {0};
    long long launches[GIC_PROF_CLASSES] = {0};
};
static Prof *g_prof[64];

static Prof &prof_of(gic_handle *h)
{
    Prof *&p = g_prof[h->device & 63];
    if (!p) p = new Prof();
    return *p;
}

static int prof_flush(gic_handle *h, Prof &pr)
{
    if (pr.used == 0) return GIC_OK;
    GIC_CUDA_TRY(cudaEventSynchronize(pr.ev[pr.used - 1]));
    for (int k = 0; k + 1 < pr.used; k += 2) {
        float t = 0.f;
        GIC_CUDA_TRY(cudaEventElapsedTime(&t, pr.ev[k], pr.ev[k + 1]));
        pr.ms[pr.cls[k / 2]] += t;
        pr.launches[pr.cls[k / 2]] += 1;
    }
    pr.used = 0;
    return GIC_OK;
}

#define PROF_BEGIN(c)                                                              \
    if (pr.on) {                                                                   \
        if (pr.used + 2 > Prof::CAP) GIC_TRY(prof_flush(h, pr));                   \
        GIC_CUDA_TRY(cudaEventRecord(pr.ev[pr.used], h->stream));                  \
        pr.cls[pr.used / 2] = (c);                                                 \
    }
#define PROF_END(c)                                                                \
    if (pr.on) {                                                                   \
        GIC_CUDA_TRY(cudaEventRecord(pr.ev[pr.used + 1], h->stream));              \
        pr.used += 2;                                                              \
    }

// Forward then backward solve of one PCG step for the mode (z in W.z or W.z32).
static int precondition(gic_handle *h, const Pattern &P, SolveMode mode, const void *Lval, const SolveWs &W)
{
    Prof &pr = prof_of(h);
    PROF_BEGIN(GIC_PROF_LSOLVE);
    switch (mode) {
    case MODE_GEN64: GIC_TRY(launch_lsolve_gen<double>(h, P, (const double *)Lval, W.invd, W.r, W.y, W.sc)); break;
    case MODE_GEN32: GIC_TRY(launch_lsolve_gen<float>(h, P, (const float *)Lval, W.invd, W.r, W.y, W.sc)); break;
    case MODE_P64: GIC_TRY(launch_lsolve_p<double>(h, P, (const double *)Lval, W.invd, W.r, W.y, W.sc)); break;
    case MODE_P32: GIC_TRY(launch_lsolve_p<float>(h, P, (const float *)Lval, W.invd32, W.r32, W.y32, W.sc)); break;
    case MODE_Q64: GIC_TRY(q_lsolve(h, P, false, W.Qf, W.r, W.y, W.sc)); break;
    case MODE_Q32: GIC_TRY(q_lsolve(h, P, true, W.Qf, W.r32, W.y32, W.sc)); break;
    case MODE_S64: GIC_TRY(s_lsolve(h, P, false, W.Qf, W.r, W.y, W.sc)); break;
    case MODE_S32: GIC_TRY(s_lsolve(h, P, true, W.Qf, W.r32, W.y32, W.sc)); break;
    case MODE_D64: GIC_TRY(p_lsolve(h, P, false, W.Qf, W.r, W.y, W.sc)); break;
    case MODE_D32: GIC_TRY(p_lsolve(h, P, true, W.Qf, W.r32, W.y32, W.sc)); break;
    default: break;
    }
    PROF_END(GIC_PROF_LSOLVE);
    PROF_BEGIN(GIC_PROF_LTSOLVE);
    switch (mode) {
    case MODE_GEN64:
        GIC_TRY((launch_ltsolve_gen<double, true>(h, P, (const double *)W.Uval, W.invd, W.y, W.z, W.r, W.partials, W.sc)));
        break;
    case MODE_GEN32:
        GIC_TRY((launch_ltsolve_gen<float, true>(h, P, (const float *)W.Uval, W.invd, W.y, W.z, W.r, W.partials, W.sc)));
        break;
    case MODE_P64:
        GIC_TRY((launch_ltsolve_p<double, true>(h, P, (const double *)W.Uval, W.invd, W.y, W.z, W.r, W.partials, W.sc)));
        break;
    case MODE_P32:
        GIC_TRY((launch_ltsolve_p<float, true>(h, P, (const float *)W.Uval, W.invd32, W.y32, W.z32, W.r, W.partials,
                                               W.sc)));
        break;
    case MODE_Q64: GIC_TRY(q_ltsolve(h, P, false, true, W.Uval, W.y, W.z, W.r, W.partials, W.sc)); break;
    case MODE_Q32: GIC_TRY(q_ltsolve(h, P, true, true, W.Uval, W.y32, W.z32, W.r, W.partials, W.sc)); break;
    case MODE_S64: GIC_TRY(s_ltsolve(h, P, false, true, W.Uval, W.y, W.z, W.r, W.partials, W.sc)); break;
    case MODE_S32: GIC_TRY(s_ltsolve(h, P, true, true, W.Uval, W.y32, W.z32, W.r, W.partials, W.sc)); break;
    case MODE_D64: GIC_TRY(p_ltsolve(h, P, false, true, W.Uval, W.y, W.z, W.r, W.partials, W.sc)); break;
    case MODE_D32: GIC_TRY(p_ltsolve(h, P, true, true, W.Uval, W.y32, W.z32, W.r, W.partials, W.sc)); break;
    default: break;
    }
    PROF_END(GIC_PROF_LTSOLVE);
    return GIC_OK;
}

// One PCG iteration: lines 11-18 of Algorithm 1 and the stop test.
static int pcg_iteration(gic_handle *h, const Pattern &P, const Pattern &PL, SolveMode mode, const double *valA,
                         const void *Lval, const SolveWs &W, double *x)
{
    const int64_t n = P.n;
    Prof &pr = prof_of(h);
    const unsigned vg = vec_grid(h, n, VEC_BLOCK);
    if (mode == MODE_IDENT) {
        PROF_BEGIN(GIC_PROF_VECTOR);
        ++h->launches;
        k_ident_rz<<<vg, VEC_BLOCK, 0, h->stream>>>(n, W.r, W.partials, W.sc);
        ++h->launches;
        k_update_p<true, double><<<vg, VEC_BLOCK, 0, h->stream>>>(n, W.z, W.p, W.r, nullptr, W.sc);
        GIC_CUDA_TRY(cudaGetLastError());
        PROF_END(GIC_PROF_VECTOR);
    } else {
        GIC_TRY(precondition(h, PL, mode, Lval, W));
        PROF_BEGIN(GIC_PROF_VECTOR);
        ++h->launches;
        if (f32_vectors(mode))
            k_update_p<false, float><<<vg, VEC_BLOCK, 0, h->stream>>>(n, W.z32, W.p, W.r,
                                                                      paired(mode) ? W.y32 : nullptr, W.sc);
        else
            k_update_p<false, double><<<vg, VEC_BLOCK, 0, h->stream>>>(n, W.z, W.p, W.r,
                                                                       paired(mode) ? W.y : nullptr, W.sc);
        GIC_CUDA_TRY(cudaGetLastError());
        PROF_END(GIC_PROF_VECTOR);
    }
    PROF_BEGIN(GIC_PROF_SPMV);
    if (P.bsr_ready) {
        GIC_TRY(bsr_spmv(h, P, 1, W.sval, W.p, W.w, nullptr, W.partials, W.sc));
    } else {
        ++h->launches;
        k_spmv_sell<1><<<spmv_grid(h, P.nslices), SPMV_BLOCK, 0, h->stream>>>(
            n, P.nslices, P.sell_ptr, P.sell_w, P.sell_col, W.sval, W.p, W.w, nullptr, W.partials, W.sc);
        GIC_CUDA_TRY(cudaGetLastError());
    }
    PROF_END(GIC_PROF_SPMV);
    PROF_BEGIN(GIC_PROF_VECTOR);
    ++h->launches;
    k_update_xr<<<vg, VEC_BLOCK, 0, h->stream>>>(n, x, W.r, W.p, W.w, f32_vectors(mode) ? W.r32 : nullptr, W.partials,
                                                 W.sc);
    GIC_CUDA_TRY(cudaGetLastError());
    PROF_END(GIC_PROF_VECTOR);
    return GIC_OK;
}

static int pcg_run(gic_handle *h, const Pattern &P, const Pattern &PL, SolveMode mode, const double *valA,
                   const void *Lval, const double *b, double *x, double rtol, int maxit, int32_t *iters, double *relres,
                   const SolveWs &W)
{
    const int64_t n = P.n;
    Prof &pr = prof_of(h);
    const unsigned vg = vec_grid(h, n, 256);
    ++h->launches;
    k_init_scalars<<<1, 1, 0, h->stream>>>(W.sc, rtol, maxit);
    if (mode != MODE_IDENT) {
        GIC_TRY(setup_factor(h, PL, mode, Lval, W));
        ++h->launches;
        if (f32_vectors(mode)) k_fill_sentinel_t<float><<<vg, 256, 0, h->stream>>>(n, W.y32, W.z32);
        else k_fill_sentinel_t<double><<<vg, 256, 0, h->stream>>>(n, W.y, W.z);
    }
    if (P.bsr_ready) {
        GIC_TRY(bsr_values(h, P, valA, W.sval));
    } else {
        ++h->launches;
        k_sell_vals<<<vec_grid(h, P.nslices * 32, 256), 256, 0, h->stream>>>(n, P.nslices, P.rowptr, valA,
                                                                              P.sell_ptr, P.sell_w, W.sval);
    }
    PROF_BEGIN(GIC_PROF_SPMV);
    if (P.bsr_ready) {
        GIC_TRY(bsr_spmv(h, P, 2, W.sval, x, W.r, b, W.partials, W.sc));
    } else {
        ++h->launches;
        k_spmv_sell<2><<<spmv_grid(h, P.nslices), SPMV_BLOCK, 0, h->stream>>>(
            n, P.nslices, P.sell_ptr, P.sell_w, P.sell_col, W.sval, x, W.r, b, W.partials, W.sc);
        GIC_CUDA_TRY(cudaGetLastError());
    }
    PROF_END(GIC_PROF_SPMV);
    if (f32_vectors(mode)) {
        ++h->launches;
        k_convert_f64_f32<<<vg, 256, 0, h->stream>>>(n, W.r, W.r32);
    }
    // Iterations are enqueued in batches; the host reads the device flag of
    // the previous batch while the next one runs (finished kernels exit at
    // once when done is set), so the GPU does not idle on the check.
    const int BATCH = 4;
    Scalars *hs = (Scalars *)h->host_pinned;
    cudaEvent_t ev_done = nullptr;
    GIC_CUDA_TRY(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
    int enq = 0, rc = GIC_OK;
    bool pending = false;
    while (true) {
        int todo = BATCH;
        if (enq + todo > maxit) todo = maxit - enq;
        for (int k = 0; k < todo && rc == GIC_OK; ++k) rc = pcg_iteration(h, P, PL, mode, valA, Lval, W, x);
        if (rc != GIC_OK) break;
        enq += todo;
        if (pending) {
            cudaError_t e = cudaEventSynchronize(ev_done);
            if (e != cudaSuccess) { set_last_cuda_error(e, "pcg sync", __FILE__, __LINE__); rc = GIC_ERR_CUDA; break; }
            if (hs->done || hs->iter >= maxit) break;
        }
        cudaError_t e = cudaMemcpyAsync(hs, W.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev_done, h->stream);
        if (e != cudaSuccess) { set_last_cuda_error(e, "pcg readback", __FILE__, __LINE__); rc = GIC_ERR_CUDA; break; }
        pending = true;
        if (enq >= maxit || todo == 0) {
            e = cudaEventSynchronize(ev_done);
            if (e != cudaSuccess) { set_last_cuda_error(e, "pcg sync", __FILE__, __LINE__); rc = GIC_ERR_CUDA; }
            break;
        }
    }
    cudaEventDestroy(ev_done);
    if (rc != GIC_OK) return rc;
    GIC_TRY(prof_flush(h, pr));
    GIC_CUDA_TRY(cudaMemcpyAsync(hs, W.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    Scalars out = *hs;
    unsigned flags = 0;
    GIC_TRY(read_and_clear_dev_err(h, &flags));
    if (iters) *iters = out.iter;
    if (relres) *relres = (out.bb > 0.0) ? sqrt(out.rr) / sqrt(out.bb) : 0.0;
    if (flags & ERR_TIMEOUT) return GIC_ERR_TIMEOUT;
    if (!out.done) return GIC_ERR_NO_CONVERGENCE;
    return out.status;
}

// Standalone forward / backward solve (gic_lsolve, gic_ltsolve).
static int standalone_solve(gic_handle *h, const Pattern &p, const void *valL, int l_dtype, const double *in,
                            double *out, void *ws, size_t ws_bytes, bool forward)
{
    const SolveMode mode = solve_mode(h, p, l_dtype);
    SolveWs W = carve(p, p, l_dtype, mode, ws);
    if (ws_bytes < W.bytes) return GIC_ERR_WORKSPACE;
    const unsigned vg = vec_grid(h, p.n, 256);
    GIC_TRY(setup_factor(h, p, mode, valL, W));
    Prof &pr = prof_of(h);
    if (f32_vectors(mode)) {
        ++h->launches;
        k_convert_f64_f32<<<vg, 256, 0, h->stream>>>(p.n, in, W.r32); // the input, whichever sweep
        ++h->launches;
        k_fill_sentinel_t<float><<<vg, 256, 0, h->stream>>>(p.n, W.y32, nullptr);
    } else {
        ++h->launches;
        k_fill_sentinel_t<double><<<vg, 256, 0, h->stream>>>(p.n, out, nullptr);
    }
    if (forward) {
        PROF_BEGIN(GIC_PROF_LSOLVE);
        switch (mode) {
        case MODE_GEN64: GIC_TRY(launch_lsolve_gen<double>(h, p, (const double *)valL, W.invd, in, out, nullptr)); break;
        case MODE_GEN32: GIC_TRY(launch_lsolve_gen<float>(h, p, (const float *)valL, W.invd, in, out, nullptr)); break;
        case MODE_P64: GIC_TRY(launch_lsolve_p<double>(h, p, (const double *)valL, W.invd, in, out, nullptr)); break;
        case MODE_P32: GIC_TRY(launch_lsolve_p<float>(h, p, (const float *)valL, W.invd32, W.r32, W.y32, nullptr)); break;
        case MODE_Q64: GIC_TRY(q_lsolve(h, p, false, W.Qf, in, out, nullptr)); break;
        case MODE_Q32: GIC_TRY(q_lsolve(h, p, true, W.Qf, W.r32, W.y32, nullptr)); break;
        case MODE_S64: GIC_TRY(s_lsolve(h, p, false, W.Qf, in, out, nullptr)); break;
        case MODE_S32: GIC_TRY(s_lsolve(h, p, true, W.Qf, W.r32, W.y32, nullptr)); break;
        case MODE_D64: GIC_TRY(p_lsolve(h, p, false, W.Qf, in, out, nullptr)); break;
        case MODE_D32: GIC_TRY(p_lsolve(h, p, true, W.Qf, W.r32, W.y32, nullptr)); break;
        default: break;
        }
        PROF_END(GIC_PROF_LSOLVE);
    } else {
        double *yy = const_cast<double *>(in); // not written when PCG = false
        PROF_BEGIN(GIC_PROF_LTSOLVE);
        switch (mode) {
        case MODE_GEN64:
            GIC_TRY((launch_ltsolve_gen<double, false>(h, p, (const double *)W.Uval, W.invd, yy, out, nullptr, nullptr, nullptr)));
            break;
        case MODE_GEN32:
            GIC_TRY((launch_ltsolve_gen<float, false>(h, p, (const float *)W.Uval, W.invd, yy, out, nullptr, nullptr, nullptr)));
            break;
        case MODE_P64:
            GIC_TRY((launch_ltsolve_p<double, false>(h, p, (const double *)W.Uval, W.invd, yy, out, nullptr, nullptr, nullptr)));
            break;
        case MODE_P32:
            GIC_TRY((launch_ltsolve_p<float, false>(h, p, (const float *)W.Uval, W.invd32, W.r32, W.y32, nullptr, nullptr,
                                                   nullptr)));
            break;
        case MODE_Q64: GIC_TRY(q_ltsolve(h, p, false, false, W.Uval, yy, out, nullptr, nullptr, nullptr)); break;
        case MODE_Q32: GIC_TRY(q_ltsolve(h, p, true, false, W.Uval, W.r32, W.y32, nullptr, nullptr, nullptr)); break;
        case MODE_S64: GIC_TRY(s_ltsolve(h, p, false, false, W.Uval, yy, out, nullptr, nullptr, nullptr)); break;
        case MODE_S32: GIC_TRY(s_ltsolve(h, p, true, false, W.Uval, W.r32, W.y32, nullptr, nullptr, nullptr)); break;
        case MODE_D64: GIC_TRY(p_ltsolve(h, p, false, false, W.Uval, yy, out, nullptr, nullptr, nullptr)); break;
        case MODE_D32: GIC_TRY(p_ltsolve(h, p, true, false, W.Uval, W.r32, W.y32, nullptr, nullptr, nullptr)); break;
        default: break;
        }
        PROF_END(GIC_PROF_LTSOLVE);
    }
    if (f32_vectors(mode)) {
        ++h->launches;
        k_convert_f32_f64<<<vg, 256, 0, h->stream>>>(p.n, W.y32, out);
    }
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

}  // namespace gic

using namespace gic;

static int check_pattern(gic_handle *h, const gic_pattern *P)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device) return GIC_ERR_INVALID_ARG;
    return GIC_OK;
}

extern "C" {

int gic_workspace_size(gic_handle *h, const gic_pattern *P, int op, int l_dtype, size_t *bytes)
{
    GIC_TRY(check_pattern(h, P));
    if (!bytes || (l_dtype != GIC_F64 && l_dtype != GIC_F32 && l_dtype != GIC_IDENTITY)) return GIC_ERR_INVALID_ARG;
    if (op != GIC_WS_SOLVE && op != GIC_WS_PCG) return GIC_ERR_INVALID_ARG;
    *bytes = carve(P->p, P->p, l_dtype, solve_mode(h, P->p, l_dtype), nullptr).bytes;
    return GIC_OK;
}

int gic_convert_f64_f32(gic_handle *h, int64_t count, const double *src, float *dst)
{
    GIC_TRY(check_handle(h));
    if (count < 0 || (count > 0 && (!src || !dst))) return GIC_ERR_INVALID_ARG;
    if (count == 0) return GIC_OK;
    ++h->launches;
    k_convert_f64_f32<<<vec_grid(h, count, 256), 256, 0, h->stream>>>(count, src, dst);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_spmv(gic_handle *h, const gic_pattern *P, const double *valA, const double *x, double *y, double *xdoty)
{
    GIC_TRY(check_pattern(h, P));
    if (!valA || !x || !y) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    // scalars + partials live in the handle's small scratch for this call
    Scalars *sc = (Scalars *)h->dev_small;
    double *partials = (double *)((char *)h->dev_small + 1024);
    unsigned grid = spmv_grid(h, p.n);
    if (xdoty && grid > (65536 - 1024) / 8) return GIC_ERR_UNSUPPORTED;
    if (xdoty) GIC_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(Scalars), h->stream));
    ++h->launches;
    k_spmv<0><<<grid, SPMV_BLOCK, 0, h->stream>>>(p.n, p.rowptr, p.col, valA, x, y, nullptr, partials, xdoty, sc);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_lsolve(gic_handle *h, const gic_pattern *P, const void *valL, int l_dtype, const double *r, double *y,
               void *ws, size_t ws_bytes)
{
    GIC_TRY(check_pattern(h, P));
    if (!valL || !r || !y || !ws || (l_dtype != GIC_F64 && l_dtype != GIC_F32)) return GIC_ERR_INVALID_ARG;
    return standalone_solve(h, P->p, valL, l_dtype, r, y, ws, ws_bytes, true);
}

int gic_ltsolve(gic_handle *h, const gic_pattern *P, const void *valL, int l_dtype, const double *y, double *z,
                void *ws, size_t ws_bytes)
{
    GIC_TRY(check_pattern(h, P));
    if (!valL || !y || !z || !ws || (l_dtype != GIC_F64 && l_dtype != GIC_F32)) return GIC_ERR_INVALID_ARG;
    return standalone_solve(h, P->p, valL, l_dtype, y, z, ws, ws_bytes, false);
}

int gic_solve_error_flags(gic_handle *h, unsigned *flags)
{
    GIC_TRY(check_handle(h));
    if (!flags) return GIC_ERR_INVALID_ARG;
    return read_and_clear_dev_err(h, flags);
}

int gic_pcg(gic_handle *h, const gic_pattern *P, const double *valA, const void *valL, int l_dtype, const double *b,
            double *x, double rtol, int maxit, int32_t *iters, double *relres, void *ws, size_t ws_bytes)
{
    return gic_pcg_split(h, P, valA, P, valL, l_dtype, b, x, rtol, maxit, iters, relres, ws, ws_bytes);
}

int gic_workspace_size_split(gic_handle *h, const gic_pattern *PA, const gic_pattern *PL, int l_dtype, size_t *bytes)
{
    GIC_TRY(check_pattern(h, PA));
    GIC_TRY(check_pattern(h, PL));
    if (!bytes || (l_dtype != GIC_F64 && l_dtype != GIC_F32 && l_dtype != GIC_IDENTITY)) return GIC_ERR_INVALID_ARG;
    if (PA->p.n != PL->p.n) return GIC_ERR_INVALID_ARG;
    *bytes = carve(PA->p, PL->p, l_dtype, solve_mode(h, PL->p, l_dtype), nullptr).bytes;
    return GIC_OK;
}

int gic_pcg_split(gic_handle *h, const gic_pattern *PA, const double *valA, const gic_pattern *PL, const void *valL,
                  int l_dtype, const double *b, double *x, double rtol, int maxit, int32_t *iters, double *relres,
                  void *ws, size_t ws_bytes)
{
    GIC_TRY(check_pattern(h, PA));
    GIC_TRY(check_pattern(h, PL));
    if (!valA || !b || !x || !ws || maxit < 0 || !(rtol >= 0.0)) return GIC_ERR_INVALID_ARG;
    if (l_dtype != GIC_IDENTITY && !valL) return GIC_ERR_INVALID_ARG;
    if (l_dtype != GIC_F64 && l_dtype != GIC_F32 && l_dtype != GIC_IDENTITY) return GIC_ERR_INVALID_ARG;
    const Pattern &p = PA->p, &pl = PL->p;
    if (p.n != pl.n) return GIC_ERR_INVALID_ARG;
    SolveMode mode = solve_mode(h, pl, l_dtype);
    SolveWs W = carve(p, pl, l_dtype, mode, ws);
    if (ws_bytes < W.bytes && (sliced(mode) || paired(mode))) { // a workspace sized before the analysis
        mode = (l_dtype == GIC_F32) ? MODE_Q32 : MODE_Q64;
        W = carve(p, pl, l_dtype, mode, ws);
    }
    if (ws_bytes < W.bytes) return GIC_ERR_WORKSPACE;
    if (p.ngroups > 0 && (spmv_grid(h, p.nslices) > MAX_PARTIALS || vec_grid(h, p.n, VEC_BLOCK) > MAX_PARTIALS))
        return GIC_ERR_UNSUPPORTED;
    return pcg_run(h, p, pl, mode, valA, valL, b, x, rtol, maxit, iters, relres, W);
}

int gic_profile_enable(gic_handle *h, int on)
{
    GIC_TRY(check_handle(h));
    Prof &pr = prof_of(h);
    GIC_TRY(prof_flush(h, pr));
    if (on && !pr.ev[0])
        for (int k = 0; k < Prof::CAP; ++k) GIC_CUDA_TRY(cudaEventCreate(&pr.ev[k]));
    pr.on = on ? 1 : 0;
    for (int k = 0; k < GIC_PROF_CLASSES; ++k) {
        pr.ms[k] = 0.0;
        pr.launches[k] = 0;
    }
    return GIC_OK;
}

int gic_profile_read(gic_handle *h, double *ms, int64_t *launches)
{
    GIC_TRY(check_handle(h));
    Prof &pr = prof_of(h);
    GIC_TRY(prof_flush(h, pr));
    for (int k = 0; k < GIC_PROF_CLASSES; ++k) {
        if (ms) ms[k] = pr.ms[k];
        if (launches) launches[k] = pr.launches[k];
    }
    return GIC_OK;
}

int gic_set_tuning(gic_handle *h, int key, int value)
{
    if (!h || value < 0) return GIC_ERR_INVALID_ARG;
    switch (key) {
    case GIC_TUNE_SOLVE_WARPS_PER_SM: h->tune_solve_warps_per_sm = value; return GIC_OK;
    case GIC_TUNE_POLL: h->tune_poll = value; return GIC_OK;
    case GIC_TUNE_PIPELINE: h->tune_pipeline = value; return GIC_OK;
    case GIC_TUNE_QDELTA: h->tune_qdelta = value; return GIC_OK;
    case GIC_TUNE_GNN_BF16: h->tune_gnn_bf16 = value; return GIC_OK;
    case GIC_TUNE_TRAIN_BF16: h->tune_train_bf16 = value; return GIC_OK;
    case GIC_TUNE_PAIR_LEVELS: h->tune_pair_levels = value; return GIC_OK;
    default: return GIC_ERR_INVALID_ARG;
    }
}

int gic_solve_kernels_chosen(gic_handle *h, const gic_pattern *P, int l_dtype, int32_t *pipeline)
{
    GIC_TRY(check_pattern(h, P));
    if (!pipeline || (l_dtype != GIC_F64 && l_dtype != GIC_F32)) return GIC_ERR_INVALID_ARG;
    switch (solve_mode(h, P->p, l_dtype)) {
    case MODE_D64: case MODE_D32: *pipeline = 5; break;
    case MODE_S64: case MODE_S32: *pipeline = 3; break;
    case MODE_Q64: case MODE_Q32: *pipeline = 2; break;
    case MODE_P64: case MODE_P32: *pipeline = 1; break;
    default: *pipeline = 0; break;
    }
    return GIC_OK;
}

int gic_pattern_spmv_layout(const gic_pattern *P, int32_t *node_blocks, int64_t *entries)
{
    if (!P) return GIC_ERR_INVALID_ARG;
    if (node_blocks) *node_blocks = P->p.bsr_ready;
    if (entries) *entries = P->p.bsr_ready ? 9 * 32 * P->p.bsr_steps : P->p.sell_nnz;
    return GIC_OK;
}

int gic_pattern_schedule(const gic_pattern *P, int32_t *nchunks, int32_t *chunked, int64_t *sell_nnz)
{
    if (!P) return GIC_ERR_INVALID_ARG;
    if (nchunks) *nchunks = P->p.nchunks;
    if (chunked) *chunked = P->p.chunked;
    if (sell_nnz) *sell_nnz = P->p.sell_nnz;
    return GIC_OK;
}

int gic_launch_count(gic_handle *h, int64_t *count)
{
    if (!h || !count) return GIC_ERR_INVALID_ARG;
    *count = h->launches;
    return GIC_OK;
}

}  // extern "C"

// ------------------------------------------------------------ no-allocation SpMV
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator hooks, services that must not touch
// the device heap after start-up, or code between stream-ordered operations
// where a synchronous allocation is not allowed. gic_spmv_dot_noalloc serves
// them: it needs no handle and no workspace, because its scratch (the
// per-block partial sums of x^T y and the reduction's completion counter)
// lives in this file-scope device array, which every GPU that loads the
// library holds until the process exits (about 8 MiB).
namespace gic {

// one partial per block; the launch uses at most min(8 per SM, this many)
constexpr int64_t NOALLOC_SLOTS = 1 << 20;
constexpr int64_t NOALLOC_MAX_ROWS = 8 * NOALLOC_SLOTS; // the stated row limit: 8,388,608 rows

struct NoallocScratch {
    Scalars sc; // only its last-block counter is used; zeroed by every call
    double partials[NOALLOC_SLOTS];
};
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of the scratch in the calling thread's current context. In
// host code the symbol only names a host-side stand-in; a kernel given it
// would fault or read the wrong memory. The address belongs to one context
// (a device's primary context, another driver context on the same device,
// or the primary context again after cudaDeviceReset each load their own
// copy of the module), so it is cached per context ID, which the driver never
// reuses within a process; the cache is filled under a mutex.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

struct NoallocCacheEntry {
    unsigned long long ctx_id;
    NoallocScratch *addr;
};
constexpr int NOALLOC_CACHE = 16;
static std::mutex g_noalloc_mu;
static NoallocCacheEntry g_noalloc_cache[NOALLOC_CACHE];
static int g_noalloc_next = 0;
static PfnCtxGetCurrent g_ctx_get_current = nullptr;
static PfnCtxGetId g_ctx_get_id = nullptr;
static bool g_noalloc_pfn_ok = false, g_noalloc_pfn_tried = false;

// current context's ID; 0 if no context is current
static int noalloc_ctx_id(unsigned long long *id)
{
    *id = 0;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return GIC_ERR_CUDA;
    if (!ctx) return GIC_OK;
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return GIC_ERR_CUDA;
    return GIC_OK;
}

static int noalloc_address(cudaStream_t s, NoallocScratch **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_pfn_tried) {
        g_noalloc_pfn_tried = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2) {
            g_ctx_get_current = (PfnCtxGetCurrent)f1;
            g_ctx_get_id = (PfnCtxGetId)f2;
            g_noalloc_pfn_ok = true;
        }
    }
    if (!g_noalloc_pfn_ok) return GIC_ERR_UNSUPPORTED;
    unsigned long long id = 0;
    GIC_TRY(noalloc_ctx_id(&id));
    if (id != 0) {
        for (int k = 0; k < NOALLOC_CACHE; ++k)
            if (g_noalloc_cache[k].ctx_id == id) {
                *out = g_noalloc_cache[k].addr;
                return GIC_OK;
            }
    }
    // first call in this context: the look-up is not made while the stream
    // is being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GIC_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return GIC_ERR_UNSUPPORTED;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    if (id == 0) GIC_TRY(noalloc_ctx_id(&id)); // the runtime made its context current just now
    if (id == 0) return GIC_ERR_CUDA;
    g_noalloc_cache[g_noalloc_next] = {id, (NoallocScratch *)ptr};
    g_noalloc_next = (g_noalloc_next + 1) % NOALLOC_CACHE;
    *out = (NoallocScratch *)ptr;
    return GIC_OK;
}

}  // namespace gic

extern "C" int gic_spmv_dot_noalloc(int64_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                                    const double *x, double *y, double *xdoty, void *stream)
{
    if (n < 1 || !rowptr || !col || !val || !x || !y || !xdoty) return GIC_ERR_INVALID_ARG;
    if (n > gic::NOALLOC_MAX_ROWS) return GIC_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    gic::NoallocScratch *scr = nullptr;
    GIC_TRY(gic::noalloc_address(s, &scr));
    int device = 0, sms = 0;
    GIC_CUDA_TRY(cudaGetDevice(&device));
    GIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    // the reduction counter must start at zero, whatever an earlier call left
    GIC_CUDA_TRY(cudaMemsetAsync(&scr->sc, 0, sizeof(gic::Scalars), s));
    // 8 warps per block, one row per warp per pass; the grid strides over the
    // rows, so it is capped at 8 blocks per SM (that also keeps the last
    // block's sum over the per-block partials short)
    int64_t blocks = (n + 7) / 8;
    const int64_t cap = 8 * (int64_t)(sms > 0 ? sms : 1);
    if (blocks > cap) blocks = cap;
    if (blocks > gic::NOALLOC_SLOTS) blocks = gic::NOALLOC_SLOTS;
    gic::k_spmv<0><<<(unsigned)blocks, gic::SPMV_BLOCK, 0, s>>>(n, rowptr, col, val, x, y, nullptr, scr->partials,
                                                                xdoty, &scr->sc);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}
