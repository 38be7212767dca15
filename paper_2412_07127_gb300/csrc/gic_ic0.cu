// gic_ic0.cu -- A3: IC(0) on the device.
//
// IC(0) (Introduction; Baseline Methods; Supplementary 2) computes L on the
// pattern of tril(A):
//   L_ij = (a_ij - sum_{k<j} L_ik L_jk) / L_jj  (j < i),
//   L_ii = sqrt(a_ii' - sum_{k<i} L_ik^2),  a_ii' = a_ii + alpha a_ii,
// with k over the pattern. Row i depends on the rows of its strictly-lower
// columns, the same DAG as the forward solve, so it uses the same
// schedule: one warp per group of rows with identical patterns, groups dealt
// round-robin to a co-resident grid, readiness = the row's diagonal entry
// (stored last, with release semantics, over a sentinel).
//
// Per group (rows s..s+G-1, shared external columns J[0..m)):
//   1. wait for the rows J[u], then gather M[u][v] = L_{J[u],J[v]} (v <= u)
//      into shared memory, row group by row group (the rows of a group share
//      their external columns, so each is looked up once);
//   2. the external part of every group row solves the same lower-triangular
//      system M l = a_J, so all G rows are swept together, column by column
//      in ascending order (the order of the sum above);
//   3. the in-group columns and the diagonal of each row follow in order;
//      the group's rows are published together (one fence).
// A pivot <= 0 or non-finite records the smallest such row (atomicMin), and
// the row publishes NaN so its dependants finish instead of waiting.
#include <limits.h>
#include <math.h>

#include "gic_internal.cuh"

namespace gic {

constexpr int IC_WARPS = 3; // warps per block (the general variant fits 5 such blocks per SM, the hex-sized one 8)

// Packed column-major lower triangle of an MD x MD block: column v holds
// rows v..MD-1 (the sweep reads a column across lanes, consecutive words,
// conflict-free); half the shared memory of the full square, so more warps
// fit per SM. The kernel is built for two sizes: external widths up to 40
// and groups up to 3 rows (hex elasticity: 39 and 3; ~9 KB per warp, 24
// warps per SM) and the general MAXDIM / GMAX.
template <int MD>
__device__ __forceinline__ int pm(int v, int u) { return v * MD - (v * (v - 1)) / 2 + (u - v); }

template <int MD, int GM>
struct IcWarpSmem {
    double M[MD * (MD + 1) / 2]; // lower triangle of the external block, M[pm(v, u)] = M[u][v], u >= v
    double invd[MD];         // 1 / M[v][v]
    double lg[GM][MD];     // external part of each group row
    double lin[GM][GM + 1];  // in-group part (and diagonal) of each group row
    int32_t J[MD];
    int32_t rs[MD];          // start of row J[u] in L
    int32_t len[MD];         // length of row J[u] in L (its diagonal included)
    // J holds whole row groups (rows of a group are identical in A, which is
    // symmetric), and a group's rows share their external columns: blocks
    int32_t bu0[MD];         // first u of block b
    int32_t bG[MD];          // rows of block b
    int32_t boff[MD + 1];    // prefix of the blocks' external lengths
    int nb;
    double dd[6];                // the group's dot products l_t . l_q, q <= t (G <= 3)
    double ain[6];               // the group's in-group entries of A, (t, q <= t) at t(t+1)/2 + q (G <= 3)
};

__device__ __forceinline__ int find_in(const int32_t *J, int lo, int hi, int32_t key)
{
    // index of key in sorted J[lo,hi), or -1
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int32_t v = J[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

template <int MD, int GM>
__global__ void __launch_bounds__(IC_WARPS * 32) k_ic0(int32_t nchunks, const int32_t *__restrict__ ord,
                                                       const int32_t *__restrict__ chunk_grp,
                                                       const int32_t *__restrict__ grp,
                                                       const int32_t *__restrict__ rowgrp,
                                                       const int32_t *__restrict__ Arowptr,
                                                       const double *__restrict__ valA,
                                                       const int32_t *__restrict__ Lrowptr,
                                                       const int32_t *__restrict__ Lcol, double *Lval,
                                                       double alpha, unsigned long long *bad_row, unsigned *err,
                                                       int poll)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    IcWarpSmem<MD, GM> &S = reinterpret_cast<IcWarpSmem<MD, GM> *>(smem_raw)[wib];
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);

    for (int64_t pos = w; pos < nchunks; pos += nw) {
      // chunks of consecutive groups, or (chunk_grp null) single groups
      const int32_t ch = ord[pos];
      const int32_t g0 = chunk_grp ? chunk_grp[ch] : ch, g1 = chunk_grp ? chunk_grp[ch + 1] : ch + 1;
      for (int32_t g = g0; g < g1; ++g) {
        const int32_t s = grp[g];
        const int G = grp[g + 1] - s;
        const int32_t b0 = Lrowptr[s];
        const int m = Lrowptr[s + 1] - b0 - 1; // external columns (host checked m <= MD)

        // 1. external columns, their readiness (relaxed polling, one fence
        // after the last wait), their row starts and lengths, and the blocks
        // (row groups) they form
        int32_t dp0 = -1, dp1 = -1;
        bool st0 = false, st1 = false;
        for (int u = lane; u < m; u += 32) {
            int32_t j = Lcol[b0 + u];
            S.J[u] = j;
            const int32_t rs = Lrowptr[j];
            const int32_t dpos = Lrowptr[j + 1] - 1;
            S.rs[u] = rs;
            S.len[u] = dpos + 1 - rs;
            const bool st = (u == 0) || (rowgrp[j] == j);
            if (u < 32) { dp0 = dpos; st0 = st; } else { dp1 = dpos; st1 = st; }
        }
        if (G <= 3 && lane < G * (G + 1) / 2) { // read now, used after the sweep
            int tt = 0;
            while ((tt + 1) * (tt + 2) / 2 <= lane) ++tt;
            const int qq = lane - tt * (tt + 1) / 2;
            S.ain[lane] = valA[(int64_t)Arowptr[s + tt] + m + qq];
        }
        const unsigned long long bits =
            (unsigned long long)__ballot_sync(0xffffffffu, st0) | ((unsigned long long)__ballot_sync(0xffffffffu, st1) << 32);
        {   // one lane at a time polls the diagonal written last
            double d0 = (dp0 >= 0) ? ld_relaxed(Lval + dp0) : 0.0;
            double d1 = (dp1 >= 0) ? ld_relaxed(Lval + dp1) : 0.0;
            wait_deps<true>(Lval, dp0, dp1, d0, d1, err, poll);
        }
        __syncwarp();
        fence_acq_rel(); // pairs with the producers' release of each diagonal
        for (int u = lane; u < m; u += 32) {
            if ((bits >> u) & 1ull) {
                const int b = __popcll(bits & ((1ull << u) - 1ull));
                const unsigned long long rest = (u + 1 < 64) ? (bits >> (u + 1)) : 0ull;
                const int u1 = rest ? u + __ffsll((long long)rest) : m;
                S.bu0[b] = u;
                S.bG[b] = u1 - u;
                S.boff[b + 1] = S.len[u] - 1; // the block's first row: every entry but the diagonal is external
            }
        }
        __syncwarp();
        if (lane == 0) {
            const int nb = __popcll(bits);
            S.nb = nb;
            S.boff[0] = 0;
            for (int b = 0; b < nb; ++b) S.boff[b + 1] += S.boff[b];
        }
        for (int idx = lane; idx < pm<MD>(m, m); idx += 32) S.M[idx] = 0.0; // columns 0..m-1
        __syncwarp();

        // 1 / L_{J[v],J[v]} (the last entry of row J[v]) first: the gather
        // stores each column already scaled by it, so the sweep's dependent
        // step is one shuffle and one FMA with no multiply per column
        for (int u = lane; u < m; u += 32) S.invd[u] = 1.0 / Lval[S.rs[u] + S.len[u] - 1];
        __syncwarp();
        // gather M[u][v] / M[v][v] = L_{J[u],J[v]} / L_{J[v],J[v]} (v < u)
        // block by block: a block's external column is looked up in J once
        // for all its rows; four (column, values) reads in flight per lane
        const int nb = S.nb, PT = S.boff[nb];
        int bcur = 0;
        for (int base = lane; base < PT; base += 128) {
            int bb[4], pp[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int idx = base + 32 * k;
                if (idx < PT) {
                    while (S.boff[bcur + 1] <= idx) ++bcur;
                    bb[k] = bcur;
                    pp[k] = idx - S.boff[bcur];
                } else {
                    bb[k] = -1;
                    pp[k] = 0;
                }
            }
            int32_t cc[4];
            double vv[4][3];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cc[k] = -1;
                if (bb[k] >= 0) {
                    const int u0 = S.bu0[bb[k]], gb = S.bG[bb[k]];
                    cc[k] = Lcol[S.rs[u0] + pp[k]];
#pragma unroll
                    for (int r = 0; r < 3; ++r) vv[k][r] = (r < gb) ? Lval[S.rs[u0 + r] + pp[k]] : 0.0;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (bb[k] < 0) continue;
                const int u0 = S.bu0[bb[k]], gb = S.bG[bb[k]];
                const int v = find_in(S.J, 0, u0, cc[k]);
                if (v < 0) continue;
                const double iv = S.invd[v];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    if (r < gb) S.M[pm<MD>(v, u0 + r)] = vv[k][r] * iv;
                for (int r = 3; r < gb; ++r) S.M[pm<MD>(v, u0 + r)] = Lval[S.rs[u0 + r] + pp[k]] * iv;
            }
        }
        // the blocks' own strictly lower triangles (in-group entries), scaled
        // the same way
        for (int b = lane; b < nb; b += 32) {
            const int u0 = S.bu0[b], gb = S.bG[b], me = S.boff[b + 1] - S.boff[b];
            for (int r = 1; r < gb; ++r)
                for (int q2 = 0; q2 < r; ++q2)
                    S.M[pm<MD>(u0 + q2, u0 + r)] = Lval[S.rs[u0 + r] + me + q2] * S.invd[u0 + q2];
        }
        __syncwarp();

        // 2. external parts of all group rows: forward sweep over v ascending.
        // Lane owns columns u = lane and lane + 32 of every row.
        double acc0[GM], acc1[GM];
#pragma unroll
        for (int t = 0; t < GM; ++t) {
            acc0[t] = 0.0;
            acc1[t] = 0.0;
            if (t < G) {
                int64_t ab = Arowptr[s + t];
                if (lane < m) acc0[t] = valA[ab + lane];
                if (lane + 32 < m) acc1[t] = valA[ab + lane + 32];
            }
        }
        // Column v's accumulator is final once the sweep reaches it, so each
        // step broadcasts it unscaled and the lanes apply their coefficient,
        // stored already divided by M[v][v]: the dependent chain per step is
        // one shuffle and one FMA; the values l = acc / M[v][v] are formed
        // once at the end.
        for (int v = 0; v < m; ++v) {
            const int owner = v & 31;
            const double mu0 = (lane > v && lane < m) ? S.M[pm<MD>(v, lane)] : 0.0;
            const double mu1 = (lane + 32 > v && lane + 32 < m) ? S.M[pm<MD>(v, lane + 32)] : 0.0;
#pragma unroll
            for (int t = 0; t < GM; ++t) {
                if (t < G) {
                    const double a = __shfl_sync(0xffffffffu, (v < 32) ? acc0[t] : acc1[t], owner);
                    acc0[t] = fma(-mu0, a, acc0[t]);
                    acc1[t] = fma(-mu1, a, acc1[t]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < GM; ++t) {
            if (t < G) {
                if (lane < m) S.lg[t][lane] = acc0[t] * S.invd[lane];
                if (lane + 32 < m) S.lg[t][lane + 32] = acc1[t] * S.invd[lane + 32];
            }
        }
        __syncwarp();

        // 3. in-group columns and diagonals: the group's dot products
        // l_t . l_q (q <= t) first (for G <= 3 all six at once, so their
        // warp reductions overlap), then the small dense Cholesky in lane 0
        if (G <= 3) {
            double d[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}; // (t, q): 00, 10, 11, 20, 21, 22
            for (int v = lane; v < m; v += 32) {
                const double l0 = S.lg[0][v], l1 = (G > 1) ? S.lg[1][v] : 0.0, l2 = (G > 2) ? S.lg[2][v] : 0.0;
                d[0] = fma(l0, l0, d[0]);
                d[1] = fma(l1, l0, d[1]);
                d[2] = fma(l1, l1, d[2]);
                d[3] = fma(l2, l0, d[3]);
                d[4] = fma(l2, l1, d[4]);
                d[5] = fma(l2, l2, d[5]);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) d[k] = warp_sum(d[k]);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) S.dd[k] = d[k];
                for (int t = 0; t < G; ++t) {
                    for (int q = 0; q < t; ++q) {
                        double x = S.ain[t * (t + 1) / 2 + q] - S.dd[t * (t + 1) / 2 + q];
                        for (int q2 = 0; q2 < q; ++q2) x = fma(-S.lin[t][q2], S.lin[q][q2], x);
                        S.lin[t][q] = x / S.lin[q][q];
                    }
                    const double a = S.ain[t * (t + 1) / 2 + t];
                    double x = __dadd_rn(a, __dmul_rn(alpha, a)) - S.dd[t * (t + 1) / 2 + t];
                    for (int q = 0; q < t; ++q) x = fma(-S.lin[t][q], S.lin[t][q], x);
                    double piv;
                    if (!(x > 0.0) || !isfinite(x)) {
                        atomicMin(bad_row, (unsigned long long)(s + t));
                        piv = qnan;
                    } else {
                        piv = sqrt(x);
                    }
                    S.lin[t][t] = piv;
                }
            }
        } else {
            for (int t = 0; t < G; ++t) {
                const int64_t ab = Arowptr[s + t];
                // in-group column s+q (q < t): (a_{i,s+q} - l_t . l_q - sum_{q'<q}) / L_{s+q,s+q}
                for (int q = 0; q < t; ++q) {
                    double d = 0.0;
                    for (int v = lane; v < m; v += 32) d = fma(S.lg[t][v], S.lg[q][v], d);
                    d = warp_sum(d);
                    if (lane == 0) {
                        double x = valA[ab + m + q] - d;
                        for (int q2 = 0; q2 < q; ++q2) x = fma(-S.lin[t][q2], S.lin[q][q2], x);
                        S.lin[t][q] = x / S.lin[q][q];
                    }
                    __syncwarp();
                }
                double d = 0.0;
                for (int v = lane; v < m; v += 32) d = fma(S.lg[t][v], S.lg[t][v], d);
                d = warp_sum(d);
                if (lane == 0) {
                    const double a = valA[ab + m + t];
                    double x = __dadd_rn(a, __dmul_rn(alpha, a)) - d;
                    for (int q = 0; q < t; ++q) x = fma(-S.lin[t][q], S.lin[t][q], x);
                    double piv;
                    if (!(x > 0.0) || !isfinite(x)) {
                        atomicMin(bad_row, (unsigned long long)(s + t));
                        piv = qnan;
                    } else {
                        piv = sqrt(x);
                    }
                    S.lin[t][t] = piv;
                }
                __syncwarp();
            }
        }
        __syncwarp();
        // publish the group: every off-diagonal entry, one fence, then each
        // row's diagonal with release (the readiness word)
        for (int t = 0; t < G; ++t) {
            const int64_t lb = Lrowptr[s + t];
            for (int v = lane; v < m; v += 32) Lval[lb + v] = S.lg[t][v];
            if (lane < t) Lval[lb + m + lane] = S.lin[t][lane];
        }
        __threadfence();
        __syncwarp();
        if (lane < G) st_release(Lval + Lrowptr[s + lane] + m + lane, S.lin[lane][lane]);
        __syncwarp();
      }
    }
}

__global__ void k_ic0_prepare(int64_t n, const int32_t *Lrowptr, double *Lval, unsigned long long *bad_row)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        Lval[Lrowptr[i + 1] - 1] = sentinel_d();
    if (blockIdx.x == 0 && threadIdx.x == 0) *bad_row = ULLONG_MAX;
}

int launch_persistent(gic_handle *h, const void *fn, int block, size_t smem, int64_t warps_needed, void **args);

static int ic0_once(gic_handle *h, const Pattern &P, const double *valA, double *valL, double alpha, int64_t *bad)
{
    if (P.max_ext_lower > MAXDIM || P.max_group > GMAX) return GIC_ERR_UNSUPPORTED;
    unsigned long long *bad_dev = (unsigned long long *)((char *)h->dev_small + 60000);
    int64_t blocks = (P.n + 255) / 256;
    if (blocks > (int64_t)h->num_sms * 8) blocks = (int64_t)h->num_sms * 8;
    ++h->launches;
    k_ic0_prepare<<<(unsigned)blocks, 256, 0, h->stream>>>(P.n, P.Lrowptr, valL, bad_dev);
    GIC_CUDA_TRY(cudaGetLastError());
    const bool small = P.max_ext_lower <= 40 && P.max_group <= 3;
    const void *fn = small ? (const void *)k_ic0<40, 3> : (const void *)k_ic0<MAXDIM, GMAX>;
    size_t smem = (small ? sizeof(IcWarpSmem<40, 3>) : sizeof(IcWarpSmem<MAXDIM, GMAX>)) * IC_WARPS;
    // set on every call (a host-side attribute of the current context; cheap)
    GIC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // single groups in group-level order where the analysis made that order
    // (warps take the next ready group instead of walking a whole chunk)
    int32_t nc = P.ic_ord ? P.ngroups : P.nchunks;
    const int32_t *ord = P.ic_ord ? P.ic_ord : P.ord_f, *cg = P.ic_ord ? nullptr : P.chunk_grp, *g = P.grp,
                  *rg = P.rowgrp, *ar = P.rowptr, *lr = P.Lrowptr, *lc = P.Lcol;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&nc, &ord, &cg, &g, &rg, &ar, &valA, &lr, &lc, &valL, &alpha, &bad_dev, &er, &poll};
    GIC_TRY(launch_persistent(h, fn, IC_WARPS * 32, smem, nc, args));
    unsigned long long *hb = (unsigned long long *)((char *)h->host_pinned + 2048);
    GIC_CUDA_TRY(cudaMemcpyAsync(hb, bad_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    unsigned flags = 0;
    GIC_TRY(read_and_clear_dev_err(h, &flags)); // synchronises
    if (flags & ERR_TIMEOUT) return GIC_ERR_TIMEOUT;
    *bad = (*hb == ULLONG_MAX) ? -1 : (int64_t)*hb;
    return (*bad >= 0) ? GIC_ERR_NOT_SPD : GIC_OK;
}

}  // namespace gic

using namespace gic;

extern "C" {

int gic_ic0(gic_handle *h, const gic_pattern *P, const double *valA, double *valL, double alpha, int64_t *bad_row)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device || !valA || !valL || !(alpha >= 0.0)) return GIC_ERR_INVALID_ARG;
    int64_t bad = -1;
    int rc = ic0_once(h, P->p, valA, valL, alpha, &bad);
    if (bad_row) *bad_row = bad;
    return rc;
}

int gic_ic0_auto(gic_handle *h, const gic_pattern *P, const double *valA, double *valL, int max_tries,
                 double *alpha_out, int64_t *bad_row)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device || !valA || !valL || max_tries < 0) return GIC_ERR_INVALID_ARG;
    double alpha = 0.0;
    int64_t bad = -1;
    int rc = GIC_ERR_NOT_SPD;
    for (int t = 0; t <= max_tries; ++t) {
        rc = ic0_once(h, P->p, valA, valL, alpha, &bad);
        if (rc != GIC_ERR_NOT_SPD) break;
        alpha = (t == 0) ? 1e-3 : 2.0 * alpha;
    }
    if (alpha_out) *alpha_out = (rc == GIC_OK) ? alpha : alpha;
    if (bad_row) *bad_row = bad;
    return rc;
}

}  // extern "C"
