// gic_bsolve.cu -- A7b: SM-local sync-free triangular solves.
//
// The sweep's dependency chain crosses one row level per step (Eq. (11),
// forward y_i = (r_i - sum_{j<i} L_ij y_j) / L_ii and its backward
// counterpart), and for the hex-element systems every node level depends on
// nodes of neighbouring pencils. When those pencils run on other SMs each
// level costs an L2 round trip. Here a CTA owns a block of BCHUNKS
// consecutive chunks (neighbouring pencils), one warp per chunk, and keeps a
// shared-memory mirror of every row the block produces: a dependency inside
// the block is read (and waited for) in shared memory, only dependencies on
// other blocks go through global memory. Blocks run in an order where every
// cross-block dependency points to an earlier block, so the earliest
// unfinished block can always progress.
//
// Per group (rows s..s+G-1, G <= 3) the warp uses the premultiplied blocks of
// q_setup (K = M L_ext, M = D^-1): with positions p < mx the group's
// external columns other than the previous group's, and mx <= p < mx + G its
// own right-hand side, every lane forms its share of
//     a_t = sum_p K_tp v_p - sum_u M_tu rr_u,
// the warp reduces the three sums, and lanes t < G finish
//     y_t = -a_t - sum_{prev} K_tj y_prev_j
// from the previous group's values held in registers. A group's static data
// (columns, coefficients, right-hand side) is loaded one group ahead, and its
// dependency values are read before the previous group is reduced and
// published, so only values still missing then cost a further round trip.
// Readiness is the value itself (signalling-NaN sentinel), in global and in
// shared memory; every wait is bounded.
#include <limits.h>
#include <math.h>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int BS_THREADS = BCHUNKS * 32;
constexpr unsigned BFULL = 0xffffffffu;

template <typename T>
struct GStat {
    int32_t s, cw;      // first row, packed counts (warp-uniform)
    int32_t c0, c1;     // dependency columns of positions lane, lane + 32 (-1: none)
    T k0[3], k1[3];     // their coefficients for rows 0..2
    T w0, w1;           // value of a right-hand-side position
    T kp[3];            // lanes t < G: coefficients of the previous group's columns
    int32_t pc[3];      // ... and those columns
    double rdv;         // lanes t < G: r in FP64 (backward sweep with PCG)
};

template <typename T, bool FWD, bool PCG>
__device__ __forceinline__ void b_load(GStat<T> &S, int32_t s, int32_t cw, int32_t b0, const int32_t *qcol,
                                       const T *Kv, const T *rhs, const double *rd, int lane)
{
    const int ne = cw & 255, nl = (cw >> 8) & 255, np = (cw >> 16) & 255, G = cw >> 24;
    const int m = ne + nl + np, mx = ne + nl;
    S.s = s;
    S.cw = cw;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int p = lane + 32 * i, u = p - mx;
        const bool dep = p < mx, own = u >= 0 && u < G;
        const int32_t c = dep ? qcol[b0 + p] : -1;
        T k[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            T v = (T)0;
            if (t < G) {
                if (dep) v = Kv[b0 + (int64_t)t * m + p];
                else if (own && (FWD ? u <= t : u >= t))
                    v = -Kv[b0 + (int64_t)G * m + (FWD ? t * (t + 1) / 2 + u : u * (u + 1) / 2 + t)];
            }
            k[t] = v;
        }
        const T w = own ? rhs[s + u] : (T)0;
        if (i == 0) {
            S.c0 = c;
            S.w0 = w;
#pragma unroll
            for (int t = 0; t < 3; ++t) S.k0[t] = k[t];
        } else {
            S.c1 = c;
            S.w1 = w;
#pragma unroll
            for (int t = 0; t < 3; ++t) S.k1[t] = k[t];
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const bool have = lane < G && j < np;
        S.kp[j] = have ? Kv[b0 + (int64_t)lane * m + mx + j] : (T)0;
        S.pc[j] = have ? qcol[b0 + mx + j] : 0;
    }
    S.rdv = (PCG && lane < G) ? rd[s + lane] : 0.0;
}

// bounded wait on a shared-memory word
template <typename T>
__device__ __forceinline__ T smem_wait(const T *p, unsigned *err)
{
    const volatile T *q = (const volatile T *)p;
    T v = *q;
    if (!is_sentinel(v)) return v;
    for (long long it = 0; it < SPIN_LIMIT; ++it) {
        v = *q;
        if (!is_sentinel(v)) return v;
        if ((it & 1023) == 1023) {
            if (*((volatile unsigned *)err) != 0u) return qnan_of<T>();
            __nanosleep(32);
        }
    }
    atomicOr(err, ERR_TIMEOUT);
    return qnan_of<T>();
}

// one read of a dependency (shared mirror or global), possibly the sentinel
template <typename T>
__device__ __forceinline__ T b_peek(int32_t c, const T *x, const T *mirror, int32_t lo, int32_t hi)
{
    if (c >= lo && c < hi) return ((const volatile T *)mirror)[c - lo];
    return ld_relaxed(x + c);
}

template <typename T>
__device__ __forceinline__ T b_fetch(int32_t c, const T *x, const T *mirror, int32_t lo, int32_t hi, unsigned *err)
{
    if (c >= lo && c < hi) return smem_wait<T>(mirror + (c - lo), err);
    T v = ld_relaxed(x + c);
    if (!is_sentinel(v)) return v;
    return wait_word(x + c, err, 0);
}

template <typename T, bool FWD, bool PCG>
__device__ __forceinline__ void b_chunk(int32_t g0, int32_t g1, const int32_t *grp, const int32_t *rowptr,
                                        const int32_t *qcol, const int32_t *qcnt, const T *Kv, const T *rhs, T *x,
                                        T *yreset, const double *rd, T *mirror, int32_t lo, int32_t hi,
                                        unsigned *err, int lane, double &dot)
{
    const int cnt = g1 - g0;
    int32_t hs = 0, hc = 0, hb = 0; // headers of 32 groups, one per lane
    int wbase = -64;
    auto header = [&](int k, int32_t &s, int32_t &cw, int32_t &b0) {
        if (k - wbase >= 32) {
            wbase = k;
            const int kk = k + lane;
            if (kk < cnt) {
                const int32_t g = FWD ? g0 + kk : g1 - 1 - kk;
                hs = grp[g];
                hc = qcnt[g];
                hb = rowptr[hs];
            }
        }
        s = __shfl_sync(BFULL, hs, k - wbase);
        cw = __shfl_sync(BFULL, hc, k - wbase);
        b0 = __shfl_sync(BFULL, hb, k - wbase);
    };
    GStat<T> cur, nxt;
    {
        int32_t s, cw, b0;
        header(0, s, cw, b0);
        b_load<T, FWD, PCG>(cur, s, cw, b0, qcol, Kv, rhs, rd, lane);
    }
    // dependency values of the current group, loaded before the previous
    // group is published (may still be the sentinel: re-polled when used)
    T v0 = (cur.c0 >= 0) ? b_peek<T>(cur.c0, x, mirror, lo, hi) : cur.w0;
    T v1 = (cur.c1 >= 0) ? b_peek<T>(cur.c1, x, mirror, lo, hi) : cur.w1;
    T p0 = 0, p1 = 0, p2 = 0; // the previous group's values
    int32_t prev_s = 0;
    for (int k = 0; k < cnt; ++k) {
        if (k + 1 < cnt) {
            int32_t s, cw, b0;
            header(k + 1, s, cw, b0);
            b_load<T, FWD, PCG>(nxt, s, cw, b0, qcol, Kv, rhs, rd, lane);
        }
        const int ne = cur.cw & 255, nl = (cur.cw >> 8) & 255, np = (cur.cw >> 16) & 255, G = cur.cw >> 24;
        const int mx = ne + nl;
        const bool two = mx + G > 32; // uniform
        if (cur.c0 >= 0 && is_sentinel(v0)) v0 = b_fetch<T>(cur.c0, x, mirror, lo, hi, err);
        if (two && cur.c1 >= 0 && is_sentinel(v1)) v1 = b_fetch<T>(cur.c1, x, mirror, lo, hi, err);
        T a[3];
        if (two) {
#pragma unroll
            for (int t = 0; t < 3; ++t) a[t] = fma(cur.k1[t], v1, cur.k0[t] * v0);
        } else {
#pragma unroll
            for (int t = 0; t < 3; ++t) a[t] = cur.k0[t] * v0;
        }
        // the next group's dependencies other than this group: in flight
        // while this group is reduced and published
        if (k + 1 < cnt) {
            v0 = (nxt.c0 >= 0) ? b_peek<T>(nxt.c0, x, mirror, lo, hi) : nxt.w0;
            v1 = (nxt.c1 >= 0) ? b_peek<T>(nxt.c1, x, mirror, lo, hi) : nxt.w1;
        }
        warp_sum_n<T, 3>(a, lane);
        T yv = 0;
        if (lane < G) {
            yv = -pick3<T>(lane, a[0], a[1], a[2]);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < np) yv = fma(-cur.kp[j], pick3<T>(cur.pc[j] - prev_s, p0, p1, p2), yv);
            const int32_t row = cur.s + lane;
            st_relaxed(x + row, yv);
            ((volatile T *)mirror)[row - lo] = yv;
            if (PCG) {
                yreset[row] = sentinel_of<T>();
                dot = fma(cur.rdv, (double)yv, dot);
            }
        }
        p0 = __shfl_sync(BFULL, yv, 0);
        p1 = __shfl_sync(BFULL, yv, 1);
        p2 = __shfl_sync(BFULL, yv, 2);
        prev_s = cur.s;
        cur = nxt;
    }
}

// FWD: L y = r (x = y, rhs = r). Backward: L^T z = y (x = z, rhs = y); with
// PCG it resets y to the sentinel for the next forward sweep and forms
// r^T z in FP64, then beta (Algorithm 1) in the last warp to finish. x must
// hold the sentinel.
template <typename T, bool FWD, bool PCG>
__global__ void __launch_bounds__(BS_THREADS, 1) k_bsolve(int32_t nchunks, int32_t ncb, const int32_t *__restrict__ cb_ord,
                                                          const int32_t *__restrict__ chunk_grp,
                                                          const int32_t *__restrict__ grp,
                                                          const int32_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ qcol,
                                                          const int32_t *__restrict__ qcnt, const T *__restrict__ Kv,
                                                          const T *rhs, T *x, T *yreset, const double *__restrict__ rd,
                                                          double *partials, unsigned *err, Scalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) unsigned char b_raw[];
    T *mirror = reinterpret_cast<T *>(b_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double dot = 0.0;
    for (int32_t bi = blockIdx.x; bi < ncb; bi += gridDim.x) {
        const int32_t cb = cb_ord[bi];
        const int32_t c0 = cb * BCHUNKS, c1 = min(c0 + BCHUNKS, nchunks);
        const int32_t lo = grp[chunk_grp[c0]], hi = grp[chunk_grp[c1]];
        for (int32_t i = threadIdx.x; i < hi - lo; i += blockDim.x) mirror[i] = sentinel_of<T>();
        __syncthreads();
        const int32_t c = c0 + w;
        if (c < c1)
            b_chunk<T, FWD, PCG>(chunk_grp[c], chunk_grp[c + 1], grp, rowptr, qcol, qcnt, Kv, rhs, x, yreset,
                                 PCG ? rd : nullptr, mirror, lo, hi, err, lane, dot);
        __syncthreads();
    }
    if (PCG) {
        dot = warp_sum(dot);
        const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        if (lane == 0) partials[wg] = dot;
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence();
            last = (atomicAdd(&sc->counter, 1u) == (unsigned)nw - 1u);
        }
        last = __shfl_sync(BFULL, last, 0);
        if (last) {
            __threadfence();
            const double rz = warp_sum_partials(partials, (int)nw);
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

template <typename T, bool FWD, bool PCG>
static int b_launch(gic_handle *h, const Pattern &P, const T *Kv, const T *rhs, T *x, T *yreset, const double *rd,
                    double *partials, Scalars *sc)
{
    if (!P.bready) return GIC_ERR_UNSUPPORTED;
    int32_t nc = P.nchunks, ncb = P.ncb;
    const int32_t *ord = FWD ? P.cb_ord_f : P.cb_ord_b, *cg = P.chunk_grp, *g = P.grp;
    const int32_t *rp = FWD ? P.Lrowptr : P.Urowptr;
    const int32_t *qc = FWD ? P.qf_col : P.qb_col, *qn = FWD ? P.qf_cnt : P.qb_cnt;
    unsigned *er = h->dev_err;
    void *args[] = {&nc, &ncb, &ord, &cg, &g, &rp, &qc, &qn, &Kv, &rhs, &x, &yreset, &rd, &partials, &er, &sc};
    const size_t smem = sizeof(T) * (size_t)(P.mirror_rows > 0 ? P.mirror_rows : 1);
    static size_t ad[64] = {};
    if (ad[h->device & 63] < smem) {
        GIC_CUDA_TRY(cudaFuncSetAttribute(k_bsolve<T, FWD, PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        ad[h->device & 63] = smem;
    }
    int64_t need = (int64_t)ncb * BCHUNKS; // warps
    if (PCG && need > MAX_PARTIALS) need = MAX_PARTIALS;
    return launch_persistent(h, (const void *)k_bsolve<T, FWD, PCG>, BS_THREADS, smem, need, args);
}

int b_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Kf, const void *r, void *y, const Scalars *sc)
{
    Scalars *s = const_cast<Scalars *>(sc);
    if (f32)
        return b_launch<float, true, false>(h, P, (const float *)Kf, (const float *)r, (float *)y, nullptr, nullptr,
                                            nullptr, s);
    return b_launch<double, true, false>(h, P, (const double *)Kf, (const double *)r, (double *)y, nullptr, nullptr,
                                         nullptr, s);
}

int b_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Kb, void *y, void *z,
              const double *rd, double *partials, Scalars *sc)
{
    if (f32) {
        if (pcg)
            return b_launch<float, false, true>(h, P, (const float *)Kb, (const float *)y, (float *)z, (float *)y, rd,
                                                partials, sc);
        return b_launch<float, false, false>(h, P, (const float *)Kb, (const float *)y, (float *)z, nullptr, nullptr,
                                             nullptr, sc);
    }
    if (pcg)
        return b_launch<double, false, true>(h, P, (const double *)Kb, (const double *)y, (double *)z, (double *)y, rd,
                                             partials, sc);
    return b_launch<double, false, false>(h, P, (const double *)Kb, (const double *)y, (double *)z, nullptr, nullptr,
                                          nullptr, sc);
}

}  // namespace gic
