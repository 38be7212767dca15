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
// (columns, coefficients, right-hand side) is staged in shared memory by
// cp.async two groups ahead, and its dependency values are read before the
// previous group is reduced and published, so only values still missing
// then cost a further round trip.
// Readiness is the value itself (signalling-NaN sentinel), in global and in
// shared memory; every wait is bounded.
#include <limits.h>
#include <math.h>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int BS_THREADS = BCHUNKS * 32;
constexpr unsigned BFULL = 0xffffffffu;

// a group's static data staged in shared memory (cp.async)
template <typename T>
struct BSlot {
    T K[3][QCOL];      // premultiplied coefficients, columns [early | late | prev]
    T Mv[6];           // M = D^-1 packed (t, u <= t)
    T rr[3];           // right-hand side rows
    double rd[3];      // backward with PCG: r in FP64
    int32_t cols[QCOL];
    int32_t s, cw;
};
constexpr int BRING = 3; // slots per warp: the current group and two ahead

template <typename T>
__device__ __forceinline__ void b_stage(BSlot<T> &S, int32_t s, int32_t cw, int64_t b0, const int32_t *qcol,
                                        const T *Kv, const T *rhs, const double *rd, int lane)
{
    const int m = (cw & 255) + ((cw >> 8) & 255) + ((cw >> 16) & 255), G = cw >> 24;
    if (lane == 0) {
        S.s = s;
        S.cw = cw;
    }
    if (lane < m) cp_async_4(&S.cols[lane], qcol + b0 + lane);
    if (lane + 32 < m) cp_async_4(&S.cols[lane + 32], qcol + b0 + lane + 32);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        if (t < G) {
            const T *row = Kv + b0 + (int64_t)t * m;
            if (lane < m) cp_async_t(&S.K[t][lane], row + lane);
            if (lane + 32 < m) cp_async_t(&S.K[t][lane + 32], row + lane + 32);
        }
    }
    if (lane < G * (G + 1) / 2) cp_async_t(&S.Mv[lane], Kv + b0 + (int64_t)G * m + lane);
    if (lane < G) cp_async_t(&S.rr[lane], rhs + s + lane);
    if (rd && lane < G) cp_async_8(&S.rd[lane], rd + s + lane);
}

// coefficient and value of position p of a staged group: p < mx a
// dependency column (K, value loaded separately), mx <= p < mx + G the
// group's own right-hand side (-M, rr)
template <typename T, bool FWD>
__device__ __forceinline__ T b_coef(const BSlot<T> &S, int t, int p, int mx, int G)
{
    if (t >= G) return (T)0;
    if (p < mx) return S.K[t][p];
    const int u = p - mx;
    if (u >= G) return (T)0;
    if (FWD) return (u <= t) ? -S.Mv[t * (t + 1) / 2 + u] : (T)0;
    return (u >= t) ? -S.Mv[u * (u + 1) / 2 + t] : (T)0;
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
        // waiting warps back off so they do not take issue slots from the
        // warps computing the values they wait for
        if (it >= 8) __nanosleep(32);
        if ((it & 1023) == 1023 && *((volatile unsigned *)err) != 0u) return qnan_of<T>();
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
                                        BSlot<T> *ring, unsigned *err, int lane, double &dot)
{
    const int cnt = g1 - g0;
    int32_t hs = 0, hc = 0, hb = 0; // headers of 32 groups, one per lane
    int wbase = -64;
    auto stage = [&](int k) {
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
        const int32_t s = __shfl_sync(BFULL, hs, k - wbase), cw = __shfl_sync(BFULL, hc, k - wbase);
        const int32_t b0 = __shfl_sync(BFULL, hb, k - wbase);
        b_stage<T>(ring[k % BRING], s, cw, b0, qcol, Kv, rhs, rd, lane);
    };
    // dependency values of a staged group (positions lane, lane + 32; the
    // previous group's columns excluded), read before the group before it is
    // published: may still be the sentinel, re-polled when used
    auto peek = [&](const BSlot<T> &S, T &v0, T &v1) {
        const int mx = (S.cw & 255) + ((S.cw >> 8) & 255);
        v0 = (lane < mx) ? b_peek<T>(S.cols[lane], x, mirror, lo, hi) : (T)0;
        v1 = (lane + 32 < mx) ? b_peek<T>(S.cols[lane + 32], x, mirror, lo, hi) : (T)0;
    };
    stage(0);
    cp_async_commit();
    if (cnt > 1) stage(1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    T v0, v1;
    peek(ring[0], v0, v1);
    T p0 = 0, p1 = 0, p2 = 0; // the previous group's values
    int32_t prev_s = 0;
    for (int k = 0; k < cnt; ++k) {
        if (k + 2 < cnt) stage(k + 2);
        cp_async_commit();
        const BSlot<T> &S = ring[k % BRING];
        const int ne = S.cw & 255, nl = (S.cw >> 8) & 255, np = (S.cw >> 16) & 255, G = S.cw >> 24;
        const int mx = ne + nl;
        if (lane < mx && is_sentinel(v0)) v0 = b_fetch<T>(S.cols[lane], x, mirror, lo, hi, err);
        if (lane + 32 < mx && is_sentinel(v1)) v1 = b_fetch<T>(S.cols[lane + 32], x, mirror, lo, hi, err);
        const T w0 = (lane < mx) ? v0 : ((lane - mx < G) ? S.rr[lane - mx] : (T)0);
        const T w1 = (lane + 32 < mx) ? v1 : ((lane + 32 - mx < G) ? S.rr[lane + 32 - mx] : (T)0);
        T a[3];
        if (mx + G > 32) { // uniform
#pragma unroll
            for (int t = 0; t < 3; ++t)
                a[t] = fma(b_coef<T, FWD>(S, t, lane + 32, mx, G), w1, b_coef<T, FWD>(S, t, lane, mx, G) * w0);
        } else {
#pragma unroll
            for (int t = 0; t < 3; ++t) a[t] = b_coef<T, FWD>(S, t, lane, mx, G) * w0;
        }
        if (k + 1 < cnt) { // the next group's data are in; its dependencies start loading
            cp_async_wait<1>();
            __syncwarp();
            peek(ring[(k + 1) % BRING], v0, v1);
        }
        warp_sum_n<T, 3>(a, lane);
        T yv = 0;
        if (lane < G) {
            yv = -pick3<T>(lane, a[0], a[1], a[2]);
            for (int j = 0; j < np; ++j)
                yv = fma(-S.K[lane][mx + j], pick3<T>(S.cols[mx + j] - prev_s, p0, p1, p2), yv);
            const int32_t row = S.s + lane;
            st_relaxed(x + row, yv);
            ((volatile T *)mirror)[row - lo] = yv;
            if (PCG) {
                yreset[row] = sentinel_of<T>();
                dot = fma(S.rd[lane], (double)yv, dot);
            }
        }
        p0 = __shfl_sync(BFULL, yv, 0);
        p1 = __shfl_sync(BFULL, yv, 1);
        p2 = __shfl_sync(BFULL, yv, 2);
        prev_s = S.s;
        __syncwarp(); // slot k is refilled two iterations later
    }
    cp_async_wait<0>();
    __syncwarp();
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
    BSlot<T> *ring = reinterpret_cast<BSlot<T> *>(b_raw) + (threadIdx.x >> 5) * BRING;
    T *mirror = reinterpret_cast<T *>(b_raw + sizeof(BSlot<T>) * BRING * BCHUNKS);
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
                                 PCG ? rd : nullptr, mirror, lo, hi, ring, err, lane, dot);
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
    const size_t smem = sizeof(BSlot<T>) * BRING * BCHUNKS + sizeof(T) * (size_t)(P.mirror_rows > 0 ? P.mirror_rows : 1);
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
