// gic_qsolve.cu -- A7b: warp-specialised sync-free triangular solves for
// patterns whose row groups have at most 3 rows and at most QCOL - 3
// external columns (the hex-element systems: one group per node, x-pencil chunks).
//
// Forward substitution (Eq. (11) read as y_i = (r_i - sum_{j<i} L_ij y_j) /
// L_ii) is done one row group at a time. With D the group's dense lower
// diagonal block and M = D^-1, the group's rows are
//     y_g = M r_g - (M L_ext) y_ext,
// so once the premultiplied coefficients K = M L_ext are formed for a factor
// (q_setup, once per PCG run), every row of a group is an independent dot
// product: no in-group substitution chain is left on the critical path.
// Backward (L^T z = y) uses z_g = M^T y_g - (M^T U_ext) z_ext on U = L^T.
//
// A team of three warps shares one chunk (a run of groups solved in order):
//  * two producers, one for the even and one for the odd groups of the
//    chunk, stage a group's columns and coefficients in shared memory
//    (cp.async, a ring of QR slots), load the "early" dependencies (finished
//    well before the group), reduce their part of the dot products across
//    lanes and leave base = -K_early y_early;
//  * the finisher (four lanes per row, one accumulation chain each) adds the
//    group's own right-hand side M r_g, the contribution of the previous
//    group of the chunk from registers and of the few "late" dependencies
//    (within a level window of the group), waiting only for those, and
//    publishes y.
// The producers' lane-parallel work runs while the finisher waits, so the
// chain from one group to the next is a handful of FMAs plus the latency of
// the dependencies themselves; with two producers their per-group cycle
// (staging, reduction, hand-off: ~1.3 us on GB300) no longer sets the
// chunk's pace. Readiness is the solution word itself (a
// signalling-NaN sentinel until written), every wait is bounded, and the
// chunk order guarantees that the earliest unfinished chunk can always run.
#include <limits.h>
#include <math.h>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int QR = 8;                    // ring slots per chunk team
constexpr int QDO = 2;                   // own groups a producer stages ahead
constexpr int QBLOCK = 192;              // threads per block: two teams of three warps
constexpr int QTEAMS = QBLOCK / 96;      // teams per block
constexpr int QTEAMS_PER_SM = 4;         // cap on resident teams per SM: < 16 chunks per SM,
constexpr int QTEAMS_PER_SM_MANY = 8;    // < 64 chunks per SM,
constexpr int QTEAMS_PER_SM_QUEUED = 16; // more
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct QSlot {
    T K[3][QCOL];      // premultiplied external coefficients, columns [early | late | prev]
    T Mv[6];           // M = D^-1, packed lower triangle (t, u <= t) at t(t+1)/2 + u
    T rr[3];           // right-hand side rows (forward: r, backward: y)
    T base[3];         // M rr - early part, written by the producer
    double rd[3];      // backward with PCG: r in FP64 for the fused r^T z
    int32_t cols[QCOL];
    int32_t s, cw;     // first row, packed counts
};

// Slot i of the ring serves groups q = i, i + QR, ...; its j-th use (j =
// q / QR) completes phase j of full[i] (producer -> finisher: staged data
// and base are in place) and phase j of freed[i] (finisher -> producer: the
// slot may be refilled). Waiting threads are suspended by the hardware
// (mbarrier try_wait) instead of spinning on shared memory.
template <typename T>
struct QRing {
    QSlot<T> slot[QR];
    unsigned long long full[QR], freed[QR];
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for the completion of the phase with the given parity; every
// calling thread waits (and acquires). False after the limit (error flag
// set) or once another thread has flagged an error.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned *err)
{
    const unsigned a = smem_addr(bar);
    for (long long it = 0; it < (SPIN_LIMIT >> 2); ++it) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 63) == 63 && *((volatile unsigned *)err) != 0u) return false;
    }
    atomicOr(err, ERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ bool warp_all(bool v) { return __all_sync(FULL, v) != 0; }

template <typename T>
__device__ __forceinline__ void q_stage(QSlot<T> &S, int32_t s, int32_t cw, int64_t b0, const int32_t *qcol,
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

// Transposed warp sum of three values (the first two butterfly levels
// exchange halves so each lane adds 2, then 1 value): 6 adds; row t's total
// ends in lanes 8t .. 8t + 7.
template <typename T>
__device__ __forceinline__ T warp_sum_3_rows(const T (&a)[3], int lane)
{
    const bool hi16 = lane & 16;
    T k0 = hi16 ? a[2] : a[0], k1 = hi16 ? (T)0 : a[1];
    const T s0 = hi16 ? a[0] : a[2], s1 = hi16 ? a[1] : (T)0;
    k0 += __shfl_xor_sync(FULL, s0, 16);
    k1 += __shfl_xor_sync(FULL, s1, 16);
    const bool b8 = lane & 8;
    T kk = b8 ? k1 : k0;
    kk += __shfl_xor_sync(FULL, b8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) kk += __shfl_xor_sync(FULL, kk, o);
    return kk;
}

// Producer of the groups k = parity, parity + 2, ... of one chunk (groups in
// sweep order k = 0..cnt-1); the team's other producer takes the others.
template <typename T, bool FWD>
__device__ __forceinline__ bool q_produce(QRing<T> &Q, int seq, int32_t g0, int32_t g1, int parity, const int32_t *grp,
                                          const int32_t *rowptr, const int32_t *qcol, const int32_t *qcnt,
                                          const T *Kv, const T *rhs, const T *x, const double *rd, unsigned *err,
                                          int poll, int lane)
{
    const int cnt = g1 - g0;
    int32_t hs = 0, hc = 0, hb = 0; // headers of 32 groups, one per lane
    int wbase = -64;
    bool ok = true;
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
        const int32_t s = __shfl_sync(FULL, hs, k - wbase), cw = __shfl_sync(FULL, hc, k - wbase);
        const int32_t b0 = __shfl_sync(FULL, hb, k - wbase);
        const int q = seq + k, use = q / QR;
        if (use > 0 && !warp_all(mbar_wait(&Q.freed[q % QR], (unsigned)(use - 1) & 1u, err))) {
            ok = false;
            return;
        }
        q_stage<T>(Q.slot[(seq + k) % QR], s, cw, b0, qcol, Kv, rhs, rd, lane);
    };
#pragma unroll
    for (int d = 0; d < QDO; ++d) {
        if (parity + 2 * d < cnt && ok) stage(parity + 2 * d);
        cp_async_commit();
    }
    // early dependency values of the group about to be reduced (loaded one
    // own group ahead so their latency overlaps the previous reduction)
    T v0 = 0, v1 = 0;
    int32_t j0 = -1, j1 = -1;
    auto load_early = [&](int k) {
        cp_async_wait<QDO - 1>();
        __syncwarp();
        const QSlot<T> &S = Q.slot[(seq + k) % QR];
        const int ne = S.cw & 255;
        j0 = (lane < ne) ? S.cols[lane] : -1;
        j1 = (lane + 32 < ne) ? S.cols[lane + 32] : -1;
        v0 = (j0 >= 0) ? ld_relaxed(x + j0) : (T)0;
        v1 = (j1 >= 0) ? ld_relaxed(x + j1) : (T)0;
    };
    if (parity < cnt && ok) load_early(parity);
    for (int k = parity; k < cnt && ok; k += 2) {
        if (k + 2 * QDO < cnt) stage(k + 2 * QDO);
        cp_async_commit();
        QSlot<T> &S = Q.slot[(seq + k) % QR];
        const int ne = S.cw & 255, G = S.cw >> 24;
        wait_pair<FWD, T>(x, j0, j1, v0, v1, err, poll);
        // a = K_early y_early over the early columns p < ne (v is 0 past
        // them); the group's own right-hand side part M rr is the
        // finisher's
        const bool two = ne > 32; // uniform over the warp
        T a[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const T c0 = (t < G && j0 >= 0) ? S.K[t][lane] : (T)0;
            if (two) {
                const T c1 = (t < G && j1 >= 0) ? S.K[t][lane + 32] : (T)0;
                a[t] = fma(c1, v1, c0 * v0);
            } else {
                a[t] = c0 * v0;
            }
        }
        if (k + 2 < cnt) load_early(k + 2);
        const T tot = warp_sum_3_rows<T>(a, lane); // row t's total in lanes 8t .. 8t + 7
        if ((lane & 7) == 0 && (lane >> 3) < G) S.base[lane >> 3] = -tot;
        // __syncwarp orders the lanes' base stores before lane 0's arrive,
        // whose release makes them visible to the finisher's acquiring wait
        __syncwarp();
        if (lane == 0) mbar_arrive(&Q.full[(seq + k) % QR]);
    }
    cp_async_wait<0>();
    __syncwarp();
    return ok;
}

// Finisher of one chunk: lane 4t + c (t < G, c < 4) accumulates chain c of
// row t and two shuffle levels add the chains. Against one lane per row this
// issues a quarter of the arithmetic and load instructions (an FP64 warp
// instruction occupies the SM's FP64 pipe as long with 3 active lanes as with
// 32) and makes the dependent chain a quarter as deep: ~25% faster sweeps in
// FP64 and ~20% in FP32 on the hex systems.
template <typename T, bool FWD, bool PCG>
__device__ __forceinline__ bool q_finish(QRing<T> &Q, int seq, int cnt, T *x, T *yreset, unsigned *err, int lane,
                                         double &dot, unsigned sleep_ns)
{
    const int t = lane >> 2, c = lane & 3;
    T yp = 0;          // the previous group of the chunk: row t in lanes 4t .. 4t + 3
    int32_t prev_s = 0;
    for (int k = 0; k < cnt; ++k) {
        const int q = seq + k;
        if (!warp_all(mbar_wait(&Q.full[q % QR], (unsigned)(q / QR) & 1u, err))) return false;
        const QSlot<T> &S = Q.slot[q % QR];
        const int32_t cw = S.cw, s = S.s;
        const int ne = cw & 255, nl = (cw >> 8) & 255, np = (cw >> 16) & 255, G = cw >> 24;
        // the previous group's columns (its rows: np <= 3, the analysis admits
        // groups of at most 3 rows) go to chains c < np, so lane (t, c) needs
        // one value: previous-group row jr, held by lanes 4 jr .. 4 jr + 3
        const int jr = (c < np) ? S.cols[ne + nl + c] - prev_s : 0;
        const T pv = __shfl_sync(FULL, yp, 4 * jr);
        T acc = 0;
        if (t < G) {
            // chain c takes late values j = c, c + 4, ... (the schedule orders
            // them farthest level first, so the one most likely to arrive
            // last is consumed last) and previous-group columns j = c, c + 4,
            // ...; chain 0 starts from the producer's base
            T lv[QLATE / 4];
#pragma unroll
            for (int i = 0; i < QLATE / 4; ++i) {
                const int j = c + 4 * i;
                lv[i] = (j < nl) ? ld_relaxed(x + S.cols[ne + j]) : (T)0;
            }
            if (c == 0) acc = S.base[t];
            // the group's own right-hand side: forward y_t gets M_tu r_u
            // (u <= t), backward z_t gets M_ut y_u (u >= t); chain c takes u = c
            if (c < G && (FWD ? c <= t : c >= t))
                acc = fma(FWD ? S.Mv[t * (t + 1) / 2 + c] : S.Mv[c * (c + 1) / 2 + t], S.rr[c], acc);
            if (c < np) acc = fma(-S.K[t][ne + nl + c], pv, acc);
#pragma unroll
            for (int i = 0; i < QLATE / 4; ++i) {
                const int j = c + 4 * i;
                if (j < nl) {
                    T v = lv[i];
                    if (is_sentinel(v)) v = wait_word(x + S.cols[ne + j], err, sleep_ns);
                    acc = fma(-S.K[t][ne + j], v, acc);
                }
            }
        }
        acc += __shfl_xor_sync(FULL, acc, 1);
        acc += __shfl_xor_sync(FULL, acc, 2); // row t's value in lanes 4t .. 4t + 3
        if (c == 0 && t < G) {
            st_relaxed(x + s + t, acc);
            if (PCG) {
                yreset[s + t] = sentinel_of<T>();
                dot = fma(S.rd[t], (double)acc, dot);
            }
        }
        yp = acc;
        __syncwarp(); // the lanes' slot reads precede lane 0's releasing arrive
        if (lane == 0) mbar_arrive(&Q.freed[q % QR]);
        prev_s = s;
    }
    return true;
}

// FWD: L y = r (x = y, rhs = r). Backward: L^T z = y (x = z, rhs = y); with
// PCG it also resets y to the sentinel for the next forward sweep and forms
// r^T z in FP64, then beta = r_k^T z_k / r_{k-1}^T z_{k-1} (Algorithm 1) in
// the last warp to finish. x must hold the sentinel.
template <typename T, bool FWD, bool PCG>
__global__ void __launch_bounds__(QBLOCK, 4) k_qsolve(int32_t nchunks, const int32_t *__restrict__ ord,
                                                        const int32_t *__restrict__ chunk_grp,
                                                        const int32_t *__restrict__ grp,
                                                        const int32_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ qcol,
                                                        const int32_t *__restrict__ qcnt, const T *__restrict__ Kv,
                                                        const T *rhs, T *x, T *yreset, const double *__restrict__ rd,
                                                        double *partials, unsigned *err, int poll, Scalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) unsigned char q_raw[];
    QRing<T> *rings = reinterpret_cast<QRing<T> *>(q_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int role = wib % 3; // 0, 1: producers of the even / odd groups; 2: finisher
    QRing<T> &Q = rings[wib / 3];
    if (role == 0 && lane < QR) {
        mbar_init(&Q.full[lane], 1);
        mbar_init(&Q.freed[lane], 1);
    }
    __syncthreads();
    const int64_t gteam = (int64_t)blockIdx.x * QTEAMS + wib / 3;
    const int64_t nteam = (int64_t)gridDim.x * QTEAMS;
    int seq = 0;
    double dot = 0.0;
    bool ok = true;
    for (int64_t pos = gteam; pos < nchunks && ok; pos += nteam) {
        const int32_t c = ord[pos];
        const int32_t g0 = chunk_grp[c], g1 = chunk_grp[c + 1];
        if (role < 2)
            ok = q_produce<T, FWD>(Q, seq, g0, g1, role, grp, rowptr, qcol, qcnt, Kv, rhs, x, PCG ? rd : nullptr, err,
                                   poll, lane);
        else
            ok = q_finish<T, FWD, PCG>(Q, seq, g1 - g0, x, yreset, err, lane, dot, (unsigned)(poll & 0xffff));
        seq += g1 - g0;
    }
    if (PCG) {
        dot = warp_sum(dot);
        const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        if (lane == 0) partials[w] = dot;
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence();
            last = (atomicAdd(&sc->counter, 1u) == (unsigned)nw - 1u);
        }
        last = __shfl_sync(FULL, last, 0);
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

// Premultiplied group blocks of a factor, computed in FP64 and stored in TL:
// forward K = M L_ext in the L layout (rows t of the group at
// Lrowptr[s] + t m, columns in the schedule's order, then M packed), backward
// K = M^T U_ext in the U layout at Urowptr[s].
template <typename TL>
__global__ void k_qsetup(int32_t ngroups, const int32_t *__restrict__ grp, const int32_t *__restrict__ Lrowptr,
                         const int32_t *__restrict__ Urowptr, const int32_t *__restrict__ tperm,
                         const uint8_t *__restrict__ qf_pos, const uint8_t *__restrict__ qb_pos,
                         const TL *__restrict__ Lval, TL *__restrict__ Kf, TL *__restrict__ Kb)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = grp[g], G = grp[g + 1] - s, e = s + G - 1;
        const int64_t b0 = Lrowptr[s];
        const int m = (int)(Lrowptr[s + 1] - b0 - 1);
        double D[3][3] = {}, M[3][3] = {};
        for (int t = 0; t < G; ++t)
            for (int u = 0; u <= t; ++u) D[t][u] = (double)Lval[Lrowptr[s + t] + m + u];
        for (int t = 0; t < G; ++t) {
            M[t][t] = 1.0 / D[t][t];
            for (int u = 0; u < t; ++u) {
                double a = 0.0;
                for (int v = u; v < t; ++v) a = fma(D[t][v], M[v][u], a);
                M[t][u] = -a * M[t][t];
            }
        }
        for (int k = 0; k < m; ++k) {
            const int j = qf_pos[b0 + k];
            for (int t = 0; t < G; ++t) {
                double a = 0.0;
                for (int u = 0; u <= t; ++u) a = fma(M[t][u], (double)Lval[Lrowptr[s + u] + j], a);
                Kf[b0 + (int64_t)t * m + k] = (TL)a;
            }
        }
        const int64_t bu = Urowptr[s];
        const int mu = (int)(Urowptr[e + 1] - Urowptr[e] - 1);
        for (int k = 0; k < mu; ++k) {
            const int j = qb_pos[bu + k];
            for (int t = 0; t < G; ++t) {
                double a = 0.0;
                for (int u = t; u < G; ++u) a = fma(M[u][t], (double)Lval[tperm[Urowptr[s + u] + (G - u) + j]], a);
                Kb[bu + (int64_t)t * mu + k] = (TL)a;
            }
        }
        for (int t = 0; t < G; ++t)
            for (int u = 0; u <= t; ++u) {
                Kf[b0 + (int64_t)G * m + t * (t + 1) / 2 + u] = (TL)M[t][u];
                Kb[bu + (int64_t)G * mu + t * (t + 1) / 2 + u] = (TL)M[t][u];
            }
    }
}

int q_setup(gic_handle *h, const Pattern &P, bool f32, const void *Lval, void *Kf, void *Kb)
{
    if (!P.qready) return GIC_ERR_UNSUPPORTED;
    int64_t b = (P.ngroups + 127) / 128, cap = (int64_t)h->num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    ++h->launches;
    if (f32)
        k_qsetup<float><<<(unsigned)b, 128, 0, h->stream>>>(P.ngroups, P.grp, P.Lrowptr, P.Urowptr, P.tperm, P.qf_pos,
                                                            P.qb_pos, (const float *)Lval, (float *)Kf, (float *)Kb);
    else
        k_qsetup<double><<<(unsigned)b, 128, 0, h->stream>>>(P.ngroups, P.grp, P.Lrowptr, P.Urowptr, P.tperm, P.qf_pos,
                                                             P.qb_pos, (const double *)Lval, (double *)Kf, (double *)Kb);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

template <typename T, bool FWD, bool PCG>
static int q_launch(gic_handle *h, const Pattern &P, const T *Kv, const T *rhs, T *x, T *yreset, const double *rd,
                    double *partials, Scalars *sc)
{
    if (!P.qready) return GIC_ERR_UNSUPPORTED;
    int32_t nc = P.nchunks;
    const int32_t *ord = FWD ? P.ord_f : P.ord_b, *cg = P.chunk_grp, *g = P.grp;
    const int32_t *rp = FWD ? P.Lrowptr : P.Urowptr;
    const int32_t *qc = FWD ? P.qf_col : P.qb_col, *qn = FWD ? P.qf_cnt : P.qb_cnt;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&nc, &ord, &cg, &g, &rp, &qc, &qn, &Kv, &rhs, &x, &yreset, &rd, &partials, &er, &poll, &sc};
    // warps: one team of three per chunk, teams capped per SM by the chunks
    // per SM (40^3 hex system: ~11 -> 4 teams, 69^3: ~32 -> 8, 148^3: ~145
    // -> 16): extra co-resident teams contend for the FP64 pipe and issue
    // slots and slow the chain, which pays only once the chunks queue.
    int64_t need = 3 * (int64_t)nc;
    int per_sm = h->tune_solve_warps_per_sm;
    const int64_t nsm = h->num_sms;
    if (per_sm == 0)
        per_sm = (nc < 16 * nsm) ? QTEAMS_PER_SM : (nc < 64 * nsm) ? QTEAMS_PER_SM_MANY : QTEAMS_PER_SM_QUEUED;
    if (per_sm > 0 && need > 3 * (int64_t)per_sm * h->num_sms) need = 3 * (int64_t)per_sm * h->num_sms;
    if (PCG && need > MAX_PARTIALS) need = MAX_PARTIALS; // grid warps <= partial slots
    const size_t smem = sizeof(QRing<T>) * QTEAMS;
    static bool ad[64] = {};
    if (!ad[h->device & 63]) {
        GIC_CUDA_TRY(cudaFuncSetAttribute(k_qsolve<T, FWD, PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        ad[h->device & 63] = true;
    }
    return launch_persistent(h, (const void *)k_qsolve<T, FWD, PCG>, QBLOCK, smem, need, args);
}

int q_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Kf, const void *r, void *y, const Scalars *sc)
{
    Scalars *s = const_cast<Scalars *>(sc);
    if (f32)
        return q_launch<float, true, false>(h, P, (const float *)Kf, (const float *)r, (float *)y, nullptr, nullptr,
                                            nullptr, s);
    return q_launch<double, true, false>(h, P, (const double *)Kf, (const double *)r, (double *)y, nullptr, nullptr,
                                         nullptr, s);
}

int q_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Kb, void *y, void *z,
              const double *rd, double *partials, Scalars *sc)
{
    if (f32) {
        if (pcg)
            return q_launch<float, false, true>(h, P, (const float *)Kb, (const float *)y, (float *)z, (float *)y, rd,
                                                partials, sc);
        return q_launch<float, false, false>(h, P, (const float *)Kb, (const float *)y, (float *)z, nullptr, nullptr,
                                             nullptr, sc);
    }
    if (pcg)
        return q_launch<double, false, true>(h, P, (const double *)Kb, (const double *)y, (double *)z, (double *)y, rd,
                                             partials, sc);
    return q_launch<double, false, false>(h, P, (const double *)Kb, (const double *)y, (double *)z, nullptr, nullptr,
                                          nullptr, sc);
}

}  // namespace gic
