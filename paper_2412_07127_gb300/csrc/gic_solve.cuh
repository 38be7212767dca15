// gic_solve.cuh -- pieces shared by the PCG driver (gic_solve.cu) and the
// warp-specialised triangular solves (gic_qsolve.cu).
#pragma once
#include "gic_internal.cuh"

namespace gic {

// Device-resident scalars of one PCG run (Supplementary Algorithm 1).
struct Scalars {
    double rz;    // r_k^T z_k
    double pw;    // p^T A p
    double alpha, beta;
    double rr, bb; // ||r||^2, ||b||^2
    double tol;
    int iter, maxit, done, status;
    unsigned counter; // last-block ticket
    unsigned pad;
};

// Block sum of one double per thread (warp sums, then thread 0 adds the
// warps' in order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    __syncthreads();
    return s;
}

// Called by thread 0 of every block after writing partials[blockIdx.x]
// (count = gridDim.x). Returns true in the one block that arrives last.
__device__ __forceinline__ bool last_block(unsigned *counter, unsigned count)
{
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    return t == count - 1;
}

constexpr int SOLVE_BLOCK = 256;
constexpr int MAX_PARTIALS = 1 << 16;

// deterministic sum of partials[0..count) by one warp (lane-strided in index
// order, then tree). The caller has fenced after seeing every producer's
// ticket; the loads bypass L1 (__ldcg) and are not volatile, so up to eight
// of a lane's loads are in flight at once instead of one after another.
__device__ __forceinline__ double warp_sum_partials(const double *partials, int count)
{
    int lane = threadIdx.x & 31;
    double s = 0.0;
#pragma unroll 8
    for (int k = lane; k < count; k += 32) s += __ldcg(partials + k);
    return warp_sum(s);
}

// Warp sum of GM values, result in every lane. For three values the first
// two butterfly levels exchange halves so each lane adds 2, then 1 value.
template <typename T, int GM>
__device__ __forceinline__ void warp_sum_n(T (&a)[GM], int lane)
{
    if (GM == 3) {
        const bool hi16 = lane & 16;
        // level 16: lanes < 16 keep {0,1}, lanes >= 16 keep {2, pad}
        T k0 = hi16 ? a[2] : a[0], k1 = hi16 ? (T)0 : a[1];
        T s0 = hi16 ? a[0] : a[2], s1 = hi16 ? a[1] : (T)0;
        k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
        k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
        // level 8: bit3 = 0 keeps k0, bit3 = 1 keeps k1
        const bool b8 = lane & 8;
        T kk = b8 ? k1 : k0, ss = b8 ? k0 : k1;
        kk += __shfl_xor_sync(0xffffffffu, ss, 8);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
        // totals: lanes 0-7 row 0, 8-15 row 1, 16-23 row 2
        a[0] = __shfl_sync(0xffffffffu, kk, 0);
        a[1] = __shfl_sync(0xffffffffu, kk, 8);
        a[2] = __shfl_sync(0xffffffffu, kk, 16);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int t = 0; t < GM; ++t) a[t] += __shfl_xor_sync(0xffffffffu, a[t], o);
    }
}

template <typename T>
__device__ __forceinline__ T pick3(int idx, T a, T b, T c) { return idx == 0 ? a : (idx == 1 ? b : c); }


int launch_persistent(gic_handle *h, const void *fn, int block, size_t smem, int64_t warps_needed, void **args);

// Warp-specialised solves (gic_qsolve.cu). q_setup writes the premultiplied
// group blocks of a factor (TL = double or float) into Kf (forward, L
// layout) and Kb (backward, U layout); the solves then run on them.
int q_setup(gic_handle *h, const Pattern &P, bool f32, const void *Lval, void *Kf, void *Kb);
int q_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Kf, const void *r, void *y, const Scalars *sc);
int q_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Kb, void *y, void *z,
              const double *rd, double *partials, Scalars *sc);

// Level-sliced solves (gic_ssolve.cu): s_setup writes a factor's
// coefficients in the slice layout into Sf (forward) and Sb (backward),
// s_values_bytes(sched, element size) bytes each.
size_t p_values_bytes(const PairSched &S, size_t es);
int p_setup(gic_handle *h, const Pattern &P, bool f32, const void *Lval, void *Vf, void *Vb);
int p_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Vf, const void *r, void *y, const Scalars *sc);
int p_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Vb, const void *y, void *z,
              const double *rd, double *partials, Scalars *sc);
size_t s_values_bytes(const SliceSched &S, size_t es);
int s_setup(gic_handle *h, const Pattern &P, bool f32, const void *Lval, void *Sf, void *Sb);
int s_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Sf, const void *r, void *y, const Scalars *sc);
int s_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Sb, void *y, void *z,
              const double *rd, double *partials, Scalars *sc);

// 3x3 node-block SpMV (gic_bsr.cu): A's values in the block layout
// (9 * 32 * P.bsr_steps doubles), and y = A x with the PCG's fused
// reductions (mode 1: p^T w and alpha; mode 2: r = b - A x, ||r||, ||b||).
int bsr_values(gic_handle *h, const Pattern &P, const double *valA, double *bval);
int bsr_spmv(gic_handle *h, const Pattern &P, int mode, const double *bval, const double *x, double *y,
             const double *b, double *partials, Scalars *sc);

// automatic solve choice: level-sliced kernels from this many chunks per SM
// Level- and pair-sliced solves: wait until no lane of the warp holds a
// sentinel among its B values. All pending words are reloaded together each
// round (the values of a wave come from several slices and land at
// different times, so polling them one at a time would serialise their
// round trips: measured 1.5x slower), with a short back-off after the first
// rounds; bounded (then ERR_TIMEOUT and NaN values).
template <typename T, int B>
__device__ __forceinline__ void slice_wait(const T *x, const int32_t (&c)[B], T (&v)[B], unsigned *err,
                                       unsigned sleep_ns, int lane)
{
    for (long long it = 0;; ++it) {
        bool pend = false;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (c[b] >= 0 && is_sentinel(v[b])) {
                v[b] = ld_relaxed(x + c[b]);
                pend |= is_sentinel(v[b]);
            }
        }
        if (!__any_sync(0xffffffffu, pend)) return;
        if (it >= SPIN_LIMIT || ((it & 255) == 255 && *((volatile unsigned *)err) != 0u)) {
            if (it >= SPIN_LIMIT && lane == 0) atomicOr(err, ERR_TIMEOUT);
#pragma unroll
            for (int b = 0; b < B; ++b)
                if (c[b] >= 0 && is_sentinel(v[b])) v[b] = qnan_of<T>();
            return;
        }
        if (it >= 32) __nanosleep(it >= 65536 ? 256 : (sleep_ns ? sleep_ns : 32));
    }
}

constexpr int SLICED_CHUNKS_PER_SM = 48;
// Automatic choice of the solve kernels by chunks (for hex elasticity the
// x-pencils) per SM, measured on the hex systems from 40^3 to 148^3: below
// SLICED_CHUNKS_PER_SM the warp-specialised kernels, up to
// PAIRED_CHUNKS_PER_SM the pair-sliced ones (whose pair schedule the
// analysis builds only then, or when the pipeline setting asks for them),
// above it the level-sliced ones.
constexpr int PAIRED_CHUNKS_PER_SM = 120;

}  // namespace gic
