// gic_gnn_tc.cu -- A5: the GNN's edge MLP on the 5th-generation tensor cores.
//
// Per layer l the edge MLP (Section "Model Architecture"; Supplementary 3)
// maps every edge's input h = [e_cur, e0, x_i, x_j] (20 values) to
//     e_new = W2 tanh(W1 h + b1) + b2,   W1: 32 x 20.
// The first layer is the only dense contraction of the method: an
// (edges x 20) by (20 x 32) product. Here a CTA takes tiles of 128 edges:
//  * each of its 128 threads gathers one edge's inputs, rounds them to BF16
//    and writes the row into shared memory in the tensor cores' K-major
//    layout without swizzle (8-row x 16-byte core matrices; K padded 20 -> 32
//    with zeros);
//  * one thread issues two tcgen05.mma kind::f16 instructions (M = 128,
//    N = 32, K = 16 each, BF16 x BF16 -> FP32) into a 32-column TMEM
//    accumulator and commits them to an mbarrier;
//  * every thread reads its edge's 32 accumulators back with tcgen05.ld and
//    finishes b1, tanh (the hardware approximation), W2 and b2 in FP32.
// W1 is rounded to BF16 once per CTA; b1, W2, b2 and the accumulation stay
// FP32. The bounded mbarrier wait sets the error flag and skips the tile on
// timeout; the TMEM columns are always released before the CTA exits.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "gic_internal.cuh"

namespace gic {

constexpr int TC_M = 128;            // edges per tile (MMA M)
constexpr int TC_N = 32;             // hidden width (MMA N)
constexpr int TC_K = 32;             // padded input width (two MMA K-steps of 16)
constexpr int TC_NP_EDGE = TC_N * 20 + TC_N + TC_N + 1;
constexpr int TC_NP_NODE = TC_N * 11 + TC_N + 9 * TC_N + 9;
constexpr uint32_t TC_COLS = 32;     // TMEM columns of the accumulator

__device__ __forceinline__ int tc_off_edge(int l) { return 27 + l * (TC_NP_EDGE + TC_NP_NODE); }

// byte offset of element (row, k) of a row-major tile in the K-major
// no-swizzle layout: core matrices of 8 rows x 8 BF16 (16 bytes per row),
// adjacent along K 128 bytes apart (LBO), adjacent along rows 512 bytes
// apart (SBO, four core matrices of K per 8 rows)
__device__ __forceinline__ uint32_t tc_off(int row, int k)
{
    return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint64_t sbo = 512)
{
    const uint64_t lbo = 128;
    return (uint64_t)((saddr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16) | (((sbo >> 4) & 0x3FFF) << 32) |
           (1ull << 46); // descriptor version 1, base offset 0, no swizzle
}

// the same layout for a tile whose K is 16 (two core matrices along K: rows
// of core matrices 256 bytes apart)
__device__ __forceinline__ uint32_t tc_off16(int row, int k)
{
    return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major,
// N = 32, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint16_t tc_bf16(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// hardware tanh (PTX tanh.approx.f32, relative error about 2^-11): finer
// than the BF16 rounding of the layer's inputs (2^-8)
__device__ __forceinline__ float tc_tanh(float v)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ uint32_t tc_pack(float a, float b)
{
    return (uint32_t)tc_bf16(a) | ((uint32_t)tc_bf16(b) << 16);
}

__global__ void __launch_bounds__(TC_M) k_edge_fwd_tc(int64_t E, const int32_t *__restrict__ Lrow,
                                                      const int32_t *__restrict__ Lcol, const float *__restrict__ ein,
                                                      const float *__restrict__ e0, const float *__restrict__ x,
                                                      const float *__restrict__ theta, int l, float *__restrict__ eout,
                                                      unsigned *err)
{
    __shared__ __align__(128) unsigned char sA[TC_M * TC_K * 2];
    __shared__ __align__(128) unsigned char sB[TC_N * TC_K * 2];
    __shared__ float b1[TC_N], W2[TC_N], b2s;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) unsigned long long mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    const float *P = theta + tc_off_edge(l);
    for (int idx = tid; idx < TC_N * TC_K; idx += TC_M) {
        const int n = idx / TC_K, k = idx % TC_K;
        *(uint16_t *)(sB + tc_off(n, k)) = tc_bf16(k < 20 ? P[n * 20 + k] : 0.0f);
    }
    if (tid < TC_N) {
        b1[tid] = P[TC_N * 20 + tid];
        W2[tid] = P[TC_N * 20 + TC_N + tid];
    }
    if (tid == 0) {
        b2s = P[TC_N * 20 + 2 * TC_N];
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t aaddr = (uint32_t)__cvta_generic_to_shared(sA), baddr = (uint32_t)__cvta_generic_to_shared(sB);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    uint32_t phase = 0;
    const int64_t ntiles = (E + TC_M - 1) / TC_M;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = tile * TC_M + tid;
        const bool valid = p < E;
        float h[20];
        if (valid) {
            const int64_t i = Lrow[p], j = Lcol[p];
            h[0] = ein[p];
            h[1] = e0[p];
#pragma unroll
            for (int f = 0; f < 9; ++f) {
                h[2 + f] = x[9 * i + f];
                h[11 + f] = x[9 * j + f];
            }
        } else {
#pragma unroll
            for (int f = 0; f < 20; ++f) h[f] = 0.0f;
        }
        // the row in four 16-byte chunks (K 0-7, 8-15, 16-23, 24-31)
        uint4 c0 = make_uint4(tc_pack(h[0], h[1]), tc_pack(h[2], h[3]), tc_pack(h[4], h[5]), tc_pack(h[6], h[7]));
        uint4 c1 = make_uint4(tc_pack(h[8], h[9]), tc_pack(h[10], h[11]), tc_pack(h[12], h[13]),
                              tc_pack(h[14], h[15]));
        uint4 c2 = make_uint4(tc_pack(h[16], h[17]), tc_pack(h[18], h[19]), 0u, 0u);
        uint4 c3 = make_uint4(0u, 0u, 0u, 0u);
        *(uint4 *)(sA + tc_off(tid, 0)) = c0;
        *(uint4 *)(sA + tc_off(tid, 8)) = c1;
        *(uint4 *)(sA + tc_off(tid, 16)) = c2;
        *(uint4 *)(sA + tc_off(tid, 24)) = c3;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint64_t ad = tc_desc(aaddr + s * 256), bd = tc_desc(baddr + s * 256);
                asm volatile("{\n\t.reg .pred acc;\n\t"
                             "setp.ne.b32 acc, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, acc;\n\t}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(s));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        // bounded wait for the two MMAs
        int done = 0;
        for (long long it = 0; it < (SPIN_LIMIT >> 2) && !done; ++it) {
            asm volatile("{\n\t.reg .pred p;\n\t"
                         "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done)
                         : "r"(mb), "r"(phase)
                         : "memory");
        }
        if (!done) atomicOr(err, ERR_TIMEOUT);
        const int all_done = __syncthreads_and(done);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!all_done) break; // the accumulator may still be written: stop using it
        uint32_t r[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                     "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                       "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                       "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float out = b2s;
#pragma unroll
        for (int u = 0; u < TC_N; ++u) out = fmaf(W2[u], tc_tanh(__uint_as_float(r[u]) + b1[u]), out);
        if (valid) eout[p] = out;
        // every thread's TMEM reads finish before the next tile's MMA
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

int edge_fwd_tc(gic_handle *h, int64_t E, const int32_t *Lrow, const int32_t *Lcol, const float *ein,
                const float *e0, const float *x, const float *theta, int l, float *eout)
{
    // up to 8 CTAs per SM (registers allow 8 of 128 threads; 8 x 32 TMEM
    // columns of the SM's 512): the tile loop has no internal overlap, so
    // co-resident CTAs hide each other's gathers
    int64_t tiles = (E + TC_M - 1) / TC_M, cap = (int64_t)h->num_sms * 8;
    if (tiles > cap) tiles = cap;
    if (tiles < 1) tiles = 1;
    ++h->launches;
    k_edge_fwd_tc<<<(unsigned)tiles, TC_M, 0, h->stream>>>(E, Lrow, Lcol, ein, e0, x, theta, l, eout, h->dev_err);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}


// ------------------------------------------------------------ node MLP
// Per block the node MLP maps every node's input u = [x (9), S, M] to
//     x_new = W4 tanh(W3 u + b3) + b4,   W3: 32 x 11, W4: 9 x 32,
// two (nodes x K) by (K x N) products: (n x 11)(11 x 32) and (n x 32)(32 x 9).
// A CTA takes tiles of 128 nodes: each thread aggregates its node's S and M,
// rounds u to BF16 into shared memory (K padded 11 -> 16), one thread issues
// the first MMA (M 128, N 32, K 16) into TMEM columns 0-31; every thread reads
// its 32 accumulators, adds b3, applies tanh (the accurate one: the hardware
// approximation's error would move the BF16 rounding of the activations that
// follows), rounds the activations to BF16
// into a second K-major tile (K = 32), and one thread issues the second
// product (N 16 with W4 padded from 9 rows, two K-steps) into columns 32-47;
// the threads read their 9 outputs and add b4.
constexpr int TN_K1 = 16;            // padded node-MLP input width
constexpr int TN_N2 = 16;            // padded output width (9)
constexpr uint32_t TN_COLS = 64;     // TMEM columns: hidden 0-31, outputs 32-47
constexpr uint32_t TN_IDESC1 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
constexpr uint32_t TN_IDESC2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN_N2 >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ int tc_off_node(int l) { return tc_off_edge(l) + TC_NP_EDGE; }

__device__ __forceinline__ bool tc_wait(uint32_t mb, uint32_t phase, unsigned *err)
{
    int done = 0;
    for (long long it = 0; it < (SPIN_LIMIT >> 2) && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mb), "r"(phase)
                     : "memory");
    }
    if (!done) atomicOr(err, ERR_TIMEOUT);
    return done != 0;
}

__global__ void __launch_bounds__(TC_M) k_node_fwd_tc(int64_t n, const int32_t *__restrict__ Lrowptr,
                                                      const int32_t *__restrict__ Urowptr,
                                                      const int32_t *__restrict__ tperm, const float *__restrict__ e,
                                                      const float *__restrict__ x, const float *__restrict__ theta,
                                                      int l, float *__restrict__ xout, unsigned *err)
{
    __shared__ __align__(128) unsigned char sA1[TC_M * TN_K1 * 2];
    __shared__ __align__(128) unsigned char sB1[TC_N * TN_K1 * 2];
    __shared__ __align__(128) unsigned char sA2[TC_M * TC_K * 2];
    __shared__ __align__(128) unsigned char sB2[TN_N2 * TC_K * 2];
    __shared__ float b3[TC_N], b4[TN_N2];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) unsigned long long mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    const float *P = theta + tc_off_node(l);
    const float *W3 = P, *W4 = P + TC_N * 11 + TC_N;
    for (int idx = tid; idx < TC_N * TN_K1; idx += TC_M) {
        const int r = idx / TN_K1, k = idx % TN_K1;
        *(uint16_t *)(sB1 + tc_off16(r, k)) = tc_bf16(k < 11 ? W3[r * 11 + k] : 0.0f);
    }
    for (int idx = tid; idx < TN_N2 * TC_K; idx += TC_M) {
        const int f = idx / TC_K, k = idx % TC_K;
        *(uint16_t *)(sB2 + tc_off(f, k)) = tc_bf16(f < 9 ? W4[f * TC_N + k] : 0.0f);
    }
    if (tid < TC_N) b3[tid] = P[TC_N * 11 + tid];
    if (tid < TN_N2) b4[tid] = (tid < 9) ? P[TC_N * 11 + TC_N + 9 * TC_N + tid] : 0.0f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                     "r"(TN_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t a1 = (uint32_t)__cvta_generic_to_shared(sA1), bb1 = (uint32_t)__cvta_generic_to_shared(sB1);
    const uint32_t a2 = (uint32_t)__cvta_generic_to_shared(sA2), bb2 = (uint32_t)__cvta_generic_to_shared(sB2);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16; // this warp's TMEM lanes
    uint32_t phase = 0;
    const int64_t ntiles = (n + TC_M - 1) / TC_M;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t v = tile * TC_M + tid;
        const bool valid = v < n;
        float u[TN_K1];
#pragma unroll
        for (int f = 0; f < TN_K1; ++f) u[f] = 0.0f;
        if (valid) {
            float S, M;
            gnn_aggregate(v, Lrowptr, Urowptr, tperm, e, S, M);
#pragma unroll
            for (int f = 0; f < 9; ++f) u[f] = x[9 * v + f];
            u[9] = S;
            u[10] = M;
        }
        *(uint4 *)(sA1 + tc_off16(tid, 0)) =
            make_uint4(tc_pack(u[0], u[1]), tc_pack(u[2], u[3]), tc_pack(u[4], u[5]), tc_pack(u[6], u[7]));
        *(uint4 *)(sA1 + tc_off16(tid, 8)) =
            make_uint4(tc_pack(u[8], u[9]), tc_pack(u[10], u[11]), tc_pack(u[12], u[13]), tc_pack(u[14], u[15]));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint64_t ad = tc_desc(a1, 256), bd = tc_desc(bb1, 256);
            asm volatile("{\n\t.reg .pred acc;\n\t"
                         "setp.ne.b32 acc, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, acc;\n\t}" ::"r"(tmem),
                         "l"(ad), "l"(bd), "r"(TN_IDESC1), "r"(0));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        const bool ok1 = tc_wait(mb, phase, err);
        phase ^= 1u;
        if (!__syncthreads_and(ok1)) break; // the accumulator may still be written: stop using it
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                     "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                       "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                       "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(tmem + lane_base));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float a[TC_N];
#pragma unroll
        for (int k = 0; k < TC_N; ++k) a[k] = tanhf(__uint_as_float(r[k]) + b3[k]); // rounded to BF16 next
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *(uint4 *)(sA2 + tc_off(tid, 8 * c)) =
                make_uint4(tc_pack(a[8 * c], a[8 * c + 1]), tc_pack(a[8 * c + 2], a[8 * c + 3]),
                           tc_pack(a[8 * c + 4], a[8 * c + 5]), tc_pack(a[8 * c + 6], a[8 * c + 7]));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const uint64_t ad = tc_desc(a2 + s2 * 256), bd = tc_desc(bb2 + s2 * 256);
                asm volatile("{\n\t.reg .pred acc;\n\t"
                             "setp.ne.b32 acc, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, acc;\n\t}" ::"r"(tmem + 32u),
                             "l"(ad), "l"(bd), "r"(TN_IDESC2), "r"(s2));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        const bool ok2 = tc_wait(mb, phase, err);
        phase ^= 1u;
        if (!__syncthreads_and(ok2)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t o[16];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                     "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                     : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]),
                       "=r"(o[7]), "=r"(o[8]), "=r"(o[9]), "=r"(o[10]), "=r"(o[11]), "=r"(o[12]), "=r"(o[13]),
                       "=r"(o[14]), "=r"(o[15])
                     : "r"(tmem + lane_base + 32u));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid) {
#pragma unroll
            for (int f = 0; f < 9; ++f) xout[9 * v + f] = __uint_as_float(o[f]) + b4[f];
        }
        // every thread's TMEM reads (and the tile's shared-memory reads by the
        // MMAs) finish before the next tile overwrites them
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN_COLS));
}

int node_fwd_tc(gic_handle *h, int64_t n, const int32_t *Lrowptr, const int32_t *Urowptr, const int32_t *tperm,
                const float *e, const float *x, const float *theta, int l, float *xout)
{
    // up to 8 CTAs per SM (8 x 64 TMEM columns = the SM's 512)
    int64_t tiles = (n + TC_M - 1) / TC_M, cap = (int64_t)h->num_sms * 8;
    if (tiles > cap) tiles = cap;
    if (tiles < 1) tiles = 1;
    ++h->launches;
    k_node_fwd_tc<<<(unsigned)tiles, TC_M, 0, h->stream>>>(n, Lrowptr, Urowptr, tperm, e, x, theta, l, xout,
                                                           h->dev_err);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

}  // namespace gic
