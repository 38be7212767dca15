// gic_gnn.cu -- A4-A6, A8-A10: graph inputs, the GNN correction of L, the
// probe loss and its gradient, the GNN backward pass and Adam.
//
// Graph (Model Architecture; Supplementary 3): nodes = rows, edges = the
// entries of tril(A) (diagonal included), edge p = (i = row, j = column).
// Inputs (Model Architecture; Supplementary 4): e0 = a_ij / s (s = population
// standard deviation of tril(A)'s values), x = 9 node features, GraphNorm on
// x. Three message-passing blocks (Eq.(7)-(9)): edge MLP 20 -> 32 -> 1 with
// tanh on [e_cur, e0, x_i, x_j]; sum and mean of the new edge values over
// the edges incident to each node; node MLP 11 -> 32 -> 9 with tanh on
// [x, sum, mean]; no node update in the last block. Output g on the edges.
// Correction (Eq.(2) with the exp-then-sqrt diagonal map): off-diagonal
// L = L_IC + sqrt(s) g, diagonal L = L_IC exp(g / 2) (in units scaled by s:
// Lhat = LhatIC + g and LhatIC exp(g / 2)).
// Probe loss (Eq.(4)-(5), Algorithms 1-2), scaled units, per graph
//   (1/m) sum_k || Lhat (Lhat^T z_k) - Ahat z_k ||^2, averaged over graphs.
//
// A batch is a block-diagonal pattern of `ngraphs` equal-size graphs; every
// per-graph statistic (s, GraphNorm, loss) is reduced per graph.
// All reductions are deterministic (per-block partials summed in order).
// Flat parameter layout (3504 float32, shared with the checkpoint format):
//   GraphNorm gamma[9], beta[9], alpha[9]; then for l = 0,1,2: edge
//   W1[32][20], b1[32], W2[32], b2; and for l = 0,1: node W3[32][11], b3[32],
//   W4[9][32], b4[9].
#include <math.h>

#include <cuda_bf16.h>

#include "gic_internal.cuh"

namespace gic {

// x rounded to the nearest BF16 (ties to even), back in FP32
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

constexpr int H = 32;
constexpr int NP_GN = 27;
constexpr int NP_EDGE = H * 20 + H + H + 1;
constexpr int NP_NODE = H * 11 + H + 9 * H + 9;
constexpr int NP_TOTAL = NP_GN + 3 * NP_EDGE + 2 * NP_NODE;
__host__ __device__ constexpr int off_edge(int l) { return NP_GN + l * (NP_EDGE + NP_NODE); }
__host__ __device__ constexpr int off_node(int l) { return off_edge(l) + NP_EDGE; }
static_assert(NP_TOTAL == 3504, "parameter layout");

constexpr int GX = 64;        // blocks per graph in per-graph reductions
constexpr int RB = 256;       // threads of reduction blocks
constexpr int TB = 128;       // threads (= edges or nodes per tile) of backward blocks

static size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

__device__ __forceinline__ double block_sum_d(double v, double *sh)
{
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    return s; // thread 0
}

// ------------------------------------------------------------ A4 features
// pass 0: sum of tril values per graph; pass 1: sum of squared deviations.
// Sums over graph g's lower-triangle entries of A (pass 0: values; pass 1:
// squared deviations from the mean): eight lanes per row (a row's lower
// entries are the first Lrowptr[i+1] - Lrowptr[i] of its A entries; full
// sectors, several loads in flight per lane), rows strided over the grid.
__global__ void k_tril_moments(int pass, int64_t ng, const int32_t *rowptr, const int32_t *Lrowptr,
                               const double *valA, const double *mean, double *partials)
{
    __shared__ double sh[RB / 32];
    const int g = blockIdx.y;
    const int64_t r0 = (int64_t)g * ng;
    const double mu = pass ? mean[g] : 0.0;
    const int sl = threadIdx.x & 7;
    const int64_t q0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int64_t nq = ((int64_t)gridDim.x * blockDim.x) >> 3;
    double acc = 0.0;
    for (int64_t i = r0 + q0; i < r0 + ng; i += nq) {
        const int32_t a = rowptr[i], cnt = Lrowptr[i + 1] - Lrowptr[i];
#pragma unroll 4
        for (int32_t k = sl; k < cnt; k += 8) {
            const double v = valA[a + k];
            acc += pass ? (v - mu) * (v - mu) : v;
        }
    }
    double s = block_sum_d(acc, sh);
    if (threadIdx.x == 0) partials[g * gridDim.x + blockIdx.x] = s;
}

__global__ void k_tril_finish(int pass, int64_t ng, const int32_t *Lrowptr, const double *partials, int nparts,
                              double *mean, double *scale)
{
    const int g = blockIdx.x;
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < nparts; ++k) s += partials[g * nparts + k];
    double cnt = (double)(Lrowptr[(int64_t)(g + 1) * ng] - Lrowptr[(int64_t)g * ng]);
    if (pass == 0) mean[g] = s / cnt;
    else scale[g] = sqrt(s / cnt);
}

// x9 per node: a warp takes 32 consecutive rows, four at a time with eight
// lanes per row (a row's entries across its lanes: full sectors, loads of
// several entries in flight per lane), the statistics reduced over the
// eight lanes and handed to the lane numbered like the row; then every
// lane finishes its own row (the divisions and the FP64 sin / cos run
// lane-parallel). Features: degree (off-diagonal count), max / min / mean /
// variance of the neighbours' degrees, diagonal dominance |a_ii| / sum
// |a_ij| and |a_ii| / max |a_ij| (j != i), and the position encoding sin /
// cos of the row's index within its graph. The degree statistics are exact
// integer sums (the variance as (cnt sum d^2 - (sum d)^2) / cnt^2, the
// exact value of the mean squared deviation), so only the |a_ij| sum costs
// an FP64 operation per entry (FP64 is this GPU's scarce pipe); positive
// doubles compare like their bit patterns, so their maximum is an integer
// maximum.
__global__ void k_features(int64_t n, int64_t ng, const int32_t *rowptr, const int32_t *col, const double *valA,
                           float *x9)
{
    const int lane = threadIdx.x & 31, sub = lane >> 3, sl = lane & 7;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = w0 * 32; base < n; base += nw * 32) {
        int m_dmax = 0, m_dmin = 0, m_cnt = 0, m_len = 0;
        long long m_dsum = 0, m_dsq = 0, m_diag = 0, m_offmax = 0;
        double m_offsum = 0.0;
        const int rows = (int)((n - base < 32) ? (n - base) : 32);
        for (int r0 = 0; r0 < rows; r0 += 4) {
            const int r = r0 + sub;
            const int64_t i = base + r;
            const bool on = r < rows;
            const int32_t a = on ? rowptr[i] : 0, b = on ? rowptr[i + 1] : 0;
            int dmax = -1, dmin = 0x7fffffff, cnt = 0;
            long long dsum = 0, dsq = 0, diag = 0, offmax = 0; // |a| as its bit pattern
            double offsum = 0.0;
#pragma unroll 4
            for (int32_t p = a + sl; p < b; p += 8) {
                const int32_t j = col[p];
                const double v = fabs(valA[p]);
                const long long vb = __double_as_longlong(v);
                if (j == i) {
                    diag = vb;
                } else {
                    const int dj = rowptr[j + 1] - rowptr[j] - 1;
                    dmax = max(dmax, dj);
                    dmin = min(dmin, dj);
                    dsum += dj;
                    dsq += (long long)dj * dj;
                    ++cnt;
                    offsum += v;
                    offmax = max(offmax, vb);
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                dsq += __shfl_xor_sync(0xffffffffu, dsq, o);
                diag = max(diag, __shfl_xor_sync(0xffffffffu, diag, o));
                offmax = max(offmax, __shfl_xor_sync(0xffffffffu, offmax, o));
                offsum += __shfl_xor_sync(0xffffffffu, offsum, o);
            }
            const int len = b - a;
#pragma unroll
            for (int q = 0; q < 4; ++q) { // row r0 + q's statistics (held by lanes 8q..8q+7) to lane r0 + q
                const int t0 = __shfl_sync(0xffffffffu, dmax, 8 * q), t1 = __shfl_sync(0xffffffffu, dmin, 8 * q);
                const int t2 = __shfl_sync(0xffffffffu, cnt, 8 * q), t3 = __shfl_sync(0xffffffffu, len, 8 * q);
                const long long t4 = __shfl_sync(0xffffffffu, dsum, 8 * q), t5 = __shfl_sync(0xffffffffu, dsq, 8 * q);
                const long long t6 = __shfl_sync(0xffffffffu, diag, 8 * q);
                const long long t7 = __shfl_sync(0xffffffffu, offmax, 8 * q);
                const double t8 = __shfl_sync(0xffffffffu, offsum, 8 * q);
                if (lane == r0 + q) {
                    m_dmax = t0; m_dmin = t1; m_cnt = t2; m_len = t3;
                    m_dsum = t4; m_dsq = t5; m_diag = t6; m_offmax = t7; m_offsum = t8;
                }
            }
        }
        if (lane < rows) {
            const int64_t i = base + lane;
            double sn, cs;
            sincos((double)(i % ng), &sn, &cs);
            float *xv = x9 + 9 * i;
            const double c = (double)m_cnt, diag = __longlong_as_double(m_diag);
            const double offmax = __longlong_as_double(m_offmax);
            xv[0] = (float)(m_len - 1);
            xv[1] = (float)(m_cnt ? m_dmax : 0);
            xv[2] = (float)(m_cnt ? m_dmin : 0);
            xv[3] = (float)(m_cnt ? (double)m_dsum / c : 0.0);
            xv[4] = (float)(m_cnt ? (double)(m_cnt * m_dsq - m_dsum * m_dsum) / (c * c) : 0.0);
            xv[5] = (float)(m_offsum > 0 ? diag / m_offsum : 0.0);
            xv[6] = (float)(offmax > 0 ? diag / offmax : 0.0);
            xv[7] = (float)sn;
            xv[8] = (float)cs;
        }
    }
}

// e0 = tril(A) / s per lower entry (one thread per entry), and, if asked,
// Ahat = A / s per entry of A; s of the entry's graph (rows g ng ..).
__global__ void k_scaled_values(int64_t nnzL, int64_t nnzA, int64_t ng, int ngraphs, const int32_t *rowptr,
                                const int32_t *Lrowptr, const int32_t *Lrow, const double *valA, const double *scale,
                                float *e0, float *Ahat)
{
    __shared__ double inv[64];
    for (int k = threadIdx.x; k < ngraphs && k < 64; k += blockDim.x) inv[k] = 1.0 / scale[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnzL; e += stride) {
        const int32_t i = Lrow[e];
        const int gi = (ngraphs == 1) ? 0 : (int)(i / ng);
        const double r = (gi < 64) ? inv[gi] : 1.0 / scale[gi];
        e0[e] = (float)(valA[rowptr[i] + (e - Lrowptr[i])] * r);
    }
    if (!Ahat) return;
    // graph boundaries in A's entries: graph k owns rowptr[k ng] ..
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnzA; p += stride) {
        int gi = 0;
        while (gi + 1 < ngraphs && rowptr[(int64_t)(gi + 1) * ng] <= p) ++gi;
        const double r = (gi < 64) ? inv[gi] : 1.0 / scale[gi];
        Ahat[p] = (float)(valA[p] * r);
    }
}

// ------------------------------------------------------------ GraphNorm
// pass 0: per-graph feature sums; pass 1: sums of (x - alpha mu)^2.
__global__ void k_gn_moments(int pass, int64_t ng, const float *x9, const float *theta, const double *mu,
                             double *partials)
{
    __shared__ double sh[9][RB / 32 + 1];
    const int g = blockIdx.y;
    const int64_t v0 = (int64_t)g * ng;
    double acc[9];
    for (int f = 0; f < 9; ++f) acc[f] = 0.0;
    for (int64_t v = v0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < v0 + ng; v += (int64_t)gridDim.x * blockDim.x) {
        for (int f = 0; f < 9; ++f) {
            double x = x9[9 * v + f];
            if (pass) {
                double c = x - (double)theta[18 + f] * mu[9 * g + f];
                acc[f] += c * c;
            } else {
                acc[f] += x;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int f = 0; f < 9; ++f) {
        double t = warp_sum(acc[f]);
        if (lane == 0) sh[f][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[threadIdx.x][k];
        partials[(g * gridDim.x + blockIdx.x) * 9 + threadIdx.x] = s;
    }
}

__global__ void k_gn_finish(int pass, int64_t ng, const double *partials, int nparts, double *mu, double *sig)
{
    const int g = blockIdx.x, f = threadIdx.x;
    if (f >= 9) return;
    double s = 0.0;
    for (int k = 0; k < nparts; ++k) s += partials[(g * nparts + k) * 9 + f];
    if (pass == 0) mu[9 * g + f] = s / (double)ng;
    else sig[9 * g + f] = sqrt(s / (double)ng + 1e-5);
}

__global__ void k_gn_apply(int64_t n, int64_t ng, int ngraphs, const float *x9, const float *theta,
                           const double *mu, const double *sig, float *x0)
{
    // per graph and feature: alpha mu and gamma / sigma (one division each)
    __shared__ double am[16 * 9], gs[16 * 9];
    for (int k = threadIdx.x; k < 9 * ngraphs && k < 16 * 9; k += blockDim.x) {
        const int f = k % 9;
        am[k] = (double)theta[18 + f] * mu[k];
        gs[k] = (double)theta[f] / sig[k];
    }
    __syncthreads();
    // one node per thread, its nine features contiguous
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int g = (ngraphs == 1) ? 0 : (int)(v / ng);
#pragma unroll
        for (int f = 0; f < 9; ++f) {
            const int k = 9 * g + f;
            const double a = (g < 16) ? am[k] : (double)theta[18 + f] * mu[k];
            const double q = (g < 16) ? gs[k] : (double)theta[f] / sig[k];
            const double c = (double)x9[9 * v + f] - a;
            x0[9 * v + f] = (float)(q * c + (double)theta[9 + f]);
        }
    }
}

// ------------------------------------------------------------ A5 forward
// Edge MLP, FP32: eout = W2 tanh(W1 [ein, e0, x_i, x_j] + b1) + b2.
__global__ void __launch_bounds__(256) k_edge_fwd(int64_t E, const int32_t *__restrict__ Lrow,
                                                  const int32_t *__restrict__ Lcol, const float *__restrict__ ein,
                                                  const float *__restrict__ e0, const float *__restrict__ x,
                                                  const float *__restrict__ theta, int l, float *__restrict__ eout)
{
    __shared__ float W1[H * 20], b1[H], W2[H], b2;
    const float *P = theta + off_edge(l);
    for (int t = threadIdx.x; t < H * 20; t += blockDim.x) W1[t] = P[t];
    if (threadIdx.x < H) {
        b1[threadIdx.x] = P[H * 20 + threadIdx.x];
        W2[threadIdx.x] = P[H * 20 + H + threadIdx.x];
    }
    if (threadIdx.x == 0) b2 = P[H * 20 + 2 * H];
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = Lrow[p], j = Lcol[p];
        float h[20];
        h[0] = ein[p];
        h[1] = e0[p];
#pragma unroll
        for (int f = 0; f < 9; ++f) {
            h[2 + f] = x[9 * i + f];
            h[11 + f] = x[9 * j + f];
        }
        float out = b2;
#pragma unroll 4
        for (int u = 0; u < H; ++u) {
            float z = b1[u];
#pragma unroll
            for (int f = 0; f < 20; ++f) z = fmaf(W1[u * 20 + f], h[f], z);
            out = fmaf(W2[u], tanhf(z), out);
        }
        eout[p] = out;
    }
}

// sum / mean aggregation of edge values at node v: its L row, then the
// off-diagonal entries of its U row (edges (i, v), i > v).
// Node MLP: xout = W4 tanh(W3 [x, S, M] + b3) + b4. Saves S, M if asked.
__global__ void __launch_bounds__(256) k_node_fwd(int64_t n, const int32_t *__restrict__ Lrowptr,
                                                  const int32_t *__restrict__ Urowptr, const int32_t *__restrict__ tperm,
                                                  const float *__restrict__ e, const float *__restrict__ x,
                                                  const float *__restrict__ theta, int l, float *__restrict__ xout,
                                                  float *Ssave, float *Msave)
{
    __shared__ float W3[H * 11], b3[H], W4[9 * H], b4[9];
    const float *P = theta + off_node(l);
    for (int t = threadIdx.x; t < H * 11; t += blockDim.x) W3[t] = P[t];
    for (int t = threadIdx.x; t < 9 * H; t += blockDim.x) W4[t] = P[H * 11 + H + t];
    if (threadIdx.x < H) b3[threadIdx.x] = P[H * 11 + threadIdx.x];
    if (threadIdx.x < 9) b4[threadIdx.x] = P[H * 11 + H + 9 * H + threadIdx.x];
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        float S, M;
        gnn_aggregate(v, Lrowptr, Urowptr, tperm, e, S, M);
        if (Ssave) {
            Ssave[v] = S;
            Msave[v] = M;
        }
        float u[11];
#pragma unroll
        for (int f = 0; f < 9; ++f) u[f] = x[9 * v + f];
        u[9] = S;
        u[10] = M;
        float o[9];
#pragma unroll
        for (int f = 0; f < 9; ++f) o[f] = b4[f];
        for (int k = 0; k < H; ++k) {
            float z = b3[k];
#pragma unroll
            for (int f = 0; f < 11; ++f) z = fmaf(W3[k * 11 + f], u[f], z);
            const float a = tanhf(z);
#pragma unroll
            for (int f = 0; f < 9; ++f) o[f] = fmaf(W4[f * H + k], a, o[f]);
        }
#pragma unroll
        for (int f = 0; f < 9; ++f) xout[9 * v + f] = o[f];
    }
}

// ------------------------------------------------------------ A6 correction
// Original units, FP64 factor: off-diagonal LIC + sqrt(s) g, diagonal
// LIC exp(g/2). bad |= 1 if a diagonal is not positive and finite.
__global__ void k_correct(int64_t E, int64_t ng, int ngraphs, const int32_t *Lrow, const int32_t *Lcol,
                          const double *LIC, const float *g, const double *scale, double *Lout, unsigned *bad)
{
    __shared__ double sq[64]; // sqrt(s) per graph, once per block
    for (int k = threadIdx.x; k < ngraphs && k < 64; k += blockDim.x) sq[k] = sqrt(scale[k]);
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = Lrow[p];
        const double gp = (double)g[p];
        if (Lcol[p] != i) { // the diagonals follow in k_correct_diag (their exp would diverge every warp)
            const int gi = (ngraphs == 1) ? 0 : (int)(i / ng);
            const double r = (gi < 64) ? sq[gi] : sqrt(scale[gi]);
            Lout[p] = LIC[p] + r * gp;
            if (!isfinite(Lout[p])) atomicOr(bad, 1u);
        }
    }
}

// The correction's diagonal entries, one thread per row (the diagonal is
// the last entry of each L row): L_ii = L_IC,ii exp(g_ii / 2).
__global__ void k_correct_diag(int64_t n, const int32_t *Lrowptr, const double *LIC, const float *g, double *Lout,
                               unsigned *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = Lrowptr[i + 1] - 1;
        const double d = LIC[p] * exp((double)g[p] / 2.0);
        Lout[p] = d;
        if (!(d > 0.0) || !isfinite(d)) atomicOr(bad, 1u);
    }
}

// Scaled units, FP32 (training): Lhat = LhatIC + g, diagonal LhatIC exp(g/2).
__global__ void k_correct_scaled(int64_t E, const int32_t *Lrow, const int32_t *Lcol, const float *LIC, const float *g,
                                 float *Lout)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x)
        Lout[p] = (Lcol[p] == Lrow[p]) ? LIC[p] * expf(0.5f * g[p]) : LIC[p] + g[p];
}

// dg from dLhat through the correction.
__global__ void k_correct_bwd(int64_t E, const int32_t *Lrow, const int32_t *Lcol, const float *Lhat, const float *dL,
                              float *dg)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x)
        dg[p] = (Lcol[p] == Lrow[p]) ? dL[p] * 0.5f * Lhat[p] : dL[p];
}

// LhatIC = LIC / sqrt(s) per graph, FP32.
__global__ void k_scale_factor(int64_t E, int64_t ng, int ngraphs, const int32_t *Lrow, const double *LIC,
                               const double *scale, float *out)
{
    __shared__ double sq[64]; // sqrt(s) per graph, once per block
    for (int k = threadIdx.x; k < ngraphs && k < 64; k += blockDim.x) sq[k] = sqrt(scale[k]);
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int g = (ngraphs == 1) ? 0 : (int)((uint32_t)Lrow[p] / (uint32_t)ng); // rows and ng fit 32 bits
        out[p] = (float)(LIC[p] / ((g < 64) ? sq[g] : sqrt(scale[g])));
    }
}

// ------------------------------------------------------------ A8 probe loss
__global__ void k_gather_f32(int64_t cnt, const int32_t *perm, const float *src, float *dst)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = src[perm[q]];
}

// out[k][j] = sum_{q in U row j} U[q] in[k][Ucol[q]]  (= (L^T in_k)_j), k < m
__global__ void k_ut_mult(int64_t n, int m, const int32_t *Urowptr, const int32_t *Ucol, const float *U,
                          const float *in, float *out)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        float acc[16];
        for (int k = 0; k < m; ++k) acc[k] = 0.f;
        for (int32_t q = Urowptr[j]; q < Urowptr[j + 1]; ++q) {
            const float u = U[q];
            const int64_t c = Ucol[q];
            for (int k = 0; k < m; ++k) acc[k] = fmaf(u, in[(int64_t)k * n + c], acc[k]);
        }
        for (int k = 0; k < m; ++k) out[(int64_t)k * n + j] = acc[k];
    }
}

// v[k][i] = (L u_k)_i - (A z_k)_i ; per-graph partial of sum_k v^2
__global__ void k_loss_v(int64_t ng, int m, const int32_t *rowptr, const int32_t *col, const float *Ahat,
                         const int32_t *Lrowptr, const int32_t *Lcol, const float *Lhat, const float *Z,
                         const float *u, float *v, int64_t n, double *partials)
{
    __shared__ double sh[RB / 32];
    const int g = blockIdx.y;
    const int64_t r0 = (int64_t)g * ng;
    double acc = 0.0;
    for (int64_t i = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < r0 + ng; i += (int64_t)gridDim.x * blockDim.x) {
        float s[16];
        for (int k = 0; k < m; ++k) s[k] = 0.f;
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
            const float l = Lhat[p];
            const int64_t c = Lcol[p];
            for (int k = 0; k < m; ++k) s[k] = fmaf(l, u[(int64_t)k * n + c], s[k]);
        }
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const float a = Ahat[p];
            const int64_t c = col[p];
            for (int k = 0; k < m; ++k) s[k] = fmaf(-a, Z[(int64_t)k * n + c], s[k]);
        }
        for (int k = 0; k < m; ++k) {
            v[(int64_t)k * n + i] = s[k];
            acc += (double)s[k] * (double)s[k];
        }
    }
    double t = block_sum_d(acc, sh);
    if (threadIdx.x == 0) partials[g * gridDim.x + blockIdx.x] = t;
}

// loss[g] = partial sum / m ; loss[ngraphs] = mean over graphs
__global__ void k_loss_finish(int ngraphs, int m, const double *partials, int nparts, float *loss)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot = 0.0;
    for (int g = 0; g < ngraphs; ++g) {
        double s = 0.0;
        for (int k = 0; k < nparts; ++k) s += partials[g * nparts + k];
        s /= m;
        loss[g] = (float)s;
        tot += s;
    }
    loss[ngraphs] = (float)(tot / ngraphs);
}

// dL[p] = c sum_k (v_k[i] u_k[j] + z_k[i] w_k[j])
__global__ void k_loss_grad(int64_t E, int m, int64_t n, const int32_t *Lrow, const int32_t *Lcol, const float *u,
                            const float *v, const float *Z, const float *w, float c, float *dL)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = Lrow[p], j = Lcol[p];
        float s = 0.f;
        for (int k = 0; k < m; ++k) {
            const int64_t o = (int64_t)k * n;
            s = fmaf(v[o + i], u[o + j], s);
            s = fmaf(Z[o + i], w[o + j], s);
        }
        dL[p] = c * s;
    }
}

// ------------------------------------------------------------ A9 backward
// Edge MLP backward for a tile of TB edges per step. Recomputes the hidden
// layer; writes dh (the 18 node parts of d h) and dec = d e_in; accumulates
// the 705 weight-gradient sums of this block into partials[block][*].
__global__ void __launch_bounds__(TB) k_edge_bwd(int64_t E, const int32_t *__restrict__ Lrow,
                                                 const int32_t *__restrict__ Lcol, const float *__restrict__ ein,
                                                 const float *__restrict__ e0, const float *__restrict__ x,
                                                 const float *__restrict__ theta, int l, const float *__restrict__ de,
                                                 float *__restrict__ dh, float *__restrict__ dec,
                                                 double *__restrict__ partials, bool bf16)
{
    __shared__ float W1[H * 20], b1[H], W2[H];
    __shared__ float s_dz[TB][H + 1];
    __shared__ float s_ad[TB][H + 1];
    __shared__ float s_h[TB][21];
    const float *P = theta + off_edge(l);
    // BF16 training: the forward's rounding of W1 and of the inputs h is
    // redone here, and the gradient passes straight through it
    for (int t = threadIdx.x; t < H * 20; t += blockDim.x) W1[t] = bf16 ? round_bf16(P[t]) : P[t];
    if (threadIdx.x < H) {
        b1[threadIdx.x] = P[H * 20 + threadIdx.x];
        W2[threadIdx.x] = P[H * 20 + H + threadIdx.x];
    }
    __syncthreads();
    // outputs owned by this thread: o = threadIdx.x + k*TB, k < 6 (705 total)
    double acc[6]; // across tiles in FP64 (one add per tile and output)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = 0.0;
    const int64_t ntiles = (E + TB - 1) / TB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = tile * TB + threadIdx.x;
        const bool valid = p < E;
        float h[20];
        float d = 0.f;
        if (valid) {
            const int64_t i = Lrow[p], j = Lcol[p];
            h[0] = ein[p];
            h[1] = e0[p];
#pragma unroll
            for (int f = 0; f < 9; ++f) {
                h[2 + f] = x[9 * i + f];
                h[11 + f] = x[9 * j + f];
            }
            d = de[p];
            if (bf16) {
#pragma unroll
                for (int f = 0; f < 20; ++f) h[f] = round_bf16(h[f]);
            }
        } else {
#pragma unroll
            for (int f = 0; f < 20; ++f) h[f] = 0.f;
        }
        float dhl[20];
#pragma unroll
        for (int f = 0; f < 20; ++f) dhl[f] = 0.f;
        for (int u = 0; u < H; ++u) {
            float z = b1[u];
#pragma unroll
            for (int f = 0; f < 20; ++f) z = fmaf(W1[u * 20 + f], h[f], z);
            const float a = tanhf(z);
            const float dz = d * W2[u] * (1.f - a * a);
            s_dz[threadIdx.x][u] = dz;
            s_ad[threadIdx.x][u] = d * a;
#pragma unroll
            for (int f = 0; f < 20; ++f) dhl[f] = fmaf(W1[u * 20 + f], dz, dhl[f]);
        }
#pragma unroll
        for (int f = 0; f < 20; ++f) s_h[threadIdx.x][f] = h[f];
        s_h[threadIdx.x][20] = d;
        if (valid) {
            dec[p] = dhl[0];
#pragma unroll
            for (int f = 0; f < 18; ++f) dh[18 * p + f] = dhl[2 + f];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int o = threadIdx.x + k * TB;
            if (o >= NP_EDGE) break;
            float s = 0.f;
            if (o < H * 20) { // dW1[u][f] = sum dz[u] h[f]
                const int u = o / 20, f = o % 20;
                for (int t = 0; t < TB; ++t) s = fmaf(s_dz[t][u], s_h[t][f], s);
            } else if (o < H * 21) { // db1
                const int u = o - H * 20;
                for (int t = 0; t < TB; ++t) s += s_dz[t][u];
            } else if (o < H * 22) { // dW2
                const int u = o - H * 21;
                for (int t = 0; t < TB; ++t) s += s_ad[t][u];
            } else { // db2
                for (int t = 0; t < TB; ++t) s += s_h[t][20];
            }
            acc[k] += (double)s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int o = threadIdx.x + k * TB;
        if (o < NP_EDGE) partials[(int64_t)blockIdx.x * NP_EDGE + o] = acc[k];
    }
}

// Node MLP backward for a tile of TB nodes per step. Given dxo = d x_{l+1},
// writes dxd (direct part of d x_l), dS, dM and the 681 weight sums.
__global__ void __launch_bounds__(TB) k_node_bwd(int64_t n, const float *__restrict__ x, const float *__restrict__ S,
                                                 const float *__restrict__ M, const float *__restrict__ theta, int l,
                                                 const float *__restrict__ dxo, float *__restrict__ dxd,
                                                 float *__restrict__ dS, float *__restrict__ dM,
                                                 double *__restrict__ partials)
{
    __shared__ float W3[H * 11], b3[H], W4[9 * H];
    __shared__ float s_dz[TB][H + 1];
    __shared__ float s_a[TB][H + 1];
    __shared__ float s_u[TB][12];
    __shared__ float s_dx[TB][10];
    const float *P = theta + off_node(l);
    for (int t = threadIdx.x; t < H * 11; t += blockDim.x) W3[t] = P[t];
    for (int t = threadIdx.x; t < 9 * H; t += blockDim.x) W4[t] = P[H * 11 + H + t];
    if (threadIdx.x < H) b3[threadIdx.x] = P[H * 11 + threadIdx.x];
    __syncthreads();
    double acc[6]; // across tiles in FP64 (one add per tile and output)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = 0.0;
    const int64_t ntiles = (n + TB - 1) / TB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t v = tile * TB + threadIdx.x;
        const bool valid = v < n;
        float u[11], dx[9];
        if (valid) {
#pragma unroll
            for (int f = 0; f < 9; ++f) {
                u[f] = x[9 * v + f];
                dx[f] = dxo[9 * v + f];
            }
            u[9] = S[v];
            u[10] = M[v];
        } else {
#pragma unroll
            for (int f = 0; f < 11; ++f) u[f] = 0.f;
#pragma unroll
            for (int f = 0; f < 9; ++f) dx[f] = 0.f;
        }
        float du[11];
#pragma unroll
        for (int f = 0; f < 11; ++f) du[f] = 0.f;
        for (int k = 0; k < H; ++k) {
            float z = b3[k];
#pragma unroll
            for (int f = 0; f < 11; ++f) z = fmaf(W3[k * 11 + f], u[f], z);
            const float a = tanhf(z);
            float da = 0.f;
#pragma unroll
            for (int f = 0; f < 9; ++f) da = fmaf(W4[f * H + k], dx[f], da);
            const float dz = da * (1.f - a * a);
            s_dz[threadIdx.x][k] = dz;
            s_a[threadIdx.x][k] = a;
#pragma unroll
            for (int f = 0; f < 11; ++f) du[f] = fmaf(W3[k * 11 + f], dz, du[f]);
        }
#pragma unroll
        for (int f = 0; f < 11; ++f) s_u[threadIdx.x][f] = u[f];
#pragma unroll
        for (int f = 0; f < 9; ++f) s_dx[threadIdx.x][f] = dx[f];
        if (valid) {
#pragma unroll
            for (int f = 0; f < 9; ++f) dxd[9 * v + f] = du[f];
            dS[v] = du[9];
            dM[v] = du[10];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int o = threadIdx.x + k * TB;
            if (o >= NP_NODE) break;
            float s = 0.f;
            if (o < H * 11) { // dW3[k][f] = sum dz[k] u[f]
                const int kk = o / 11, f = o % 11;
                for (int t = 0; t < TB; ++t) s = fmaf(s_dz[t][kk], s_u[t][f], s);
            } else if (o < H * 12) { // db3
                const int kk = o - H * 11;
                for (int t = 0; t < TB; ++t) s += s_dz[t][kk];
            } else if (o < H * 12 + 9 * H) { // dW4[f][k] = sum dx[f] a[k]
                const int q = o - H * 12, f = q / H, kk = q % H;
                for (int t = 0; t < TB; ++t) s = fmaf(s_dx[t][f], s_a[t][kk], s);
            } else { // db4
                const int f = o - H * 12 - 9 * H;
                for (int t = 0; t < TB; ++t) s += s_dx[t][f];
            }
            acc[k] += (double)s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int o = threadIdx.x + k * TB;
        if (o < NP_NODE) partials[(int64_t)blockIdx.x * NP_NODE + o] = acc[k];
    }
}

// de[p] = dec[p] + dS_i + dM_i/deg_i (+ the same at j for an off-diagonal edge)
__global__ void k_agg_bwd(int64_t E, const int32_t *Lrow, const int32_t *Lcol, const int32_t *Lrowptr,
                          const int32_t *Urowptr, const float *dec, const float *dS, const float *dM, float *de)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = Lrow[p], j = Lcol[p];
        const float di = (float)((Lrowptr[i + 1] - Lrowptr[i]) + (Urowptr[i + 1] - Urowptr[i]) - 1);
        float s = dec[p] + dS[i] + dM[i] / di;
        if (j != i) {
            const float dj = (float)((Lrowptr[j + 1] - Lrowptr[j]) + (Urowptr[j + 1] - Urowptr[j]) - 1);
            s += dS[j] + dM[j] / dj;
        }
        de[p] = s;
    }
}

// dx[v] = dxd[v] + sum over L row v of the i-parts + sum over U row v of the
// j-parts of dh.
__global__ void k_dx_gather(int64_t n, const int32_t *Lrowptr, const int32_t *Urowptr, const int32_t *tperm,
                            const float *dh, const float *dxd, float *dx)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        float s[9];
#pragma unroll
        for (int f = 0; f < 9; ++f) s[f] = dxd ? dxd[9 * v + f] : 0.f;
        for (int32_t p = Lrowptr[v]; p < Lrowptr[v + 1]; ++p)
#pragma unroll
            for (int f = 0; f < 9; ++f) s[f] += dh[18 * (int64_t)p + f];
        for (int32_t q = Urowptr[v]; q < Urowptr[v + 1]; ++q) {
            const int64_t p = tperm[q];
#pragma unroll
            for (int f = 0; f < 9; ++f) s[f] += dh[18 * p + 9 + f];
        }
#pragma unroll
        for (int f = 0; f < 9; ++f) dx[9 * v + f] = s[f];
    }
}

// GraphNorm backward. pass 0: per graph/feature sums of dout, dout*c,
// dout*gamma*c; pass 1: sums of dc.
__global__ void k_gn_bwd_moments(int pass, int64_t ng, const float *x9, const float *theta, const double *mu,
                                 const double *sig, const float *dout, const double *sdsig, double *partials)
{
    __shared__ double sh[27][RB / 32 + 1];
    const int g = blockIdx.y;
    const int64_t v0 = (int64_t)g * ng;
    double acc[27];
    for (int k = 0; k < 27; ++k) acc[k] = 0.0;
    for (int64_t v = v0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < v0 + ng; v += (int64_t)gridDim.x * blockDim.x) {
        for (int f = 0; f < 9; ++f) {
            const double m = mu[9 * g + f], s = sig[9 * g + f], gam = theta[f];
            const double c = (double)x9[9 * v + f] - (double)theta[18 + f] * m;
            const double d = dout[9 * v + f];
            if (pass == 0) {
                acc[f] += d;
                acc[9 + f] += d * c / s;
                acc[18 + f] += d * gam * c * (-1.0 / (s * s));
            } else {
                acc[f] += d * gam / s + sdsig[9 * g + f] * c / ((double)ng * s);
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int K = pass == 0 ? 27 : 9;
    for (int k = 0; k < K; ++k) {
        double t = warp_sum(acc[k]);
        if (lane == 0) sh[k][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[threadIdx.x][w];
        partials[(g * gridDim.x + blockIdx.x) * 27 + threadIdx.x] = s;
    }
}

// pass 0: dbeta, dgamma (summed over graphs) and sdsig per graph;
// pass 1: dalpha = sum_g -mu_g * sum dc.
__global__ void k_gn_bwd_finish(int pass, int ngraphs, const double *partials, int nparts, const double *mu,
                                double *sdsig, float *dtheta)
{
    const int f = threadIdx.x;
    if (f >= 9 || blockIdx.x != 0) return;
    double db = 0.0, dg = 0.0, da = 0.0;
    for (int g = 0; g < ngraphs; ++g) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < nparts; ++k) {
            const double *pp = partials + (g * nparts + k) * 27;
            s0 += pp[f];
            s1 += pp[9 + f];
            s2 += pp[18 + f];
        }
        if (pass == 0) {
            db += s0;
            dg += s1;
            sdsig[9 * g + f] = s2;
        } else {
            da += -mu[9 * g + f] * s0;
        }
    }
    if (pass == 0) {
        dtheta[f] = (float)dg;
        dtheta[9 + f] = (float)db;
    } else {
        dtheta[18 + f] = (float)da;
    }
}

// out[k] = sum over blocks b of partials[b][k], in block order
__global__ void k_reduce_partials(const double *partials, int nblocks, int count, float *out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * count + k];
        out[k] = (float)s;
    }
}

// ------------------------------------------------------------ A10 Adam
__global__ void k_adam(int64_t np, float *theta, const float *grad, float *m1, float *m2, float lr, float c1, float c2)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[k];
        const float a = b1 * m1[k] + (1.f - b1) * g;
        const float b = b2 * m2[k] + (1.f - b2) * g * g;
        m1[k] = a;
        m2[k] = b;
        theta[k] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

// ------------------------------------------------------------ host side
static unsigned grid1(gic_handle *h, int64_t n, int block = 256, int per_sm = 8)
{
    int64_t b = (n + block - 1) / block;
    int64_t cap = (int64_t)h->num_sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

static int check_batch(gic_handle *h, const gic_pattern *P, int ngraphs)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device || ngraphs < 1 || P->p.n % ngraphs != 0) return GIC_ERR_INVALID_ARG;
    if (ngraphs > 4096) return GIC_ERR_UNSUPPORTED;
    return GIC_OK;
}

// Inference workspace: stats, two edge buffers, two node buffers.
struct InferWs {
    double *mu, *sig, *parts;
    float *ea, *eb, *xa, *xb;
    size_t bytes;
};

static InferWs carve_infer(int64_t n, int64_t E, int ngraphs, void *base)
{
    InferWs o = {};
    char *c = (char *)base;
    size_t off = 0;
    o.mu = (double *)(c + off); off += al(8 * 9 * (size_t)ngraphs);
    o.sig = (double *)(c + off); off += al(8 * 9 * (size_t)ngraphs);
    o.parts = (double *)(c + off); off += al(8 * 27 * (size_t)GX * ngraphs);
    o.ea = (float *)(c + off); off += al(4 * (size_t)E);
    o.eb = (float *)(c + off); off += al(4 * (size_t)E);
    o.xa = (float *)(c + off); off += al(4 * 9 * (size_t)n);
    o.xb = (float *)(c + off); off += al(4 * 9 * (size_t)n);
    o.bytes = off;
    return o;
}

size_t gnn_infer_ws_bytes(int64_t n, int64_t nnzL)
{
    // plus what gnn_correct_inplace needs: theta, x9, e0, g, scale, mean, Lout
    return carve_infer(n, nnzL, 1, nullptr).bytes + al(4 * NP_TOTAL) + al(4 * 9 * (size_t)n) +
           3 * al(4 * (size_t)nnzL) + 2 * al(8 * 16) + al(8 * (size_t)nnzL) + al(8 * 2 * GX);
}

static int graphnorm(gic_handle *h, const Pattern &p, int ngraphs, const float *theta, const float *x9, float *x0,
                     double *mu, double *sig, double *parts)
{
    const int64_t ng = p.n / ngraphs;
    dim3 gr(GX, ngraphs);
    ++h->launches;
    k_gn_moments<<<gr, RB, 0, h->stream>>>(0, ng, x9, theta, mu, parts);
    ++h->launches;
    k_gn_finish<<<ngraphs, 32, 0, h->stream>>>(0, ng, parts, GX, mu, sig);
    ++h->launches;
    k_gn_moments<<<gr, RB, 0, h->stream>>>(1, ng, x9, theta, mu, parts);
    ++h->launches;
    k_gn_finish<<<ngraphs, 32, 0, h->stream>>>(1, ng, parts, GX, mu, sig);
    ++h->launches;
    k_gn_apply<<<grid1(h, p.n), 256, 0, h->stream>>>(p.n, ng, ngraphs, x9, theta, mu, sig, x0);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

// Forward pass. x[l] / ein[l] / eout[l] / S[l] / M[l] point at caller
// buffers (training keeps every layer; inference ping-pongs two buffers).
struct FwdBufs {
    float *x[3];
    float *ein[3];
    float *eout[3];
    float *S[2], *M[2];
};

int edge_fwd_tc(gic_handle *h, int64_t E, const int32_t *Lrow, const int32_t *Lcol, const float *ein,
                const float *e0, const float *x, const float *theta, int l, float *eout);
int node_fwd_tc(gic_handle *h, int64_t n, const int32_t *Lrowptr, const int32_t *Urowptr, const int32_t *tperm,
                const float *e, const float *x, const float *theta, int l, float *xout);

// bf16: the edge MLP's first layer on the tensor cores (BF16 inputs and W1,
// FP32 accumulation; gic_gnn_tc.cu), else FP32 on the CUDA cores; bf16_node:
// the node MLP's two layers too (inference only: the training backward of
// the node MLP is FP32)
static int gnn_forward_impl(gic_handle *h, const Pattern &p, int ngraphs, const float *theta, const float *x9,
                            const float *e0, const FwdBufs &B, double *mu, double *sig, double *parts,
                            bool bf16 = false, bool bf16_node = false)
{
    GIC_TRY(graphnorm(h, p, ngraphs, theta, x9, B.x[0], mu, sig, parts));
    const int64_t E = p.nnzL;
    for (int l = 0; l < 3; ++l) {
        if (bf16) {
            GIC_TRY(edge_fwd_tc(h, E, p.Lrow, p.Lcol, B.ein[l], e0, B.x[l], theta, l, B.eout[l]));
        } else {
            ++h->launches;
            k_edge_fwd<<<grid1(h, E), 256, 0, h->stream>>>(E, p.Lrow, p.Lcol, B.ein[l], e0, B.x[l], theta, l,
                                                           B.eout[l]);
        }
        if (l < 2) {
            if (bf16_node && !B.S[l]) {
                GIC_TRY(node_fwd_tc(h, p.n, p.Lrowptr, p.Urowptr, p.tperm, B.eout[l], B.x[l], theta, l, B.x[l + 1]));
            } else {
                ++h->launches;
                k_node_fwd<<<grid1(h, p.n), 256, 0, h->stream>>>(p.n, p.Lrowptr, p.Urowptr, p.tperm, B.eout[l],
                                                                B.x[l], theta, l, B.x[l + 1], B.S[l], B.M[l]);
            }
        }
        GIC_CUDA_TRY(cudaGetLastError());
    }
    return GIC_OK;
}

// Training workspace: every layer's inputs and the backward buffers.
struct TrainWs {
    double *mu, *sig, *parts, *sdsig;
    float *x[3], *eout[3], *S[2], *M[2];
    float *de, *dec, *dh, *dxa, *dxb, *dxd, *dS, *dM;
    double *pe, *pn; // weight-gradient partials
    size_t bytes;
};

static TrainWs carve_train(int64_t n, int64_t E, int ngraphs, int gE, int gN, void *base)
{
    TrainWs o = {};
    char *c = (char *)base;
    size_t off = 0;
    o.mu = (double *)(c + off); off += al(8 * 9 * (size_t)ngraphs);
    o.sig = (double *)(c + off); off += al(8 * 9 * (size_t)ngraphs);
    o.sdsig = (double *)(c + off); off += al(8 * 9 * (size_t)ngraphs);
    o.parts = (double *)(c + off); off += al(8 * 27 * (size_t)GX * ngraphs);
    for (int l = 0; l < 3; ++l) { o.x[l] = (float *)(c + off); off += al(4 * 9 * (size_t)n); }
    for (int l = 0; l < 3; ++l) { o.eout[l] = (float *)(c + off); off += al(4 * (size_t)E); }
    for (int l = 0; l < 2; ++l) {
        o.S[l] = (float *)(c + off); off += al(4 * (size_t)n);
        o.M[l] = (float *)(c + off); off += al(4 * (size_t)n);
    }
    o.de = (float *)(c + off); off += al(4 * (size_t)E);
    o.dec = (float *)(c + off); off += al(4 * (size_t)E);
    o.dh = (float *)(c + off); off += al(4 * 18 * (size_t)E);
    o.dxa = (float *)(c + off); off += al(4 * 9 * (size_t)n);
    o.dxb = (float *)(c + off); off += al(4 * 9 * (size_t)n);
    o.dxd = (float *)(c + off); off += al(4 * 9 * (size_t)n);
    o.dS = (float *)(c + off); off += al(4 * (size_t)n);
    o.dM = (float *)(c + off); off += al(4 * (size_t)n);
    o.pe = (double *)(c + off); off += al(8 * (size_t)gE * NP_EDGE);
    o.pn = (double *)(c + off); off += al(8 * (size_t)gN * NP_NODE);
    o.bytes = off;
    return o;
}

static void train_grids(gic_handle *h, const Pattern &p, int &gE, int &gN)
{
    gE = (int)grid1(h, p.nnzL, TB, 4);
    gN = (int)grid1(h, p.n, TB, 4);
}

}  // namespace gic

using namespace gic;

extern "C" {

int gic_gnn_param_count(void) { return NP_TOTAL; }

int gic_features(gic_handle *h, const gic_pattern *P, int ngraphs, const double *valA, float *x9, float *e0,
                 float *Ahat, double *scale_dev, double *scale_host)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!valA || !x9 || !e0 || !scale_dev) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    const int64_t ng = p.n / ngraphs;
    double *mean = (double *)h->dev_small;            // ngraphs <= 4096
    double *parts = (double *)h->dev_small + 4096;    // GX * ngraphs, checked below
    if ((size_t)(4096 + GX * ngraphs) * 8 > 60000) return GIC_ERR_UNSUPPORTED;
    // the moments: as many blocks per graph as the partials area holds, up
    // to 8 per SM in all
    const int gx = (int)std::max<int64_t>(GX, std::min<int64_t>((int64_t)h->num_sms * 8 / ngraphs,
                                                               (60000 / 8 - 4096) / ngraphs));
    dim3 gr(gx, ngraphs);
    ++h->launches;
    k_tril_moments<<<gr, RB, 0, h->stream>>>(0, ng, p.rowptr, p.Lrowptr, valA, mean, parts);
    ++h->launches;
    k_tril_finish<<<ngraphs, 32, 0, h->stream>>>(0, ng, p.Lrowptr, parts, gx, mean, scale_dev);
    ++h->launches;
    k_tril_moments<<<gr, RB, 0, h->stream>>>(1, ng, p.rowptr, p.Lrowptr, valA, mean, parts);
    ++h->launches;
    k_tril_finish<<<ngraphs, 32, 0, h->stream>>>(1, ng, p.Lrowptr, parts, gx, mean, scale_dev);
    ++h->launches;
    k_features<<<grid1(h, p.n), 256, 0, h->stream>>>(p.n, ng, p.rowptr, p.col, valA, x9);
    ++h->launches;
    k_scaled_values<<<grid1(h, p.nnzL), 256, 0, h->stream>>>(p.nnzL, p.nnzA, ng, ngraphs, p.rowptr, p.Lrowptr, p.Lrow,
                                                            valA, scale_dev, e0, Ahat);
    GIC_CUDA_TRY(cudaGetLastError());
    if (scale_host) {
        GIC_CUDA_TRY(cudaMemcpyAsync(scale_host, scale_dev, 8 * (size_t)ngraphs, cudaMemcpyDeviceToHost, h->stream));
        GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    return GIC_OK;
}

int gic_gnn_workspace_size(gic_handle *h, const gic_pattern *P, int ngraphs, int training, size_t *bytes)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!bytes) return GIC_ERR_INVALID_ARG;
    if (training) {
        int gE, gN;
        train_grids(h, P->p, gE, gN);
        *bytes = carve_train(P->p.n, P->p.nnzL, ngraphs, gE, gN, nullptr).bytes;
    } else {
        *bytes = carve_infer(P->p.n, P->p.nnzL, ngraphs, nullptr).bytes;
    }
    return GIC_OK;
}

int gic_gnn_forward(gic_handle *h, const gic_pattern *P, int ngraphs, const float *theta, const float *x9,
                    const float *e0, float *g, void *ws, size_t ws_bytes)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!theta || !x9 || !e0 || !g || !ws) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    InferWs W = carve_infer(p.n, p.nnzL, ngraphs, ws);
    if (ws_bytes < W.bytes) return GIC_ERR_WORKSPACE;
    FwdBufs B = {};
    B.x[0] = W.xa; B.x[1] = W.xb; B.x[2] = W.xa;
    B.ein[0] = const_cast<float *>(e0); B.eout[0] = W.ea;
    B.ein[1] = W.ea; B.eout[1] = W.eb;
    B.ein[2] = W.eb; B.eout[2] = g;
    return gnn_forward_impl(h, p, ngraphs, theta, x9, e0, B, W.mu, W.sig, W.parts, h->tune_gnn_bf16 != 0,
                            h->tune_gnn_bf16 != 0);
}

int gic_gnn_forward_train(gic_handle *h, const gic_pattern *P, int ngraphs, const float *theta, const float *x9,
                          const float *e0, float *g, void *ws, size_t ws_bytes)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!theta || !x9 || !e0 || !g || !ws) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    int gE, gN;
    train_grids(h, p, gE, gN);
    TrainWs W = carve_train(p.n, p.nnzL, ngraphs, gE, gN, ws);
    if (ws_bytes < W.bytes) return GIC_ERR_WORKSPACE;
    FwdBufs B = {};
    for (int l = 0; l < 3; ++l) { B.x[l] = W.x[l]; B.eout[l] = W.eout[l]; }
    B.ein[0] = const_cast<float *>(e0); B.ein[1] = W.eout[0]; B.ein[2] = W.eout[1];
    for (int l = 0; l < 2; ++l) { B.S[l] = W.S[l]; B.M[l] = W.M[l]; }
    GIC_TRY(gnn_forward_impl(h, p, ngraphs, theta, x9, e0, B, W.mu, W.sig, W.parts, h->tune_train_bf16 != 0));
    GIC_CUDA_TRY(cudaMemcpyAsync(g, W.eout[2], 4 * (size_t)p.nnzL, cudaMemcpyDeviceToDevice, h->stream));
    return GIC_OK;
}

int gic_gnn_backward(gic_handle *h, const gic_pattern *P, int ngraphs, const float *theta, const float *x9,
                     const float *e0, const float *dg, float *dtheta, void *ws, size_t ws_bytes)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!theta || !x9 || !e0 || !dg || !dtheta || !ws) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    int gE, gN;
    train_grids(h, p, gE, gN);
    TrainWs W = carve_train(p.n, p.nnzL, ngraphs, gE, gN, ws);
    if (ws_bytes < W.bytes) return GIC_ERR_WORKSPACE;
    const int64_t E = p.nnzL, n = p.n, ng = n / ngraphs;
    const float *ein[3] = {e0, W.eout[0], W.eout[1]};
    cudaStream_t s = h->stream;
    GIC_CUDA_TRY(cudaMemcpyAsync(W.de, dg, 4 * (size_t)E, cudaMemcpyDeviceToDevice, s));
    float *dx_next = W.dxa, *dx_cur = W.dxb;
    for (int l = 2; l >= 0; --l) {
        if (l < 2) {
            ++h->launches;
            k_node_bwd<<<gN, TB, 0, s>>>(n, W.x[l], W.S[l], W.M[l], theta, l, dx_next, W.dxd, W.dS, W.dM, W.pn);
            ++h->launches;
            k_reduce_partials<<<(NP_NODE + 255) / 256, 256, 0, s>>>(W.pn, gN, NP_NODE, dtheta + off_node(l));
            ++h->launches;
            k_agg_bwd<<<grid1(h, E), 256, 0, s>>>(E, p.Lrow, p.Lcol, p.Lrowptr, p.Urowptr, W.dec, W.dS, W.dM, W.de);
        }
        ++h->launches;
        k_edge_bwd<<<gE, TB, 0, s>>>(E, p.Lrow, p.Lcol, ein[l], e0, W.x[l], theta, l, W.de, W.dh, W.dec, W.pe,
                                     h->tune_train_bf16 != 0);
        ++h->launches;
        k_reduce_partials<<<(NP_EDGE + 255) / 256, 256, 0, s>>>(W.pe, gE, NP_EDGE, dtheta + off_edge(l));
        ++h->launches;
        k_dx_gather<<<grid1(h, n), 256, 0, s>>>(n, p.Lrowptr, p.Urowptr, p.tperm, W.dh, l < 2 ? W.dxd : nullptr, dx_cur);
        GIC_CUDA_TRY(cudaGetLastError());
        float *t = dx_next; dx_next = dx_cur; dx_cur = t; // dx_next now holds d x[l]
    }
    // GraphNorm backward with d x[0] in dx_next
    dim3 gr(GX, ngraphs);
    ++h->launches;
    k_gn_bwd_moments<<<gr, RB, 0, s>>>(0, ng, x9, theta, W.mu, W.sig, dx_next, W.sdsig, W.parts);
    ++h->launches;
    k_gn_bwd_finish<<<1, 32, 0, s>>>(0, ngraphs, W.parts, GX, W.mu, W.sdsig, dtheta);
    ++h->launches;
    k_gn_bwd_moments<<<gr, RB, 0, s>>>(1, ng, x9, theta, W.mu, W.sig, dx_next, W.sdsig, W.parts);
    ++h->launches;
    k_gn_bwd_finish<<<1, 32, 0, s>>>(1, ngraphs, W.parts, GX, W.mu, W.sdsig, dtheta);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_gnn_correct(gic_handle *h, const gic_pattern *P, int ngraphs, const double *LIC, const float *g,
                    const double *scale_dev, double *Lout, int *diag_ok)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!LIC || !g || !scale_dev || !Lout) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    unsigned *bad = (unsigned *)((char *)h->dev_small + 61000);
    GIC_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, h->stream));
    ++h->launches;
    k_correct<<<grid1(h, p.nnzL), 256, 0, h->stream>>>(p.nnzL, p.n / ngraphs, ngraphs, p.Lrow, p.Lcol, LIC, g,
                                                       scale_dev, Lout, bad);
    ++h->launches;
    k_correct_diag<<<grid1(h, p.n), 256, 0, h->stream>>>(p.n, p.Lrowptr, LIC, g, Lout, bad);
    GIC_CUDA_TRY(cudaGetLastError());
    if (diag_ok) {
        unsigned *hb = (unsigned *)((char *)h->host_pinned + 3000);
        GIC_CUDA_TRY(cudaMemcpyAsync(hb, bad, 4, cudaMemcpyDeviceToHost, h->stream));
        GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
        *diag_ok = (*hb == 0u);
    }
    return GIC_OK;
}

int gic_scale_factor(gic_handle *h, const gic_pattern *P, int ngraphs, const double *LIC, const double *scale_dev,
                     float *LIChat)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!LIC || !scale_dev || !LIChat) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    ++h->launches;
    k_scale_factor<<<grid1(h, p.nnzL), 256, 0, h->stream>>>(p.nnzL, p.n / ngraphs, ngraphs, p.Lrow, LIC, scale_dev,
                                                            LIChat);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_gnn_correct_scaled(gic_handle *h, const gic_pattern *P, const float *LIChat, const float *g, float *Lhat)
{
    GIC_TRY(check_batch(h, P, 1));
    if (!LIChat || !g || !Lhat) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    ++h->launches;
    k_correct_scaled<<<grid1(h, p.nnzL), 256, 0, h->stream>>>(p.nnzL, p.Lrow, p.Lcol, LIChat, g, Lhat);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_gnn_correct_backward(gic_handle *h, const gic_pattern *P, const float *Lhat, const float *dLhat, float *dg)
{
    GIC_TRY(check_batch(h, P, 1));
    if (!Lhat || !dLhat || !dg) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    ++h->launches;
    k_correct_bwd<<<grid1(h, p.nnzL), 256, 0, h->stream>>>(p.nnzL, p.Lrow, p.Lcol, Lhat, dLhat, dg);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_probe_workspace_size(gic_handle *h, const gic_pattern *P, int ngraphs, int m, size_t *bytes)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!bytes || m < 1 || m > 16) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    *bytes = al(4 * (size_t)p.nnzL) + 3 * al(4 * (size_t)m * p.n) + al(8 * (size_t)GX * ngraphs);
    return GIC_OK;
}

int gic_probe_loss(gic_handle *h, const gic_pattern *P, int ngraphs, const float *Ahat, const float *Lhat,
                   const float *Z, int m, float *loss, float *dLhat, void *ws, size_t ws_bytes)
{
    GIC_TRY(check_batch(h, P, ngraphs));
    if (!Ahat || !Lhat || !Z || !loss || !ws || m < 1 || m > 16) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    size_t need = 0;
    GIC_TRY(gic_probe_workspace_size(h, P, ngraphs, m, &need));
    if (ws_bytes < need) return GIC_ERR_WORKSPACE;
    char *c = (char *)ws;
    size_t off = 0;
    float *U = (float *)(c + off); off += al(4 * (size_t)p.nnzL);
    float *u = (float *)(c + off); off += al(4 * (size_t)m * p.n);
    float *v = (float *)(c + off); off += al(4 * (size_t)m * p.n);
    float *w = (float *)(c + off); off += al(4 * (size_t)m * p.n);
    double *parts = (double *)(c + off);
    cudaStream_t s = h->stream;
    const int64_t n = p.n, ng = n / ngraphs;
    ++h->launches;
    k_gather_f32<<<grid1(h, p.nnzL), 256, 0, s>>>(p.nnzL, p.tperm, Lhat, U);
    ++h->launches;
    k_ut_mult<<<grid1(h, n), 256, 0, s>>>(n, m, p.Urowptr, p.Ucol, U, Z, u); // Algorithm 2, first round
    dim3 gr(GX, ngraphs);
    ++h->launches;
    k_loss_v<<<gr, RB, 0, s>>>(ng, m, p.rowptr, p.col, Ahat, p.Lrowptr, p.Lcol, Lhat, Z, u, v, n, parts);
    ++h->launches;
    k_loss_finish<<<1, 32, 0, s>>>(ngraphs, m, parts, GX, loss);
    if (dLhat) {
        ++h->launches;
        k_ut_mult<<<grid1(h, n), 256, 0, s>>>(n, m, p.Urowptr, p.Ucol, U, v, w);
        ++h->launches;
        k_loss_grad<<<grid1(h, p.nnzL), 256, 0, s>>>(p.nnzL, m, n, p.Lrow, p.Lcol, u, v, Z, w,
                                                    2.0f / ((float)m * (float)ngraphs), dLhat);
    }
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int gic_adam_step(gic_handle *h, int64_t np, float *theta, const float *grad, float *m1, float *m2, int t, double lr)
{
    GIC_TRY(check_handle(h));
    if (np < 1 || !theta || !grad || !m1 || !m2 || t < 1) return GIC_ERR_INVALID_ARG;
    const double c1 = 1.0 - pow(0.9, t), c2 = 1.0 - pow(0.999, t);
    ++h->launches;
    k_adam<<<grid1(h, np), 256, 0, h->stream>>>(np, theta, grad, m1, m2, (float)lr, (float)c1, (float)c2);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

}  // extern "C"

namespace gic {

// gic_solve_host's correction: features, GNN forward, correction; keeps the
// corrected factor only if its diagonal is positive and finite.
int gnn_correct_inplace(gic_handle *h, const gic_pattern *P, const double *valA, const float *theta_host, double *L,
                        void *ws, size_t ws_bytes, int *kept)
{
    const Pattern &p = P->p;
    const int64_t n = p.n, E = p.nnzL;
    InferWs Wi = carve_infer(n, E, 1, ws);
    char *c = (char *)ws + Wi.bytes;
    size_t off = 0;
    float *theta = (float *)(c + off); off += al(4 * NP_TOTAL);
    float *x9 = (float *)(c + off); off += al(4 * 9 * (size_t)n);
    float *e0 = (float *)(c + off); off += al(4 * (size_t)E);
    float *g = (float *)(c + off); off += al(4 * (size_t)E);
    off += al(4 * (size_t)E);
    double *scale = (double *)(c + off); off += al(8 * 16);
    off += al(8 * 16);
    double *Lout = (double *)(c + off); off += al(8 * (size_t)E);
    if (Wi.bytes + off > ws_bytes) return GIC_ERR_WORKSPACE;
    GIC_CUDA_TRY(cudaMemcpyAsync(theta, theta_host, 4 * NP_TOTAL, cudaMemcpyHostToDevice, h->stream));
    GIC_TRY(gic_features(h, P, 1, valA, x9, e0, nullptr, scale, nullptr));
    GIC_TRY(gic_gnn_forward(h, P, 1, theta, x9, e0, g, ws, Wi.bytes));
    int ok = 0;
    GIC_TRY(gic_gnn_correct(h, P, 1, L, g, scale, Lout, &ok));
    if (ok) GIC_CUDA_TRY(cudaMemcpyAsync(L, Lout, 8 * (size_t)E, cudaMemcpyDeviceToDevice, h->stream));
    *kept = ok;
    return GIC_OK;
}

}  // namespace gic
