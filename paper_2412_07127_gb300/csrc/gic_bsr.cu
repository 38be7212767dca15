// gic_bsr.cu -- A7a: SpMV of the PCG on 3x3 node blocks (BSR in SELL-32
// order) for patterns made of them: every run of 3 rows starting at a
// multiple of 3 (a node's dofs) has identical columns, and those come in
// aligned triples (the dofs of a neighbour node). Hex elasticity has this
// shape; other patterns keep the SELL-32 CSR kernel.
//
// Why: on this GPU one FP64 warp instruction holds the SM's FP64 pipe for
// ~17-20 cycles, so an FP64 SpMV is bound by its FMAs as much as by its
// bytes (at 148^3: 788M FMAs need 1.56 ms at the measured FP64 rate, the
// CSR's 9.5 GB 1.39 ms at the measured copy bandwidth). A block costs one
// int32 column for 9 values instead of 9, so the bytes fall to ~8.4 per
// nonzero and the FMAs alone set the pace; every FMA is a full-warp
// instruction (one node row per lane, three row accumulators, no cross-lane
// reduction).
//
// Layout: slices of 32 consecutive nodes (one per lane); inside a slice
// block step k of lane l holds its 9 values at bval[((bptr + k) * 9 + e) * 32
// + l] (e = 3r + c, row-major) and its node column at bcol[(bptr + k) * 32 +
// l], so each load instruction reads 32 consecutive words; a slice is padded
// to its widest node with zero blocks on the node itself.
#include <vector>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int BSR_BLOCK = 256;

// bad |= 1 where node-row block b (rows 3b..3b+2) is not a run of three
// identical rows whose columns come in aligned triples; nb[b] = its blocks
__global__ void k_bsr_check(int64_t nodes, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                            int32_t *nb, unsigned *bad)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nodes; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a0 = rowptr[3 * b], len = rowptr[3 * b + 1] - a0;
        bool ok = (len % 3 == 0);
        for (int r = 1; r < 3 && ok; ++r) {
            const int32_t ar = rowptr[3 * b + r];
            if (rowptr[3 * b + r + 1] - ar != len) { ok = false; break; }
            for (int32_t j = 0; j < len; ++j)
                if (col[ar + j] != col[a0 + j]) { ok = false; break; }
        }
        for (int32_t j = 0; j < len && ok; j += 3) {
            const int32_t c = col[a0 + j];
            if (c % 3 != 0 || col[a0 + j + 1] != c + 1 || col[a0 + j + 2] != c + 2) ok = false;
        }
        nb[b] = len / 3;
        if (!ok) atomicOr(bad, 1u);
    }
}

// node columns of the slices (padding: the node itself, with zero values)
__global__ void k_bsr_cols(int64_t nodes, int64_t nsl, const int32_t *__restrict__ rowptr,
                           const int32_t *__restrict__ col, const int64_t *__restrict__ bptr,
                           const int32_t *__restrict__ bw, int32_t *bcol)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsl * 32; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i >> 5, b = i;
        const int l = (int)(i & 31);
        const int32_t a0 = (b < nodes) ? rowptr[3 * b] : 0;
        const int32_t nbk = (b < nodes) ? (rowptr[3 * b + 1] - a0) / 3 : 0;
        const int32_t self = (b < nodes) ? (int32_t)b : 0;
        for (int32_t k = 0; k < bw[sl]; ++k)
            bcol[(bptr[sl] + k) * 32 + l] = (k < nbk) ? col[a0 + 3 * k] / 3 : self;
    }
}

// values of A in the slice layout
__global__ void k_bsr_vals(int64_t nodes, int64_t nsl, const int32_t *__restrict__ rowptr,
                           const double *__restrict__ val, const int64_t *__restrict__ bptr,
                           const int32_t *__restrict__ bw, double *bval)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsl * 32; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i >> 5, b = i;
        const int l = (int)(i & 31);
        const int32_t nbk = (b < nodes) ? (rowptr[3 * b + 1] - rowptr[3 * b]) / 3 : 0;
        for (int32_t k = 0; k < bw[sl]; ++k) {
            double *o = bval + (bptr[sl] + k) * 288 + l;
            for (int r = 0; r < 3; ++r) {
                const int32_t ar = (b < nodes) ? rowptr[3 * b + r] : 0;
                for (int c = 0; c < 3; ++c) o[(3 * r + c) * 32] = (k < nbk) ? val[ar + 3 * k + c] : 0.0;
            }
        }
    }
}

// MODE 1: w = A p, p^T w, alpha = r^T z / p^T w (Algorithm 1);
// MODE 2: r = b - A x, ||r||^2, ||b||^2 and the stop test (its first line).
// LPN lanes per node: 1 = a warp per slice of 32 nodes; 2 or 4 = a warp per
// half or quarter slice, the LPN lanes of a node taking every LPN-th block
// step (LPN times the warps and 1/LPN of the chain per lane, for systems whose
// slices are too few to fill the SMs), their sums added by shuffles.
template <int MODE, int LPN>
__global__ void __launch_bounds__(BSR_BLOCK) k_spmv_bsr(int64_t n, int64_t nsl, const int64_t *__restrict__ bptr,
                                                        const int32_t *__restrict__ bw,
                                                        const int32_t *__restrict__ bcol,
                                                        const double *__restrict__ bval,
                                                        const double *__restrict__ x, double *__restrict__ y,
                                                        const double *__restrict__ b, double *partials,
                                                        Scalars *sc)
{
    if (sc->done) return;
    __shared__ double sh[BSR_BLOCK / 32];
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nodes = n / 3;
    const int col_lane = lane / LPN;  // the node's column in its part of the slice
    const int kpar = lane % LPN;      // this lane's block steps: kpar, kpar + LPN, ...
    double d1 = 0.0, d2 = 0.0;
    for (int64_t item = w; item < nsl * LPN; item += nw) {
        const int64_t sl = item / LPN;
        const int sub = (int)(item % LPN) * (32 / LPN) + col_lane; // the node's column in the slice
        const int64_t node = sl * 32 + sub;
        const int32_t width = (node < nodes) ? bw[sl] : 0; // lanes past the last node load nothing
        const int64_t o = bptr[sl];
        // two accumulators per row (alternate block steps of this lane); U
        // block steps per iteration, their loads in flight together (more for
        // the half-slice variant, whose warps are few per SM)
        constexpr int U = (LPN == 1) ? 2 : 4;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, c0 = 0.0, c1 = 0.0, c2 = 0.0;
        int32_t k = kpar;
        for (; k + (U - 1) * LPN < width; k += U * LPN) {
            int32_t j[U];
            double v[U][9], xv[U][3];
#pragma unroll
            for (int u = 0; u < U; ++u) j[u] = __ldg(bcol + (o + k + u * LPN) * 32 + sub);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < 9; ++e) v[u][e] = __ldg(bval + ((o + k + u * LPN) * 9 + e) * 32 + sub);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < 3; ++c) xv[u][c] = __ldg(x + 3 * (int64_t)j[u] + c);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (u & 1) {
                        c0 = fma(v[u][c], xv[u][c], c0);
                        c1 = fma(v[u][3 + c], xv[u][c], c1);
                        c2 = fma(v[u][6 + c], xv[u][c], c2);
                    } else {
                        a0 = fma(v[u][c], xv[u][c], a0);
                        a1 = fma(v[u][3 + c], xv[u][c], a1);
                        a2 = fma(v[u][6 + c], xv[u][c], a2);
                    }
                }
        }
        for (; k < width; k += LPN) {
            const int32_t j0 = __ldg(bcol + (o + k) * 32 + sub);
            double v0[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) v0[e] = __ldg(bval + ((o + k) * 9 + e) * 32 + sub);
            const double x00 = __ldg(x + 3 * (int64_t)j0), x01 = __ldg(x + 3 * (int64_t)j0 + 1),
                         x02 = __ldg(x + 3 * (int64_t)j0 + 2);
            a0 = fma(v0[0], x00, a0); a1 = fma(v0[3], x00, a1); a2 = fma(v0[6], x00, a2);
            a0 = fma(v0[1], x01, a0); a1 = fma(v0[4], x01, a1); a2 = fma(v0[7], x01, a2);
            a0 = fma(v0[2], x02, a0); a1 = fma(v0[5], x02, a1); a2 = fma(v0[8], x02, a2);
        }
        double s[3] = {a0 + c0, a1 + c1, a2 + c2};
#pragma unroll
        for (int o = 1; o < LPN; o <<= 1)
#pragma unroll
            for (int r = 0; r < 3; ++r) s[r] += __shfl_xor_sync(0xffffffffu, s[r], o);
        if (node < nodes && kpar == 0) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int64_t i = 3 * node + r;
                if (MODE == 2) {
                    const double bi = b[i];
                    const double ri = bi - s[r];
                    y[i] = ri;
                    d1 = fma(ri, ri, d1);
                    d2 = fma(bi, bi, d2);
                } else {
                    y[i] = s[r];
                    d1 = fma(x[i], s[r], d1);
                }
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

static unsigned bgrid(gic_handle *h, int64_t items, int per_sm)
{
    int64_t b = (items + 255) / 256, cap = (int64_t)h->num_sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

void free_bsr(Pattern &P)
{
    cudaFree(P.bsr_ptr);
    cudaFree(P.bsr_w);
    cudaFree(P.bsr_col);
    P.bsr_ptr = nullptr;
    P.bsr_w = nullptr;
    P.bsr_col = nullptr;
    P.bsr_ready = 0;
    P.bsr_nsl = P.bsr_steps = 0;
}

int build_bsr(gic_handle *h, Pattern &P)
{
    P.bsr_ready = 0;
    if (P.n % 3 != 0 || P.n < 3) return GIC_OK;
    const int64_t nodes = P.n / 3, nsl = (nodes + 31) / 32;
    int32_t *nb = nullptr;
    unsigned *bad = (unsigned *)((char *)h->dev_small + 61000);
    GIC_CUDA_TRY(cudaMalloc(&nb, 4 * (size_t)nodes));
    unsigned hb = 1;
    std::vector<int32_t> hnb(nodes);
    cudaError_t e = cudaMemsetAsync(bad, 0, 4, h->stream);
    if (e == cudaSuccess) {
        ++h->launches;
        k_bsr_check<<<bgrid(h, nodes, 16), 256, 0, h->stream>>>(nodes, P.rowptr, P.col, nb, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hnb.data(), nb, 4 * (size_t)nodes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(nb);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "build_bsr", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    if (hb != 0) return GIC_OK; // not made of 3x3 node blocks
    std::vector<int32_t> w(nsl);
    std::vector<int64_t> ptr(nsl + 1);
    ptr[0] = 0;
    for (int64_t s = 0; s < nsl; ++s) {
        int32_t m = 0;
        for (int64_t b = s * 32; b < std::min(nodes, s * 32 + 32); ++b) m = std::max(m, hnb[b]);
        w[s] = m;
        ptr[s + 1] = ptr[s] + m;
    }
    GIC_CUDA_TRY(cudaMalloc(&P.bsr_ptr, 8 * (size_t)(nsl + 1)));
    GIC_CUDA_TRY(cudaMalloc(&P.bsr_w, 4 * (size_t)nsl));
    GIC_CUDA_TRY(cudaMalloc(&P.bsr_col, 4 * 32 * (size_t)(ptr[nsl] > 0 ? ptr[nsl] : 1)));
    GIC_CUDA_TRY(cudaMemcpyAsync(P.bsr_ptr, ptr.data(), 8 * (size_t)(nsl + 1), cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(P.bsr_w, w.data(), 4 * (size_t)nsl, cudaMemcpyHostToDevice, h->stream));
    ++h->launches;
    k_bsr_cols<<<bgrid(h, nsl * 32, 16), 256, 0, h->stream>>>(nodes, nsl, P.rowptr, P.col, P.bsr_ptr, P.bsr_w,
                                                              P.bsr_col);
    GIC_CUDA_TRY(cudaGetLastError());
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    P.bsr_nsl = nsl;
    P.bsr_steps = ptr[nsl];
    P.bsr_ready = 1;
    return GIC_OK;
}

int bsr_values(gic_handle *h, const Pattern &P, const double *valA, double *bval)
{
    ++h->launches;
    k_bsr_vals<<<bgrid(h, P.bsr_nsl * 32, 16), 256, 0, h->stream>>>(P.n / 3, P.bsr_nsl, P.rowptr, valA, P.bsr_ptr,
                                                                    P.bsr_w, bval);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

int bsr_spmv(gic_handle *h, const Pattern &P, int mode, const double *bval, const double *x, double *y,
             const double *b, double *partials, Scalars *sc)
{
    ++h->launches;
    // a warp per slice of 32 nodes, the grid striding over the slices; with
    // fewer slices than 24 warps per SM, a warp per half slice (measured at
    // 40^3: 55.5 us with whole slices, 50.0 us with halves, 53.0 us with
    // quarters)
    const int lpn = (P.bsr_nsl < 24 * (int64_t)h->num_sms) ? 2 : 1;
    const unsigned grid = bgrid(h, P.bsr_nsl * 32 * lpn, 8);
    const int64_t n = P.n, ns = P.bsr_nsl;
    if (mode == 1) {
        if (lpn == 2)
            k_spmv_bsr<1, 2><<<grid, BSR_BLOCK, 0, h->stream>>>(n, ns, P.bsr_ptr, P.bsr_w, P.bsr_col, bval, x, y,
                                                                 nullptr, partials, sc);
        else
            k_spmv_bsr<1, 1><<<grid, BSR_BLOCK, 0, h->stream>>>(n, ns, P.bsr_ptr, P.bsr_w, P.bsr_col, bval, x, y,
                                                                 nullptr, partials, sc);
    } else {
        if (lpn == 2)
            k_spmv_bsr<2, 2><<<grid, BSR_BLOCK, 0, h->stream>>>(n, ns, P.bsr_ptr, P.bsr_w, P.bsr_col, bval, x, y, b,
                                                                 partials, sc);
        else
            k_spmv_bsr<2, 1><<<grid, BSR_BLOCK, 0, h->stream>>>(n, ns, P.bsr_ptr, P.bsr_w, P.bsr_col, bval, x, y, b,
                                                                 partials, sc);
    }
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

}  // namespace gic
