// gic_analyze.cu -- A2: device-side analysis of a symmetric CSR pattern.
//
// From A's CSR (sorted columns, stored diagonal, symmetric pattern) build:
//   * L = tril(A): a prefix of every row of A, so L entry p of row i is A
//     entry rowptr[i] + (p - Lrowptr[i]);
//   * U = L^T: by symmetry row j of U is the suffix of A's row j that starts
//     at the diagonal; tperm maps every U entry (j,i) to L entry (i,j);
//   * groups: maximal runs (cut every GMAX rows) of consecutive rows with
//     identical column sets. Inside a group the diagonal block is dense and
//     all rows share their columns outside it, so one warp solves a whole
//     group (for hex elasticity a group is the 3 dofs of a node);
//   * row levels of the lower-triangular dependency DAG.
// Everything runs on the device; no host pass over the rows.
#include <limits.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "gic_internal.cuh"

namespace gic {

// ---------------------------------------------------------------- scans
// Exclusive prefix scan of int64 values (op = sum or max) in three passes.
constexpr int SCAN_BLOCK = 1024;

template <bool MAX>
__device__ __forceinline__ long long scan_op(long long a, long long b) { return MAX ? (a > b ? a : b) : a + b; }

template <bool MAX>
__device__ long long block_inclusive_scan(long long v, long long *sh)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = scan_op<MAX>(v, t);
    }
    if (lane == 31) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : (MAX ? LLONG_MIN : 0);
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = scan_op<MAX>(w, t);
        }
        sh[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v = scan_op<MAX>(v, sh[wid - 1]);
    __syncthreads();
    return v;
}

// in: int32 values; inclusive scan written to out64; block totals to bsum.
template <bool MAX>
__global__ void k_scan_blocks(const int32_t *in, int64_t n, long long *out64, long long *bsum)
{
    __shared__ long long sh[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    long long v = (i < n) ? (long long)in[i] : (MAX ? LLONG_MIN : 0);
    long long s = block_inclusive_scan<MAX>(v, sh);
    if (i < n) out64[i] = s;
    if (threadIdx.x == SCAN_BLOCK - 1) bsum[blockIdx.x] = s;
}

// exclusive scan of the block totals in place (single block, any count)
template <bool MAX>
__global__ void k_scan_totals(long long *bsum, int64_t nb, long long *total)
{
    __shared__ long long sh[32];
    long long carry = MAX ? LLONG_MIN : 0;
    for (int64_t base = 0; base < nb; base += SCAN_BLOCK) {
        int64_t i = base + threadIdx.x;
        long long v = (i < nb) ? bsum[i] : (MAX ? LLONG_MIN : 0);
        long long s = block_inclusive_scan<MAX>(v, sh);
        long long excl = __shfl_up_sync(0xffffffffu, s, 1);
        // exclusive value of element i within this chunk
        __shared__ long long last;
        if (threadIdx.x == SCAN_BLOCK - 1) last = s;
        long long prev_lane = excl;
        if ((threadIdx.x & 31) == 0) prev_lane = (threadIdx.x == 0) ? (MAX ? LLONG_MIN : 0) : sh[(threadIdx.x >> 5) - 1];
        __syncthreads();
        if (i < nb) bsum[i] = scan_op<MAX>(carry, prev_lane);
        carry = scan_op<MAX>(carry, last);
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// out[i] = exclusive value at i (out has n+1 entries for sum scans)
template <bool MAX>
__global__ void k_scan_finish(const int32_t *in, int64_t n, const long long *incl, const long long *bsum,
                              int32_t *out, int with_total, const long long *total)
{
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) {
        long long v = scan_op<MAX>(bsum[blockIdx.x], incl[i]);
        if (MAX) {
            out[i] = (int32_t)v; // inclusive max
        } else {
            out[i] = (int32_t)(v - in[i]); // exclusive sum
        }
    }
    if (with_total && i == 0) out[n] = (int32_t)*total;
}

// Host wrapper. MAX = false: out[0..n] exclusive sums, *total (host) = sum.
// MAX = true: out[0..n) inclusive running maxima.
template <bool MAX>
static int scan_i32(gic_handle *h, const int32_t *in, int64_t n, int32_t *out, long long *total_host)
{
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb == 0) nb = 1;
    long long *tmp = nullptr;
    GIC_CUDA_TRY(cudaMalloc(&tmp, sizeof(long long) * (size_t)(n + nb + 1)));
    long long *incl = tmp, *bsum = tmp + n, *total = tmp + n + nb;
    ++h->launches;
    k_scan_blocks<MAX><<<(unsigned)nb, SCAN_BLOCK, 0, h->stream>>>(in, n, incl, bsum);
    ++h->launches;
    k_scan_totals<MAX><<<1, SCAN_BLOCK, 0, h->stream>>>(bsum, nb, total);
    ++h->launches;
    k_scan_finish<MAX><<<(unsigned)nb, SCAN_BLOCK, 0, h->stream>>>(in, n, incl, bsum, out, MAX ? 0 : 1, total);
    cudaError_t e = cudaGetLastError();
    long long t = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&t, total, sizeof t, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "scan", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    if (total_host) *total_host = t;
    return GIC_OK;
}

int scan_excl_i32(gic_handle *h, const int32_t *in, int64_t n, int32_t *out, long long *total)
{
    return scan_i32<false>(h, in, n, out, total);
}

// ---------------------------------------------------------------- checks
// Per row: bounds, strictly increasing columns, stored diagonal; Lcnt[i] =
// number of entries with column <= i; same[i] = row i has the same columns
// as row i-1.
__global__ void k_validate(int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, int32_t *Lcnt,
                           int32_t *same, unsigned *err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = rowptr[i], b = rowptr[i + 1];
        if (i == 0 && a != 0) atomicOr(err, 4u);
        if (i == n - 1 && (int64_t)b != nnz) atomicOr(err, 4u);
        if (b < a || a < 0 || (int64_t)b > nnz) {
            atomicOr(err, 4u);
            Lcnt[i] = 0;
            same[i] = 0;
            continue;
        }
        int cnt = 0, diag = 0, prev = -1;
        for (int32_t p = a; p < b; ++p) {
            int32_t c = col[p];
            if (c <= prev || c < 0 || c >= n) atomicOr(err, 8u);
            if (c <= i) cnt++;
            if (c == i) diag = 1;
            prev = c;
        }
        if (!diag) atomicOr(err, 16u);
        Lcnt[i] = cnt;
        int sm = 0;
        if (i > 0) {
            int32_t a0 = rowptr[i - 1], b0 = rowptr[i];
            if (a0 >= 0 && b0 >= a0 && b0 - a0 == b - a) {
                sm = 1;
                for (int32_t k = 0; k < b - a; ++k)
                    if (col[a0 + k] != col[a + k]) { sm = 0; break; }
            }
        }
        same[i] = sm;
    }
}

__device__ __forceinline__ int32_t find_col(const int32_t *col, int32_t lo, int32_t hi, int32_t key)
{
    // first position in [lo,hi) with col >= key
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Symmetry: every (i,j) has a stored (j,i).
__global__ void k_symcheck(int64_t n, const int32_t *rowptr, const int32_t *col, unsigned *err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j < 0 || j >= n) continue;
            int32_t q = find_col(col, rowptr[j], rowptr[j + 1], (int32_t)i);
            if (q >= rowptr[j + 1] || col[q] != i) { atomicOr(err, 32u); return; }
        }
    }
}

__global__ void k_fill_L(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *Lrowptr, int32_t *Lcol,
                         int32_t *Ucnt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = rowptr[i], lb = Lrowptr[i], lc = Lrowptr[i + 1] - lb;
        for (int32_t k = 0; k < lc; ++k) Lcol[lb + k] = col[a + k];
        Ucnt[i] = rowptr[i + 1] - a - lc + 1;
    }
}

__global__ void k_fill_Lrow(int64_t n, const int32_t *Lrowptr, int32_t *Lrow)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) Lrow[p] = (int32_t)i;
}

__global__ void k_fill_U(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *Lrowptr,
                         const int32_t *Urowptr, int32_t *Ucol, int32_t *tperm)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t ub = Urowptr[j], uc = Urowptr[j + 1] - ub;
        int32_t d = rowptr[j] + (Lrowptr[j + 1] - Lrowptr[j]) - 1; // diagonal of row j in A
        for (int32_t k = 0; k < uc; ++k) {
            int32_t i = col[d + k]; // U entry (j, i), i >= j  <=>  L entry (i, j)
            Ucol[ub + k] = i;
            int32_t q = find_col(col, rowptr[i], rowptr[i + 1], (int32_t)j);
            tperm[ub + k] = Lrowptr[i] + (q - rowptr[i]);
        }
    }
}

// key[i] = i where a new run of identical rows begins, else -1
__global__ void k_run_keys(int64_t n, const int32_t *same, int32_t *key)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = same[i] ? -1 : (int32_t)i;
}

// Greatest common divisor of the run lengths (a run ends where the next row
// differs): the pattern's natural block size, e.g. 3 for a hex node's dofs.
__device__ __forceinline__ int32_t gcd_i32(int32_t a, int32_t b)
{
    while (b) {
        const int32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

__global__ void k_run_gcd(int64_t n, const int32_t *same, const int32_t *runstart, int32_t *out)
{
    int32_t g = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (i == n - 1 || !same[i + 1]) g = gcd_i32(g, (int32_t)(i + 1 - runstart[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g = gcd_i32(g, __shfl_xor_sync(0xffffffffu, g, o));
    if ((threadIdx.x & 31) == 0 && g > 0) {
        int32_t old = *((volatile int32_t *)out);
        for (;;) {
            const int32_t nv = gcd_i32(old, g);
            if (nv == old) break;
            const int32_t prev = atomicCAS(out, old, nv);
            if (prev == old) break;
            old = prev;
        }
    }
}

// group starts: run start, or every gcut rows inside a run, gcut being the
// natural block size when it is 2 .. GMAX, else GMAX. Cutting runs at the
// block size keeps one group per block where blocks of a thinned pattern
// happen to have identical rows.
__global__ void k_group_flags(int64_t n, const int32_t *runstart, int32_t gcut, int32_t *gflag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gflag[i] = ((i - runstart[i]) % gcut) == 0;
}

__global__ void k_group_starts(int64_t n, const int32_t *gflag, const int32_t *gid, int32_t *grp, int32_t ngroups)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (gflag[i]) grp[gid[i]] = (int32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) grp[ngroups] = (int32_t)n;
}

// Per-group maxima: external lower / upper counts and group size.
// first row of every row's group
__global__ void k_row_group(int32_t ngroups, const int32_t *grp, int32_t *rowgrp)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
        for (int32_t i = grp[g]; i < grp[g + 1]; ++i) rowgrp[i] = grp[g];
}

__global__ void k_group_stats(int32_t ngroups, const int32_t *grp, const int32_t *Lrowptr, const int32_t *Urowptr,
                              int32_t *stats)
{
    int mL = 0, mU = 0, mG = 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = grp[g], e = grp[g + 1] - 1;
        int eL = Lrowptr[s + 1] - Lrowptr[s] - 1;
        int eU = Urowptr[e + 1] - Urowptr[e] - 1;
        mL = max(mL, eL);
        mU = max(mU, eU);
        mG = max(mG, e - s + 1);
    }
    atomicMax(&stats[0], mL);
    atomicMax(&stats[1], mU);
    atomicMax(&stats[2], mG);
}

// Chains for k_levels: group g continues the chain of group g-1 when its
// first row reads a row of group g-1 (the last external lower column of that
// row is at or after group g-1's first row; columns are sorted ascending).
__global__ void k_chain_flags(int32_t ngroups, const int32_t *grp, const int32_t *Lrowptr, const int32_t *Lcol,
                              int32_t *cflag)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = grp[g];
        const int32_t m = Lrowptr[s + 1] - Lrowptr[s] - 1; // external lower columns of the first row
        cflag[g] = (g == 0) || m == 0 || Lcol[Lrowptr[s + 1] - 2] < grp[g - 1];
    }
}

// Row levels, sync-free: level[] starts at -1 and every row's level is written
// once. A warp takes one chain (a maximal run of consecutive groups each of
// which reads the one before it) and does its groups in order, waiting
// (bounded) for the levels of each group's external lower columns; chains
// are taken in round-robin order by a co-resident grid, so the first
// unfinished chain always progresses (its inputs lie in earlier chains or
// earlier in itself). Chains rather than single groups: taking groups one by
// one in index order keeps at most one grid's worth of consecutive groups in
// flight, and on a structured mesh that window is a fraction of a plane of
// nodes whose dependency chains then serialise plane after plane. A chain is
// itself sequential (each group's level exceeds its predecessor's), so
// walking it in one warp replaces a cross-warp hand-off per group by a step
// within the warp; on a lexicographic mesh the chains are the rows of nodes
// along x.
// With rowstep = 0 the same walk gives group levels: every row of a group
// gets 1 + the largest level among the group's external lower columns.
__global__ void k_levels(int32_t nchains, const int32_t *chain, const int32_t *grp, const int32_t *Lrowptr,
                         const int32_t *Lcol, int rowstep, int32_t *level, int32_t *maxlev, unsigned *err)
{
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int mx_all = 0;
    for (int64_t c = w; c < nchains; c += nw) {
        const int32_t g1 = chain[c + 1];
        for (int32_t g = chain[c]; g < g1; ++g) {
            int32_t s = grp[g], e = grp[g + 1] - 1;
            int32_t b0 = Lrowptr[s];
            int32_t m = Lrowptr[s + 1] - b0 - 1;
            int mx = -1;
            for (int32_t k = lane; k < m; k += 64) {
                // two columns per lane in flight at once
                bool two = k + 32 < m;
                int32_t j0 = Lcol[b0 + k], j1 = two ? Lcol[b0 + k + 32] : j0;
                int v0 = ld_acquire_i32(level + j0), v1 = ld_acquire_i32(level + j1);
                long long it = 0;
                while ((v0 < 0 || v1 < 0) && it < SPIN_LIMIT) {
                    if (it > 32) __nanosleep(64);
                    if (v0 < 0) v0 = ld_acquire_i32(level + j0);
                    if (v1 < 0) v1 = ld_acquire_i32(level + j1);
                    ++it;
                    if ((it & 1023) == 0 && *((volatile unsigned *)err) != 0u) break;
                }
                if (v0 < 0 || v1 < 0) { atomicOr(err, ERR_TIMEOUT); v0 = max(v0, 0); v1 = max(v1, 0); }
                mx = max(mx, max(v0, v1));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane <= e - s) st_release_i32(level + s + lane, mx + 1 + rowstep * lane);
            mx_all = max(mx_all, mx + 1 + rowstep * (e - s));
            __syncwarp(); // this group's levels are visible to the warp's next group
        }
    }
    if (lane == 0) atomicMax(maxlev, mx_all);
}

// ------------------------------------------------------------ schedule
__global__ void k_chunk_flags(int32_t ngroups, const int32_t *grp, const int32_t *level, int32_t *cflag)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
        cflag[g] = (g == 0) || (level[grp[g]] <= level[grp[g] - 1]);
}

__global__ void k_chunk_starts(int32_t ngroups, const int32_t *cflag, const int32_t *cid, int32_t *chunk_grp,
                               int32_t nchunks)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
        if (cflag[g]) chunk_grp[cid[g]] = (int32_t)g;
    if (blockIdx.x == 0 && threadIdx.x == 0) chunk_grp[nchunks] = ngroups;
}

// start and end level of every chunk
__global__ void k_chunk_levels(int32_t nchunks, const int32_t *chunk_grp, const int32_t *grp, const int32_t *level,
                               int32_t *lv_s, int32_t *lv_e)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += (int64_t)gridDim.x * blockDim.x) {
        lv_s[c] = level[grp[chunk_grp[c]]];
        lv_e[c] = level[grp[chunk_grp[c + 1]] - 1];
    }
}

__global__ void k_inverse_perm(int32_t cnt, const int32_t *ord, int32_t *pos)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x)
        pos[ord[k]] = (int32_t)k;
}

// row -> chunk position maps, then: every external dependency of a group
// must sit in a chunk that comes earlier in the sweep's order
__global__ void k_row_chunk(int32_t nchunks, const int32_t *chunk_grp, const int32_t *grp, int32_t *rowchunk)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += (int64_t)gridDim.x * blockDim.x)
        for (int32_t i = grp[chunk_grp[c]]; i < grp[chunk_grp[c + 1]]; ++i) rowchunk[i] = (int32_t)c;
}

// Topological sweep keys of the chunks, used when ordering the chunks by
// their first (forward) or last (backward) row level would put a chunk before
// one it reads, which thinning a factor can do. Forward:
// key[c] = max(lv_s[c], key[c'] + 1 over every other chunk c' that chunk c's
// groups read); backward: key[c] = max(maxlev - lv_e[c], key[c'] + 1 over the
// chunks that read chunk c). A sweep that takes the chunks in ascending key
// order then finds every input finished, and where the level order was
// already valid the keys mostly repeat it. One warp per chunk, sync-free as
// k_levels: key[] starts at -1, the inputs of a chunk have lower (forward) or
// higher (backward) chunk indices, and chunks are taken round-robin in that
// order by a co-resident grid, so the first unfinished chunk always
// progresses; every wait is bounded.
template <bool BACKWARD>
__global__ void k_chunk_keys(int32_t nchunks, const int32_t *chunk_grp, const int32_t *grp, const int32_t *Xrowptr,
                             const int32_t *Xcol, const int32_t *rowchunk, const int32_t *lv, int32_t maxlev,
                             int32_t *key, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = w; t < nchunks; t += nw) {
        const int32_t c = BACKWARD ? (int32_t)(nchunks - 1 - t) : (int32_t)t;
        int mx = (BACKWARD ? maxlev - lv[c] : lv[c]) - 1;
        for (int32_t g = chunk_grp[c]; g < chunk_grp[c + 1]; ++g) {
            // forward: the first row's lower columns other than the diagonal;
            // backward: the last row's upper columns other than the diagonal
            const int32_t r = BACKWARD ? grp[g + 1] - 1 : grp[g];
            const int32_t b0 = Xrowptr[r] + (BACKWARD ? 1 : 0), m = Xrowptr[r + 1] - Xrowptr[r] - 1;
            for (int32_t k = lane; k < m; k += 32) {
                const int32_t cj = rowchunk[Xcol[b0 + k]];
                if (cj == c) continue;
                int v = ld_acquire_i32(key + cj);
                long long it = 0;
                while (v < 0 && it < SPIN_LIMIT) {
                    if (it > 32) __nanosleep(64);
                    v = ld_acquire_i32(key + cj);
                    ++it;
                    if ((it & 1023) == 0 && *((volatile unsigned *)err) != 0u) break;
                }
                if (v < 0) { atomicOr(err, ERR_TIMEOUT); v = 0; }
                mx = max(mx, v);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) st_release_i32(key + c, mx + 1);
    }
}

__global__ void k_check_order(int32_t ngroups, const int32_t *grp, const int32_t *Lrowptr, const int32_t *Lcol,
                              const int32_t *Urowptr, const int32_t *Ucol, const int32_t *rowchunk,
                              const int32_t *pos_f, const int32_t *pos_b, unsigned *bad)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = grp[g], e = grp[g + 1] - 1;
        const int32_t c = rowchunk[s];
        for (int32_t p = Lrowptr[s]; p < Lrowptr[s + 1] - 1; ++p) {
            const int32_t cj = rowchunk[Lcol[p]];
            if (cj != c && pos_f[cj] >= pos_f[c]) atomicOr(bad, 1u);
        }
        for (int32_t q = Urowptr[e] + 1; q < Urowptr[e + 1]; ++q) {
            const int32_t cj = rowchunk[Ucol[q]];
            if (cj != c && pos_b[cj] >= pos_b[c]) atomicOr(bad, 2u);
        }
    }
}

// ------------------------------------------------------------ SELL-32
__global__ void k_sell_widths(int64_t n, int64_t nslices, const int32_t *rowptr, int32_t *w)
{
    for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = 0;
        for (int64_t i = sl * 32; i < min(n, sl * 32 + 32); ++i) m = max(m, rowptr[i + 1] - rowptr[i]);
        w[sl] = m;
    }
}

// every lane of every slice is written: padding of a real row points at the
// row itself, lanes past the last row (partial last slice) at column 0
__global__ void k_sell_cols(int64_t n, int64_t nslices, const int32_t *rowptr, const int32_t *col,
                            const int64_t *sptr, const int32_t *w, int32_t *scol)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslices * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i >> 5;
        const int t = (int)(i & 31);
        const int32_t a = (i < n) ? rowptr[i] : 0, len = (i < n) ? rowptr[i + 1] - a : 0;
        const int32_t pad = (i < n) ? (int32_t)i : 0;
        for (int32_t k = 0; k < w[sl]; ++k) scol[sptr[sl] + (int64_t)k * 32 + t] = (k < len) ? col[a + k] : pad;
    }
}

// ------------------------------------------------------------ warp-specialised solve schedule
__global__ void k_group_chunk(int32_t nchunks, const int32_t *chunk_grp, int32_t *gchunk)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += (int64_t)gridDim.x * blockDim.x)
        for (int32_t g = chunk_grp[c]; g < chunk_grp[c + 1]; ++g) gchunk[g] = (int32_t)c;
}

// Classify and order the m external columns (cols[0..m)) of one group.
// prev: rows [prev_lo, prev_hi); late: key[j] within the window (forward:
// level >= lev - delta; backward: level <= lev + delta). At most QLATE late
// columns are kept, those closest in level; the order written is early
// (original order), late (farthest level first, i.e. expected arrival
// order), prev (original order).
__device__ void q_classify(int m, const int32_t *cols, const int32_t *level, int32_t lev, int delta, bool forward,
                           int32_t prev_lo, int32_t prev_hi, int32_t *qcol, uint8_t *qpos, int32_t *counts)
{
    unsigned long long late = 0, prev = 0;
    int nl = 0, np = 0;
    for (int j = 0; j < m; ++j) {
        const int32_t c = cols[j];
        if (c >= prev_lo && c < prev_hi) { prev |= 1ull << j; ++np; continue; }
        const int32_t lc = level[c];
        if (forward ? (lc >= lev - delta) : (lc <= lev + delta)) { late |= 1ull << j; ++nl; }
    }
    while (nl > QLATE) { // demote the late column farthest in level
        int worst = -1;
        int32_t wl = 0;
        for (int j = 0; j < m; ++j) {
            if (!((late >> j) & 1ull)) continue;
            const int32_t lc = level[cols[j]];
            if (worst < 0 || (forward ? lc < wl : lc > wl)) { worst = j; wl = lc; }
        }
        late &= ~(1ull << worst);
        --nl;
    }
    int k = 0;
    for (int j = 0; j < m; ++j)
        if (!(((late | prev) >> j) & 1ull)) { qcol[k] = cols[j]; qpos[k] = (uint8_t)j; ++k; }
    const int ne = k;
    unsigned long long left = late;
    while (left) { // selection by level: farthest first
        int best = -1;
        int32_t bl = 0;
        for (int j = 0; j < m; ++j) {
            if (!((left >> j) & 1ull)) continue;
            const int32_t lc = level[cols[j]];
            if (best < 0 || (forward ? lc < bl : lc > bl)) { best = j; bl = lc; }
        }
        left &= ~(1ull << best);
        qcol[k] = cols[best];
        qpos[k] = (uint8_t)best;
        ++k;
    }
    for (int j = 0; j < m; ++j)
        if ((prev >> j) & 1ull) { qcol[k] = cols[j]; qpos[k] = (uint8_t)j; ++k; }
    counts[0] = ne;
    counts[1] = nl;
    counts[2] = np;
}

__global__ void k_qsched(int32_t ngroups, const int32_t *grp, const int32_t *Lrowptr, const int32_t *Lcol,
                         const int32_t *Urowptr, const int32_t *Ucol, const int32_t *level, const int32_t *chunk_grp,
                         const int32_t *gchunk, int delta, int32_t *qf_col, uint8_t *qf_pos, int32_t *qf_cnt,
                         int32_t *qb_col, uint8_t *qb_pos, int32_t *qb_cnt)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = grp[g], G = grp[g + 1] - s, e = s + G - 1;
        const int32_t c = gchunk[g];
        const bool first = chunk_grp[c] == (int32_t)g, last = chunk_grp[c + 1] == (int32_t)g + 1;
        int cnt[3];
        // forward: external columns of row s, prev = the group before in the chunk
        const int32_t b0 = Lrowptr[s];
        const int m = Lrowptr[s + 1] - b0 - 1;
        q_classify(m, Lcol + b0, level, level[s], delta, true, first ? 0 : grp[g - 1], first ? 0 : s,
                   qf_col + b0, qf_pos + b0, cnt);
        qf_cnt[g] = cnt[0] | (cnt[1] << 8) | (cnt[2] << 16) | (G << 24);
        // backward: external columns of U row e, prev = the group after in the chunk
        const int32_t be = Urowptr[e], bu = Urowptr[s];
        const int mu = Urowptr[e + 1] - be - 1;
        q_classify(mu, Ucol + be + 1, level, level[e], delta, false, last ? 0 : grp[g + 1], last ? 0 : grp[g + 2],
                   qb_col + bu, qb_pos + bu, cnt);
        qb_cnt[g] = cnt[0] | (cnt[1] << 8) | (cnt[2] << 16) | (G << 24);
    }
}

static const int T_ROWS = 256;

static unsigned grid_rows(gic_handle *h, int64_t n)
{
    int64_t b = (n + T_ROWS - 1) / T_ROWS;
    int64_t cap = (int64_t)h->num_sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace gic

namespace gic {

int launch_persistent(gic_handle *h, const void *fn, int block, size_t smem, int64_t warps_needed, void **args)
{
    int per_sm = 0;
    GIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem));
    if (per_sm < 1) return GIC_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)per_sm * h->num_sms;
    int64_t need = (warps_needed * 32 + block - 1) / block;
    if (need < 1) need = 1;
    if (grid > need) grid = need;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++h->launches;
    GIC_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, args));
    return GIC_OK;
}

}  // namespace gic

using namespace gic;

static void free_pattern(Pattern &p)
{
    cudaFree(p.Lrowptr);
    cudaFree(p.Lcol);
    cudaFree(p.Urowptr);
    cudaFree(p.Ucol);
    cudaFree(p.tperm);
    cudaFree(p.grp);
    cudaFree(p.rowgrp);
    cudaFree(p.level);
    cudaFree(p.Lrow);
    cudaFree(p.chunk_grp);
    cudaFree(p.ord_f);
    cudaFree(p.ord_b);
    cudaFree(p.sell_ptr);
    cudaFree(p.sell_w);
    cudaFree(p.sell_col);
    cudaFree(p.qf_col);
    cudaFree(p.qb_col);
    cudaFree(p.qf_pos);
    cudaFree(p.qb_pos);
    cudaFree(p.qf_cnt);
    cudaFree(p.qb_cnt);
    free_ssched(p.sf);
    free_ssched(p.sb);
    free_psched(p.pf);
    free_psched(p.pb);
    cudaFree(p.glev);
    cudaFree(p.ic_ord);
    free_bsr(p);
    p = Pattern();
}

// Chunks, their sweep orders and the dependency check (see Pattern).
// Attempt 0: level-monotone runs of groups, swept in order of their first
// (forward) and last (backward) level. Attempt 1: the same runs in the order
// of their topological keys (k_chunk_keys). Attempt 2: one group per chunk in
// level order, which is always valid.
static int build_schedule(gic_handle *h, Pattern &P, int32_t *cflag, int32_t *cid, int32_t *lv_s, int32_t *lv_e)
{
    const int32_t ng = P.ngroups;
    unsigned gr = grid_rows(h, ng);
    long long tot = 0;
    ++h->launches;
    k_chunk_flags<<<gr, T_ROWS, 0, h->stream>>>(ng, P.grp, P.level, cflag);
    GIC_CUDA_TRY(cudaGetLastError());
    GIC_TRY(scan_i32<false>(h, cflag, ng, cid, &tot));
    int32_t nc = (int32_t)tot;
    int32_t *rowchunk = nullptr, *pos = nullptr, *keys = nullptr;
    unsigned *bad = (unsigned *)((char *)h->dev_small + 62000);
    std::vector<int32_t> hs, he, of, ob;
    int rc = GIC_OK;
    cudaError_t e = cudaMalloc(&rowchunk, sizeof(int32_t) * (size_t)P.n);
    for (int attempt = 0; attempt < 3 && e == cudaSuccess && rc == GIC_OK; ++attempt) {
        if (attempt != 1) {
            cudaFree(P.chunk_grp); cudaFree(P.ord_f); cudaFree(P.ord_b);
            cudaFree(pos); cudaFree(keys);
            P.chunk_grp = P.ord_f = P.ord_b = pos = keys = nullptr;
            if (attempt == 2) nc = ng;
            if ((e = cudaMalloc(&P.chunk_grp, sizeof(int32_t) * (size_t)(nc + 1))) != cudaSuccess) break;
            if ((e = cudaMalloc(&P.ord_f, sizeof(int32_t) * (size_t)nc)) != cudaSuccess) break;
            if ((e = cudaMalloc(&P.ord_b, sizeof(int32_t) * (size_t)nc)) != cudaSuccess) break;
            if ((e = cudaMalloc(&pos, sizeof(int32_t) * 2 * (size_t)nc)) != cudaSuccess) break;
            if ((e = cudaMalloc(&keys, sizeof(int32_t) * 2 * (size_t)nc)) != cudaSuccess) break;
            if (attempt == 0) {
                ++h->launches;
                k_chunk_starts<<<gr, T_ROWS, 0, h->stream>>>(ng, cflag, cid, P.chunk_grp, nc);
            } else {
                std::vector<int32_t> id(nc + 1);
                for (int32_t k = 0; k <= nc; ++k) id[k] = k;
                if ((e = cudaMemcpyAsync(P.chunk_grp, id.data(), sizeof(int32_t) * (size_t)(nc + 1),
                                         cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) break;
            }
            ++h->launches;
            k_chunk_levels<<<grid_rows(h, nc), T_ROWS, 0, h->stream>>>(nc, P.chunk_grp, P.grp, P.level, lv_s, lv_e);
            ++h->launches;
            k_row_chunk<<<grid_rows(h, nc), T_ROWS, 0, h->stream>>>(nc, P.chunk_grp, P.grp, rowchunk);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
        }
        const int32_t *ks = lv_s, *ke = lv_e;
        if (attempt == 1) {
            if ((e = cudaMemsetAsync(keys, 0xff, sizeof(int32_t) * 2 * (size_t)nc, h->stream)) != cudaSuccess) break;
            int32_t nc_ = nc, ml = P.nlevels - 1;
            const int32_t *cg = P.chunk_grp, *g_ = P.grp, *rc_ = rowchunk, *lr = P.Lrowptr, *lc = P.Lcol,
                          *ur = P.Urowptr, *uc = P.Ucol;
            int32_t *kf = keys, *kb = keys + nc;
            unsigned *er = h->dev_err;
            void *af[] = {&nc_, &cg, &g_, &lr, &lc, &rc_, &ks, &ml, &kf, &er};
            if ((rc = launch_persistent(h, (const void *)k_chunk_keys<false>, 256, 0, nc, af)) != GIC_OK) break;
            void *ab[] = {&nc_, &cg, &g_, &ur, &uc, &rc_, &ke, &ml, &kb, &er};
            if ((rc = launch_persistent(h, (const void *)k_chunk_keys<true>, 256, 0, nc, ab)) != GIC_OK) break;
            unsigned flags = 0;
            if ((rc = read_and_clear_dev_err(h, &flags)) != GIC_OK) break;
            if (flags) continue; // a key wait gave up: one group per chunk
            ks = kf;
            ke = kb;
        }
        hs.resize(nc); he.resize(nc); of.resize(nc); ob.resize(nc);
        if ((e = cudaMemcpyAsync(hs.data(), ks, sizeof(int32_t) * (size_t)nc, cudaMemcpyDeviceToHost, h->stream)) !=
            cudaSuccess) break;
        if ((e = cudaMemcpyAsync(he.data(), ke, sizeof(int32_t) * (size_t)nc, cudaMemcpyDeviceToHost, h->stream)) !=
            cudaSuccess) break;
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) break;
        for (int32_t k = 0; k < nc; ++k) of[k] = ob[k] = k;
        std::stable_sort(of.begin(), of.end(), [&](int32_t a, int32_t b) { return hs[a] < hs[b]; });
        if (attempt == 1) // backward keys ascend along the sweep
            std::stable_sort(ob.begin(), ob.end(), [&](int32_t a, int32_t b) { return he[a] < he[b]; });
        else
            std::stable_sort(ob.begin(), ob.end(), [&](int32_t a, int32_t b) { return he[a] > he[b]; });
        if ((e = cudaMemcpyAsync(P.ord_f, of.data(), sizeof(int32_t) * (size_t)nc, cudaMemcpyHostToDevice,
                                 h->stream)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(P.ord_b, ob.data(), sizeof(int32_t) * (size_t)nc, cudaMemcpyHostToDevice,
                                 h->stream)) != cudaSuccess) break;
        if (attempt == 2) { // level order per group is always valid
            P.chunked = 0;
            break;
        }
        ++h->launches;
        k_inverse_perm<<<grid_rows(h, nc), T_ROWS, 0, h->stream>>>(nc, P.ord_f, pos);
        ++h->launches;
        k_inverse_perm<<<grid_rows(h, nc), T_ROWS, 0, h->stream>>>(nc, P.ord_b, pos + nc);
        if ((e = cudaMemsetAsync(bad, 0, 4, h->stream)) != cudaSuccess) break;
        ++h->launches;
        k_check_order<<<gr, T_ROWS, 0, h->stream>>>(ng, P.grp, P.Lrowptr, P.Lcol, P.Urowptr, P.Ucol, rowchunk, pos,
                                                    pos + nc, bad);
        unsigned hb = 1;
        if ((e = cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) break;
        if (hb == 0) {
            P.chunked = (nc < ng) ? 1 + attempt : 0;
            break;
        }
    }
    cudaFree(rowchunk);
    cudaFree(pos);
    cudaFree(keys);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "gic_pattern_create", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    if (rc != GIC_OK) return rc;
    P.nchunks = nc;
    return GIC_OK;
}

static int build_sell(gic_handle *h, Pattern &P)
{
    P.nslices = (P.n + 31) / 32;
    GIC_CUDA_TRY(cudaMalloc(&P.sell_w, sizeof(int32_t) * (size_t)P.nslices));
    GIC_CUDA_TRY(cudaMalloc(&P.sell_ptr, sizeof(int64_t) * (size_t)(P.nslices + 1)));
    ++h->launches;
    k_sell_widths<<<grid_rows(h, P.nslices), T_ROWS, 0, h->stream>>>(P.n, P.nslices, P.rowptr, P.sell_w);
    GIC_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> w(P.nslices);
    std::vector<int64_t> ptr(P.nslices + 1);
    GIC_CUDA_TRY(cudaMemcpyAsync(w.data(), P.sell_w, sizeof(int32_t) * (size_t)P.nslices, cudaMemcpyDeviceToHost,
                                 h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    ptr[0] = 0;
    for (int64_t k = 0; k < P.nslices; ++k) ptr[k + 1] = ptr[k] + 32 * (int64_t)w[k];
    P.sell_nnz = ptr[P.nslices];
    GIC_CUDA_TRY(cudaMemcpyAsync(P.sell_ptr, ptr.data(), sizeof(int64_t) * (size_t)(P.nslices + 1),
                                 cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMalloc(&P.sell_col, sizeof(int32_t) * (size_t)P.sell_nnz));
    ++h->launches;
    k_sell_cols<<<grid_rows(h, P.nslices * 32), T_ROWS, 0, h->stream>>>(P.n, P.nslices, P.rowptr, P.col, P.sell_ptr,
                                                                        P.sell_w, P.sell_col);
    GIC_CUDA_TRY(cudaGetLastError());
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return GIC_OK;
}

// Schedule of the warp-specialised solves, where every group fits them.
static int build_qsched(gic_handle *h, Pattern &P)
{
    P.qready = 0;
    // a group's early columns and its own right-hand side share the 64 lane slots
    if (P.ngroups == 0 || P.max_group > 3 || P.max_ext_lower > QCOL - 3 || P.max_ext_upper > QCOL - 3) return GIC_OK;
    const size_t nL = (size_t)(P.nnzL > 0 ? P.nnzL : 1);
    GIC_CUDA_TRY(cudaMalloc(&P.qf_col, sizeof(int32_t) * nL));
    GIC_CUDA_TRY(cudaMalloc(&P.qb_col, sizeof(int32_t) * nL));
    GIC_CUDA_TRY(cudaMalloc(&P.qf_pos, nL));
    GIC_CUDA_TRY(cudaMalloc(&P.qb_pos, nL));
    GIC_CUDA_TRY(cudaMalloc(&P.qf_cnt, sizeof(int32_t) * (size_t)P.ngroups));
    GIC_CUDA_TRY(cudaMalloc(&P.qb_cnt, sizeof(int32_t) * (size_t)P.ngroups));
    int32_t *gchunk = nullptr;
    GIC_CUDA_TRY(cudaMalloc(&gchunk, sizeof(int32_t) * (size_t)P.ngroups));
    ++h->launches;
    k_group_chunk<<<grid_rows(h, P.nchunks), T_ROWS, 0, h->stream>>>(P.nchunks, P.chunk_grp, gchunk);
    ++h->launches;
    k_qsched<<<grid_rows(h, P.ngroups), T_ROWS, 0, h->stream>>>(P.ngroups, P.grp, P.Lrowptr, P.Lcol, P.Urowptr, P.Ucol,
                                                                 P.level, P.chunk_grp, gchunk, h->tune_qdelta,
                                                                 P.qf_col, P.qf_pos, P.qf_cnt, P.qb_col, P.qb_pos,
                                                                 P.qb_cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(gchunk);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "build_qsched", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    P.qdelta = h->tune_qdelta;
    P.qready = 1;
    return GIC_OK;
}


__global__ void k_group_glev(int32_t ngroups, const int32_t *grp, const int32_t *glev, int32_t *out)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
        out[g] = glev[grp[g]];
}

// IC(0)'s schedule: the groups in group-level order (stable counting sort
// on the host; index order within a level). Every dependency of a group is
// at a lower level, so a co-resident grid taking them round-robin always
// has the first unfinished one runnable.
static int build_ic_order(gic_handle *h, Pattern &P, int32_t *tmp)
{
    const int32_t ng = P.ngroups;
    if (ng == 0 || P.nglev <= 0) return GIC_OK;
    ++h->launches;
    k_group_glev<<<grid_rows(h, ng), T_ROWS, 0, h->stream>>>(ng, P.grp, P.glev, tmp);
    GIC_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> gl(ng), ord(ng);
    std::vector<int64_t> cnt((size_t)P.nglev + 1, 0);
    GIC_CUDA_TRY(cudaMemcpyAsync(gl.data(), tmp, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int32_t g = 0; g < ng; ++g) {
        if (gl[g] < 0 || gl[g] >= P.nglev) return GIC_ERR_INVALID_ARG;
        ++cnt[gl[g] + 1];
    }
    for (int32_t k = 0; k < P.nglev; ++k) cnt[k + 1] += cnt[k];
    for (int32_t g = 0; g < ng; ++g) ord[cnt[gl[g]]++] = g;
    GIC_CUDA_TRY(cudaMalloc(&P.ic_ord, 4 * (size_t)ng));
    GIC_CUDA_TRY(cudaMemcpyAsync(P.ic_ord, ord.data(), 4 * (size_t)ng, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return GIC_OK;
}

static int analyze_impl(gic_handle *h, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, Pattern &P)
{
    P.n = n;
    P.nnzA = nnz;
    P.rowptr = rowptr;
    P.col = col;
    P.device = h->device;
    int32_t *tmp = nullptr; // Lcnt | same | Ucnt | key | runstart | gflag | gid | stats(4)
    GIC_CUDA_TRY(cudaMalloc(&tmp, sizeof(int32_t) * (size_t)(7 * (n + 1) + 8)));
    int32_t *Lcnt = tmp, *same = tmp + (n + 1), *Ucnt = tmp + 2 * (n + 1), *key = tmp + 3 * (n + 1);
    int32_t *runstart = tmp + 4 * (n + 1), *gflag = tmp + 5 * (n + 1), *gid = tmp + 6 * (n + 1);
    int32_t *stats = tmp + 7 * (n + 1);
    int32_t *tmp2_a = key, *tmp2_b = runstart; // free again once the groups are built
    int rc = GIC_OK;
    long long tot = 0;
    unsigned flags = 0;
    unsigned gr = grid_rows(h, n);
#define STEP(x) do { rc = (x); if (rc != GIC_OK) goto out; } while (0)
#define CUDA_STEP(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda_error(e_, #x, __FILE__, __LINE__); rc = GIC_ERR_CUDA; goto out; } } while (0)
    CUDA_STEP(cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned), h->stream));
    CUDA_STEP(cudaMemsetAsync(stats, 0, sizeof(int32_t) * 8, h->stream));
    ++h->launches;
    k_validate<<<gr, T_ROWS, 0, h->stream>>>(n, nnz, rowptr, col, Lcnt, same, h->dev_err);
    CUDA_STEP(cudaGetLastError());
    STEP(read_and_clear_dev_err(h, &flags));
    if (flags) { rc = GIC_ERR_INVALID_ARG; goto out; }
    // only once every row is known to be in bounds
    ++h->launches;
    k_symcheck<<<gr, T_ROWS, 0, h->stream>>>(n, rowptr, col, h->dev_err);
    CUDA_STEP(cudaGetLastError());
    STEP(read_and_clear_dev_err(h, &flags));
    if (flags) { rc = GIC_ERR_INVALID_ARG; goto out; }

    CUDA_STEP(cudaMalloc(&P.Lrowptr, sizeof(int32_t) * (size_t)(n + 1)));
    STEP(scan_i32<false>(h, Lcnt, n, P.Lrowptr, &tot));
    P.nnzL = tot;
    CUDA_STEP(cudaMalloc(&P.Lcol, sizeof(int32_t) * (size_t)(P.nnzL > 0 ? P.nnzL : 1)));
    ++h->launches;
    k_fill_L<<<gr, T_ROWS, 0, h->stream>>>(n, rowptr, col, P.Lrowptr, P.Lcol, Ucnt);
    CUDA_STEP(cudaGetLastError());
    CUDA_STEP(cudaMalloc(&P.Lrow, sizeof(int32_t) * (size_t)(P.nnzL > 0 ? P.nnzL : 1)));
    ++h->launches;
    k_fill_Lrow<<<gr, T_ROWS, 0, h->stream>>>(n, P.Lrowptr, P.Lrow);
    CUDA_STEP(cudaMalloc(&P.Urowptr, sizeof(int32_t) * (size_t)(n + 1)));
    STEP(scan_i32<false>(h, Ucnt, n, P.Urowptr, &tot));
    if (tot != P.nnzL) { rc = GIC_ERR_INVALID_ARG; goto out; }
    CUDA_STEP(cudaMalloc(&P.Ucol, sizeof(int32_t) * (size_t)(P.nnzL > 0 ? P.nnzL : 1)));
    CUDA_STEP(cudaMalloc(&P.tperm, sizeof(int32_t) * (size_t)(P.nnzL > 0 ? P.nnzL : 1)));
    ++h->launches;
    k_fill_U<<<gr, T_ROWS, 0, h->stream>>>(n, rowptr, col, P.Lrowptr, P.Urowptr, P.Ucol, P.tperm);
    CUDA_STEP(cudaGetLastError());

    ++h->launches;

    k_run_keys<<<gr, T_ROWS, 0, h->stream>>>(n, same, key);
    STEP(scan_i32<true>(h, key, n, runstart, nullptr));
    {
        int32_t *bs = stats + 4, hb = 0;
        ++h->launches;
        k_run_gcd<<<gr, T_ROWS, 0, h->stream>>>(n, same, runstart, bs);
        CUDA_STEP(cudaGetLastError());
        CUDA_STEP(cudaMemcpyAsync(&hb, bs, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
        CUDA_STEP(cudaStreamSynchronize(h->stream));
        P.block_rows = (hb >= 2 && hb <= GMAX) ? hb : GMAX;
    }
    ++h->launches;
    k_group_flags<<<gr, T_ROWS, 0, h->stream>>>(n, runstart, P.block_rows, gflag);
    STEP(scan_i32<false>(h, gflag, n, gid, &tot));
    P.ngroups = (int32_t)tot;
    CUDA_STEP(cudaMalloc(&P.grp, sizeof(int32_t) * (size_t)(P.ngroups + 1)));
    ++h->launches;
    k_group_starts<<<gr, T_ROWS, 0, h->stream>>>(n, gflag, gid, P.grp, P.ngroups);
    CUDA_STEP(cudaMalloc(&P.rowgrp, sizeof(int32_t) * (size_t)(n > 0 ? n : 1)));
    ++h->launches;
    k_row_group<<<grid_rows(h, P.ngroups), T_ROWS, 0, h->stream>>>(P.ngroups, P.grp, P.rowgrp);
    ++h->launches;
    k_group_stats<<<grid_rows(h, P.ngroups), T_ROWS, 0, h->stream>>>(P.ngroups, P.grp, P.Lrowptr, P.Urowptr, stats);
    CUDA_STEP(cudaGetLastError());

    CUDA_STEP(cudaMalloc(&P.level, sizeof(int32_t) * (size_t)n));
    CUDA_STEP(cudaMemsetAsync(P.level, 0xff, sizeof(int32_t) * (size_t)n, h->stream));
    {
        // chains of groups (flags in gflag, their index in gid, starts in key)
        int32_t ng = P.ngroups;
        ++h->launches;
        k_chain_flags<<<grid_rows(h, ng), T_ROWS, 0, h->stream>>>(ng, P.grp, P.Lrowptr, P.Lcol, gflag);
        CUDA_STEP(cudaGetLastError());
        STEP(scan_i32<false>(h, gflag, ng, gid, &tot));
        int32_t nch = (int32_t)tot;
        ++h->launches;
        k_group_starts<<<grid_rows(h, ng), T_ROWS, 0, h->stream>>>(ng, gflag, gid, key, nch);
        CUDA_STEP(cudaGetLastError());
        const int32_t *ch = key, *g_ = P.grp, *lr = P.Lrowptr, *lc = P.Lcol;
        int32_t *lv = P.level, *ml = stats + 3;
        unsigned *er = h->dev_err;
        int rowstep = 1;
        void *args[] = {&nch, &ch, &g_, &lr, &lc, &rowstep, &lv, &ml, &er};
        STEP(launch_persistent(h, (const void *)k_levels, 256, 0, nch, args));
        // group levels (same chains), for the pair-sliced schedule
        CUDA_STEP(cudaMalloc(&P.glev, sizeof(int32_t) * (size_t)n));
        CUDA_STEP(cudaMemsetAsync(P.glev, 0xff, sizeof(int32_t) * (size_t)n, h->stream));
        lv = P.glev;
        ml = stats + 5;
        rowstep = 0;
        STEP(launch_persistent(h, (const void *)k_levels, 256, 0, nch, args));
    }
    {
        int32_t *hs = (int32_t *)h->host_pinned;
        CUDA_STEP(cudaMemcpyAsync(hs, stats, sizeof(int32_t) * 6, cudaMemcpyDeviceToHost, h->stream));
        CUDA_STEP(cudaStreamSynchronize(h->stream));
        P.max_ext_lower = hs[0];
        P.max_ext_upper = hs[1];
        P.max_group = hs[2];
        P.nlevels = n > 0 ? hs[3] + 1 : 0; // levels are 0-based
        P.nglev = n > 0 ? hs[5] + 1 : 0;
    }
    STEP(read_and_clear_dev_err(h, &flags));
    if (flags & ERR_TIMEOUT) { rc = GIC_ERR_TIMEOUT; goto out; }
    STEP(build_ic_order(h, P, gflag));
    STEP(build_schedule(h, P, gflag, gid, tmp2_a, tmp2_b));
    STEP(build_bsr(h, P));
    if (!P.bsr_ready) STEP(build_sell(h, P)); // the SELL-32 copy serves only patterns without node blocks
    STEP(build_qsched(h, P));
    STEP(build_ssched(h, P));
    STEP(build_psched(h, P));
out:
#undef STEP
#undef CUDA_STEP
    cudaFree(tmp);
    return rc;
}

extern "C" {

int gic_analyze(gic_handle *h, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, gic_pattern **P)
{
    GIC_TRY(check_handle(h));
    if (!P || !rowptr || !col || n < 1 || nnz < n) return GIC_ERR_INVALID_ARG;
    if (nnz >= (1ll << 31) || n >= (1ll << 31)) return GIC_ERR_TOO_LARGE;
    *P = nullptr;
    gic_pattern *out = new gic_pattern();
    int rc = analyze_impl(h, n, nnz, rowptr, col, out->p);
    if (rc != GIC_OK) {
        free_pattern(out->p);
        delete out;
        return rc;
    }
    *P = out;
    return GIC_OK;
}

int gic_pattern_destroy(gic_pattern *P)
{
    if (!P) return GIC_OK;
    cudaSetDevice(P->p.device);
    free_pattern(P->p);
    delete P;
    return GIC_OK;
}

int gic_pattern_info(const gic_pattern *P, int64_t *n, int64_t *nnzA, int64_t *nnzL, int32_t *nlevels,
                     int32_t *ngroups)
{
    if (!P) return GIC_ERR_INVALID_ARG;
    if (n) *n = P->p.n;
    if (nnzA) *nnzA = P->p.nnzA;
    if (nnzL) *nnzL = P->p.nnzL;
    if (nlevels) *nlevels = P->p.nlevels;
    if (ngroups) *ngroups = P->p.ngroups;
    return GIC_OK;
}

int gic_pattern_solve_kernels(const gic_pattern *P, int32_t *warp_specialised, int32_t *level_sliced,
                              int32_t *slices)
{
    if (!P) return GIC_ERR_INVALID_ARG;
    if (warp_specialised) *warp_specialised = P->p.qready;
    if (level_sliced) *level_sliced = P->p.sready;
    if (slices) *slices = P->p.sf.nsl;
    return GIC_OK;
}

int gic_pattern_pair_schedule(const gic_pattern *P, int32_t *mode, int32_t *slices, int32_t *glevels)
{
    if (!P) return GIC_ERR_INVALID_ARG;
    if (mode) *mode = P->p.pready ? P->p.pready : -P->p.pwhy;
    if (slices) *slices = P->p.pf.nsl;
    if (glevels) *glevels = P->p.nglev;
    return GIC_OK;
}

int gic_pattern_export(gic_handle *h, const gic_pattern *P, int32_t *Lrowptr, int32_t *Lcol, int32_t *level,
                       int32_t *group_start)
{
    GIC_TRY(check_handle(h));
    if (!P) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    if (Lrowptr)
        GIC_CUDA_TRY(cudaMemcpyAsync(Lrowptr, p.Lrowptr, sizeof(int32_t) * (size_t)(p.n + 1), cudaMemcpyDeviceToDevice, h->stream));
    if (Lcol)
        GIC_CUDA_TRY(cudaMemcpyAsync(Lcol, p.Lcol, sizeof(int32_t) * (size_t)p.nnzL, cudaMemcpyDeviceToDevice, h->stream));
    if (level)
        GIC_CUDA_TRY(cudaMemcpyAsync(level, p.level, sizeof(int32_t) * (size_t)p.n, cudaMemcpyDeviceToDevice, h->stream));
    if (group_start)
        GIC_CUDA_TRY(cudaMemcpyAsync(group_start, p.grp, sizeof(int32_t) * (size_t)(p.ngroups + 1), cudaMemcpyDeviceToDevice, h->stream));
    return GIC_OK;
}

}  // extern "C"
