// gic_extras.cu -- fill-in dropout (Supplementary 5, Eq. (10)), the factor
// deviation diagnostic of the paper's Figure 5, and the base factor of the
// direct-prediction variant (Eq. (1)).
#include <math.h>

#include "gic_internal.cuh"

namespace gic {

constexpr int X_BLOCK = 256;

static unsigned x_grid(gic_handle *h, int64_t n)
{
    int64_t b = (n + X_BLOCK - 1) / X_BLOCK, cap = (int64_t)h->num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// keep[p] for every L entry: the diagonal, and off-diagonal |L| > thr
__global__ void k_drop_keep(int64_t n, const int32_t *Lrowptr, const int32_t *Lcol, const double *Lval, double thr,
                            unsigned char *keep, int32_t *lcnt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        for (int32_t p = Lrowptr[i]; p < Lrowptr[i + 1]; ++p) {
            const bool k = (Lcol[p] == (int32_t)i) || (fabs(Lval[p]) > thr);
            keep[p] = k ? 1 : 0;
            c += k ? 1 : 0;
        }
        lcnt[i] = c;
    }
}

// Node-granular variant: the factor is cut into blocks by the row groups. An
// external block (rows of group g, columns of an earlier group h) stays whole
// if any of its entries exceeds thr and leaves whole otherwise; g's own lower
// block always stays. The rows of a group keep identical lower patterns and,
// through the transpose, identical upper ones, so the thinned factor keeps
// the row groups and the solve kernels built on them. One thread per group;
// a column's group is found by binary search over the group starts.
__global__ void k_drop_keep_grouped(int32_t ngroups, const int32_t *grp, const int32_t *Lrowptr, const int32_t *Lcol,
                                    const double *Lval, double thr, unsigned char *keep, int32_t *lcnt)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = grp[g], e = grp[g + 1];
        const int32_t b0 = Lrowptr[s];
        const int32_t m = Lrowptr[s + 1] - b0 - 1; // external columns, shared by the group's rows
        int32_t kept = 0;
        for (int32_t k = 0; k < m;) {
            const int32_t c = Lcol[b0 + k];
            int32_t lo = 0, hi = (int32_t)g; // the group h with grp[h] <= c < grp[h + 1]
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (grp[mid] <= c) lo = mid;
                else hi = mid;
            }
            const int32_t hend = grp[lo + 1];
            int32_t kend = k + 1;
            while (kend < m && Lcol[b0 + kend] < hend) ++kend;
            bool any = false;
            for (int32_t r = s; r < e; ++r)
                for (int32_t q = k; q < kend; ++q) any = any || (fabs(Lval[Lrowptr[r] + q]) > thr);
            for (int32_t r = s; r < e; ++r)
                for (int32_t q = k; q < kend; ++q) keep[Lrowptr[r] + q] = any ? 1 : 0;
            kept += any ? kend - k : 0;
            k = kend;
        }
        for (int32_t r = s; r < e; ++r) {
            for (int32_t p = Lrowptr[r] + m; p < Lrowptr[r + 1]; ++p) keep[p] = 1;
            lcnt[r] = kept + (Lrowptr[r + 1] - Lrowptr[r] - m);
        }
    }
}

// Per row of A: which entries stay in S = L' + L'^T. Lower entries map to L
// positions in order; upper entries of row i are the off-diagonal entries of
// U row i (the transpose of L) in the same order, whose L positions tperm
// holds.
__global__ void k_drop_rows(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *Lrowptr,
                            const int32_t *Urowptr, const int32_t *tperm, const unsigned char *keep, int32_t *scnt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0, lp = Lrowptr[i], uq = Urowptr[i] + 1;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int32_t j = col[p];
            if (j <= (int32_t)i) c += keep[lp++];
            else c += keep[tperm[uq++]];
        }
        scnt[i] = c;
    }
}

__global__ void k_drop_fill(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *Lrowptr,
                            const int32_t *Urowptr, const int32_t *tperm, const unsigned char *keep,
                            const double *Lval, const int32_t *Srowptr, const int32_t *Lout_ptr, int32_t *Scol,
                            double *Lout)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t lp = Lrowptr[i], uq = Urowptr[i] + 1, s = Srowptr[i], o = Lout_ptr[i];
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int32_t j = col[p];
            if (j <= (int32_t)i) {
                if (keep[lp]) {
                    Scol[s++] = j;
                    Lout[o++] = Lval[lp];
                }
                ++lp;
            } else {
                if (keep[tperm[uq]]) Scol[s++] = j;
                ++uq;
            }
        }
    }
}

// per-block partial sums of the deviation (deterministic: partials summed in
// block order by one thread)
__global__ void k_deviation(int64_t nnzL, const int32_t *Lrow, const int32_t *Lcol, const double *LIC,
                            const double *Lp, double *part)
{
    __shared__ double sh[6][X_BLOCK];
    double sd = 0.0, md = 0.0, so = 0.0, mo = 0.0, cd = 0.0, co = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnzL; p += (int64_t)gridDim.x * blockDim.x) {
        const double a = LIC[p];
        if (a == 0.0) continue;
        const double r = fabs(Lp[p] - a) / fabs(a);
        if (Lrow[p] == Lcol[p]) {
            sd += r;
            md = fmax(md, r);
            cd += 1.0;
        } else {
            so += r;
            mo = fmax(mo, r);
            co += 1.0;
        }
    }
    const int t = threadIdx.x;
    sh[0][t] = sd; sh[1][t] = md; sh[2][t] = so; sh[3][t] = mo; sh[4][t] = cd; sh[5][t] = co;
    __syncthreads();
    for (int o = X_BLOCK / 2; o > 0; o >>= 1) {
        if (t < o) {
            sh[0][t] += sh[0][t + o];
            sh[1][t] = fmax(sh[1][t], sh[1][t + o]);
            sh[2][t] += sh[2][t + o];
            sh[3][t] = fmax(sh[3][t], sh[3][t + o]);
            sh[4][t] += sh[4][t + o];
            sh[5][t] += sh[5][t + o];
        }
        __syncthreads();
    }
    if (t < 6) part[blockIdx.x * 6 + t] = sh[t][0];
}

__global__ void k_deviation_finish(int nb, const double *part, double *out)
{
    double sd = 0.0, md = 0.0, so = 0.0, mo = 0.0, cd = 0.0, co = 0.0;
    for (int b = 0; b < nb; ++b) {
        sd += part[b * 6 + 0];
        md = fmax(md, part[b * 6 + 1]);
        so += part[b * 6 + 2];
        mo = fmax(mo, part[b * 6 + 3]);
        cd += part[b * 6 + 4];
        co += part[b * 6 + 5];
    }
    out[0] = cd > 0.0 ? sd / cd : 0.0;
    out[1] = md;
    out[2] = co > 0.0 ? so / co : 0.0;
    out[3] = mo;
    out[4] = cd;
    out[5] = co;
}

__global__ void k_identity_factor(int64_t nnzL, int64_t ng_rows, const int32_t *Lrow, const int32_t *Lcol,
                                  const double *scale, double *L, float *Lhat)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnzL; p += (int64_t)gridDim.x * blockDim.x) {
        const bool diag = Lrow[p] == Lcol[p];
        if (L) L[p] = diag ? (scale ? sqrt(scale[Lrow[p] / ng_rows]) : 1.0) : 0.0;
        if (Lhat) Lhat[p] = diag ? 1.0f : 0.0f;
    }
}

}  // namespace gic

using namespace gic;

extern "C" {

static int dropout_impl(gic_handle *h, const gic_pattern *P, const double *valL, double threshold, bool grouped,
                        int32_t *Srowptr, int32_t *Scol, double *Lval_out, int64_t *nnzS, int64_t *nnzL_out)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device || !valL || !Srowptr || !Scol || !Lval_out || !(threshold >= 0.0))
        return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    const int64_t n = p.n;
    unsigned char *keep = nullptr;
    int32_t *cnt = nullptr;
    GIC_CUDA_TRY(cudaMalloc(&keep, (size_t)(p.nnzL > 0 ? p.nnzL : 1)));
    cudaError_t e = cudaMalloc(&cnt, sizeof(int32_t) * (size_t)(2 * n + 1));
    if (e != cudaSuccess) {
        cudaFree(keep);
        set_last_cuda_error(e, "gic_dropout", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    int32_t *lcnt = cnt, *lptr = cnt + n; // lptr: n + 1 entries
    long long tl = 0, ts = 0;
    int rc = GIC_OK;
    const unsigned g = x_grid(h, n);
    ++h->launches;
    if (grouped)
        k_drop_keep_grouped<<<x_grid(h, p.ngroups), X_BLOCK, 0, h->stream>>>(p.ngroups, p.grp, p.Lrowptr, p.Lcol,
                                                                            valL, threshold, keep, lcnt);
    else
        k_drop_keep<<<g, X_BLOCK, 0, h->stream>>>(n, p.Lrowptr, p.Lcol, valL, threshold, keep, lcnt);
    e = cudaGetLastError();
    if (e == cudaSuccess) rc = scan_excl_i32(h, lcnt, n, lptr, &tl);
    if (e == cudaSuccess && rc == GIC_OK) {
        ++h->launches;
        k_drop_rows<<<g, X_BLOCK, 0, h->stream>>>(n, p.rowptr, p.col, p.Lrowptr, p.Urowptr, p.tperm, keep, lcnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && rc == GIC_OK) rc = scan_excl_i32(h, lcnt, n, Srowptr, &ts);
    if (e == cudaSuccess && rc == GIC_OK) {
        ++h->launches;
        k_drop_fill<<<g, X_BLOCK, 0, h->stream>>>(n, p.rowptr, p.col, p.Lrowptr, p.Urowptr, p.tperm, keep, valL,
                                                  Srowptr, lptr, Scol, Lval_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && rc == GIC_OK) e = cudaStreamSynchronize(h->stream);
    cudaFree(keep);
    cudaFree(cnt);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "gic_dropout", __FILE__, __LINE__);
        return GIC_ERR_CUDA;
    }
    if (rc != GIC_OK) return rc;
    if (nnzS) *nnzS = ts;
    if (nnzL_out) *nnzL_out = tl;
    return GIC_OK;
}

int gic_dropout(gic_handle *h, const gic_pattern *P, const double *valL, double threshold, int32_t *Srowptr,
                int32_t *Scol, double *Lval_out, int64_t *nnzS, int64_t *nnzL_out)
{
    return dropout_impl(h, P, valL, threshold, false, Srowptr, Scol, Lval_out, nnzS, nnzL_out);
}

int gic_dropout_grouped(gic_handle *h, const gic_pattern *P, const double *valL, double threshold, int32_t *Srowptr,
                        int32_t *Scol, double *Lval_out, int64_t *nnzS, int64_t *nnzL_out)
{
    return dropout_impl(h, P, valL, threshold, true, Srowptr, Scol, Lval_out, nnzS, nnzL_out);
}

int gic_factor_deviation(gic_handle *h, const gic_pattern *P, const double *LIC, const double *Lpred, double *out)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device || !LIC || !Lpred || !out) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    const unsigned nb = x_grid(h, p.nnzL);
    double *part = (double *)h->dev_small; // nb * 6 + 6 doubles <= 64 KiB
    if ((size_t)(nb * 6 + 6) * sizeof(double) > 60000) return GIC_ERR_UNSUPPORTED;
    ++h->launches;
    k_deviation<<<nb, X_BLOCK, 0, h->stream>>>(p.nnzL, p.Lrow, p.Lcol, LIC, Lpred, part);
    ++h->launches;
    k_deviation_finish<<<1, 1, 0, h->stream>>>((int)nb, part, part + nb * 6);
    GIC_CUDA_TRY(cudaGetLastError());
    double *hp = (double *)h->host_pinned;
    GIC_CUDA_TRY(cudaMemcpyAsync(hp, part + nb * 6, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 6; ++k) out[k] = hp[k];
    return GIC_OK;
}

int gic_identity_factor(gic_handle *h, const gic_pattern *P, int ngraphs, const double *scale, double *L, float *Lhat)
{
    GIC_TRY(check_handle(h));
    if (!P || P->p.device != h->device || ngraphs < 1 || P->p.n % ngraphs != 0) return GIC_ERR_INVALID_ARG;
    const Pattern &p = P->p;
    if (!L && !Lhat) return GIC_OK;
    ++h->launches;
    k_identity_factor<<<x_grid(h, p.nnzL), X_BLOCK, 0, h->stream>>>(p.nnzL, p.n / ngraphs, p.Lrow, p.Lcol, scale, L,
                                                                     Lhat);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

}  // extern "C"
