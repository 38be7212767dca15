// gic_host.cu -- end-to-end solve from host buffers (the black-box view of
// PCG in Supplementary 2: A and b in, x out), built from the other entry
// points: H2D copies, analysis, IC(0) with shift restart, optional GNN
// correction, PCG, D2H copy of x.
#include "gic_internal.cuh"

namespace gic {

static size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

struct HostWs {
    int32_t *rowptr, *col;
    double *val, *b, *x, *L;
    float *L32;
    void *gnn;
    void *pcg;
    size_t pcg_bytes, gnn_bytes, bytes;
};

static HostWs carve_host(int64_t n, int64_t nnz, int with_gnn, int l_dtype, void *base)
{
    HostWs o = {};
    char *c = (char *)base;
    size_t off = 0;
    int64_t nnzL = (nnz + n) / 2;
    o.rowptr = (int32_t *)(c + off); off += al(4 * (size_t)(n + 1));
    o.col = (int32_t *)(c + off); off += al(4 * (size_t)nnz);
    o.val = (double *)(c + off); off += al(8 * (size_t)nnz);
    o.b = (double *)(c + off); off += al(8 * (size_t)n);
    o.x = (double *)(c + off); off += al(8 * (size_t)n);
    o.L = (double *)(c + off); off += al(8 * (size_t)nnzL);
    o.L32 = (float *)(c + off); off += (l_dtype == GIC_F32) ? al(4 * (size_t)nnzL) : 0;
    o.gnn_bytes = with_gnn ? gnn_infer_ws_bytes(n, nnzL) : 0;
    o.gnn = c + off; off += al(o.gnn_bytes);
    // SELL-32 padding: at most 31 entries of padding per row beyond A's own
    o.pcg_bytes = pcg_ws_bytes(n, nnzL, nnz + 32 * n, l_dtype);
    o.pcg = c + off; off += al(o.pcg_bytes);
    o.bytes = off;
    return o;
}

}  // namespace gic

using namespace gic;

extern "C" {

int gic_solve_host_workspace_size(gic_handle *h, int64_t n, int64_t nnz, int with_gnn, int l_dtype, size_t *bytes)
{
    if (!h || !bytes || n < 1 || nnz < n || (l_dtype != GIC_F64 && l_dtype != GIC_F32)) return GIC_ERR_INVALID_ARG;
    *bytes = carve_host(n, nnz, with_gnn, l_dtype, nullptr).bytes;
    return GIC_OK;
}

int gic_solve_host(gic_handle *h, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                   const double *val, const double *b, double *x, const float *theta, int l_dtype, double rtol,
                   int maxit, int32_t *iters, double *relres, double *alpha, int *used_gnn, void *ws,
                   size_t ws_bytes)
{
    GIC_TRY(check_handle(h));
    if (!rowptr || !col || !val || !b || !x || !ws || n < 1 || nnz < n) return GIC_ERR_INVALID_ARG;
    if (l_dtype != GIC_F64 && l_dtype != GIC_F32) return GIC_ERR_INVALID_ARG;
    if (nnz >= (1ll << 31)) return GIC_ERR_TOO_LARGE;
    HostWs W = carve_host(n, nnz, theta != nullptr, l_dtype, ws);
    if (ws_bytes < W.bytes) return GIC_ERR_WORKSPACE;
    cudaStream_t s = h->stream;
    GIC_CUDA_TRY(cudaMemcpyAsync(W.rowptr, rowptr, 4 * (size_t)(n + 1), cudaMemcpyHostToDevice, s));
    GIC_CUDA_TRY(cudaMemcpyAsync(W.col, col, 4 * (size_t)nnz, cudaMemcpyHostToDevice, s));
    GIC_CUDA_TRY(cudaMemcpyAsync(W.val, val, 8 * (size_t)nnz, cudaMemcpyHostToDevice, s));
    GIC_CUDA_TRY(cudaMemcpyAsync(W.b, b, 8 * (size_t)n, cudaMemcpyHostToDevice, s));
    GIC_CUDA_TRY(cudaMemsetAsync(W.x, 0, 8 * (size_t)n, s));
    gic_pattern *P = nullptr;
    int rc = gic_analyze(h, n, nnz, W.rowptr, W.col, &P);
    if (rc != GIC_OK) return rc;
    double a = 0.0;
    int64_t bad = -1;
    int gnn_kept = 0;
    rc = gic_ic0_auto(h, P, W.val, W.L, 20, &a, &bad);
    if (rc == GIC_OK && theta) rc = gnn_correct_inplace(h, P, W.val, theta, W.L, W.gnn, W.gnn_bytes, &gnn_kept);
    if (rc == GIC_OK && l_dtype == GIC_F32) rc = gic_convert_f64_f32(h, P->p.nnzL, W.L, W.L32);
    if (rc == GIC_OK) {
        const void *Lp = (l_dtype == GIC_F32) ? (const void *)W.L32 : (const void *)W.L;
        rc = gic_pcg(h, P, W.val, Lp, l_dtype, W.b, W.x, rtol, maxit, iters, relres, W.pcg, W.pcg_bytes);
    }
    if (rc == GIC_OK || rc == GIC_ERR_NO_CONVERGENCE) {
        cudaError_t e = cudaMemcpyAsync(x, W.x, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_last_cuda_error(e, "gic_solve_host readback", __FILE__, __LINE__);
            rc = GIC_ERR_CUDA;
        }
    }
    gic_pattern_destroy(P);
    if (alpha) *alpha = a;
    if (used_gnn) *used_gnn = gnn_kept;
    return rc;
}

}  // extern "C"
