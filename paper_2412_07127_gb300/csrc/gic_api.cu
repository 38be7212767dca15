// gic_api.cu -- handle lifecycle, status text and error plumbing of the C-ABI.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gic_internal.cuh"

namespace gic {

static char g_last_cuda_error[512] = "";

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s (%d) in %s at %s:%d",
             cudaGetErrorString(e), (int)e, what, file, line);
}

int check_handle(gic_handle *h)
{
    if (!h) return GIC_ERR_INVALID_ARG;
    GIC_CUDA_TRY(cudaSetDevice(h->device));
    return GIC_OK;
}

int read_and_clear_dev_err(gic_handle *h, unsigned *flags)
{
    unsigned *hp = (unsigned *)h->host_pinned;
    GIC_CUDA_TRY(cudaMemcpyAsync(hp, h->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned), h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    *flags = hp[0];
    return GIC_OK;
}

}  // namespace gic

extern "C" {

int gic_create(gic_handle **out, int device, void *stream)
{
    if (!out) return GIC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    GIC_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return GIC_ERR_INVALID_ARG;
    GIC_CUDA_TRY(cudaSetDevice(device));
    gic_handle *h = new gic_handle();
    h->device = device;
    h->stream = (cudaStream_t)stream;
    cudaError_t e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&h->dev_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&h->dev_small, 65536);
    if (e == cudaSuccess) e = cudaMallocHost(&h->host_pinned, 4096);
    if (e != cudaSuccess) {
        gic::set_last_cuda_error(e, "gic_create", __FILE__, __LINE__);
        gic_destroy(h);
        return GIC_ERR_CUDA;
    }
    *out = h;
    return GIC_OK;
}

int gic_set_stream(gic_handle *h, void *stream)
{
    if (!h) return GIC_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return GIC_OK;
}

int gic_destroy(gic_handle *h)
{
    if (!h) return GIC_OK;
    cudaSetDevice(h->device);
    if (h->dev_err) cudaFree(h->dev_err);
    if (h->dev_small) cudaFree(h->dev_small);
    if (h->host_pinned) cudaFreeHost(h->host_pinned);
    delete h;
    return GIC_OK;
}

const char *gic_status_string(int s)
{
    switch (s) {
    case GIC_OK: return "ok";
    case GIC_ERR_INVALID_ARG: return "invalid argument";
    case GIC_ERR_NOT_SPD: return "IC(0) pivot not positive (matrix not SPD enough for IC(0))";
    case GIC_ERR_NO_CONVERGENCE: return "PCG reached the iteration limit";
    case GIC_ERR_TIMEOUT: return "a bounded device wait ran out";
    case GIC_ERR_CUDA: return "CUDA runtime error";
    case GIC_ERR_TOO_LARGE: return "sizes beyond int32 indexing";
    case GIC_ERR_UNSUPPORTED: return "pattern outside the kernels' limits";
    case GIC_ERR_BREAKDOWN: return "PCG breakdown (r^T z <= 0 or p^T A p <= 0)";
    case GIC_ERR_WORKSPACE: return "workspace too small";
    default: return "unknown status";
    }
}

const char *gic_last_cuda_error(void) { return gic::g_last_cuda_error; }

}  // extern "C"

namespace gic {
// one warp waits on a word that nothing writes, with a caller-chosen limit
__global__ void k_selftest_wait(double *cell, unsigned *err, long long limit)
{
    if (threadIdx.x == 0) wait_value(cell, err, limit);
}
__global__ void k_selftest_arm(double *cell) { *cell = sentinel_d(); }
}  // namespace gic

extern "C" {

int gic_selftest_wait_timeout(gic_handle *h, int64_t polls)
{
    GIC_TRY(gic::check_handle(h));
    if (polls < 1 || polls > (1ll << 21)) return GIC_ERR_INVALID_ARG;
    double *cell = (double *)((char *)h->dev_small + 63000);
    ++h->launches;
    gic::k_selftest_arm<<<1, 1, 0, h->stream>>>(cell);
    ++h->launches;
    gic::k_selftest_wait<<<1, 32, 0, h->stream>>>(cell, h->dev_err, (long long)polls);
    GIC_CUDA_TRY(cudaGetLastError());
    unsigned flags = 0;
    GIC_TRY(gic::read_and_clear_dev_err(h, &flags));
    return (flags & gic::ERR_TIMEOUT) ? GIC_ERR_TIMEOUT : GIC_OK;
}

}  // extern "C"
