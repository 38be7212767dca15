// gic_fem.cu -- A1: assembly of the synthetic 3-D elasticity systems.
//
// The paper's matrices come from 3-D static structural FE analysis
// (Experiments, Datasets; Supplementary 1). Stand-in: the unit cube cut into
// N^3 trilinear hex elements of side h = 1/N, isotropic material with
// Poisson ratio nu and per-element Young modulus E_e, z = 0 face clamped.
//
// Element matrix: for local nodes a, b and directions i, j
//   K_ab[i][j] = sum_gauss detJ * (lam dNa_i dNb_j + mu dNa_j dNb_i
//                                  + mu delta_ij grad Na . grad Nb)
// (the isotropic form of B^T D B), 2x2x2 Gauss points, E = 1.
// Global assembly is row-wise and atomic-free: every thread owns one row and
// sums, for each column, the contributions of the (at most 8) elements shared
// by the two nodes in ascending element order. rowptr is a closed form.
#include "gic_internal.cuh"

namespace gic {

// Ke (24x24, row-major, local dof 3a+i with a = ax + 2ay + 4az), E = 1.
__global__ void k_element_matrix(double nu, double h, double *Ke)
{
    int r = threadIdx.x / 24, c = threadIdx.x % 24;
    if (threadIdx.x >= 576) return;
    int a = r / 3, i = r % 3, b = c / 3, j = c % 3;
    double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = 0.5 / (1.0 + nu);
    double g = rsqrt(3.0);
    double detJ = 0.125 * h * h * h;
    double sum = 0.0;
    for (int q = 0; q < 8; ++q) {
        double p[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
        double ga[3], gb[3];
        for (int d = 0; d < 3; ++d) {
            // derivative of prod_k (1 + p_k s_k)/2 along d, times 2/h
            double fa = 1.0, fb = 1.0;
            for (int k = 0; k < 3; ++k) {
                double sa = ((a >> k) & 1) ? 1.0 : -1.0;
                double sb = ((b >> k) & 1) ? 1.0 : -1.0;
                fa *= (k == d) ? 0.5 * sa : 0.5 * (1.0 + p[k] * sa);
                fb *= (k == d) ? 0.5 * sb : 0.5 * (1.0 + p[k] * sb);
            }
            ga[d] = fa * 2.0 / h;
            gb[d] = fb * 2.0 / h;
        }
        double dot = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        sum += detJ * (lam * ga[i] * gb[j] + mu * ga[j] * gb[i] + (i == j ? mu * dot : 0.0));
    }
    Ke[r * 24 + c] = sum;
}

// 1D neighbour counts and their prefix sums along x/y (0..N) and z (1..N).
__device__ __forceinline__ int cnt_xy(int x, int N) { return 1 + (x > 0) + (x < N); }
__device__ __forceinline__ int pre_xy(int x) { return x == 0 ? 0 : 2 + 3 * (x - 1); }
__device__ __forceinline__ int cnt_z(int z, int N) { return 1 + (z > 1) + (z < N); }
__device__ __forceinline__ int pre_z(int z, int N)
{
    // sum of cnt_z over 1 <= z' < z
    if (z <= 1) return 0;
    if (N == 1) return 1;
    return 2 + 3 * (z - 2);
}

__global__ void k_assemble(int N, int nb, const double *E, const double *Ke_g, int32_t *rowptr, int32_t *col,
                           double *val, int64_t n1, int64_t nnz1)
{
    __shared__ double Ke[576];
    for (int t = threadIdx.x; t < 576; t += blockDim.x) Ke[t] = Ke_g[t];
    __syncthreads();
    const int M = N + 1;
    const int64_t W = 3 * (int64_t)N + 1;
    int64_t total = n1 * nb;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = gi / n1, i = gi % n1;
        int64_t node = i / 3;
        int c = (int)(i % 3);
        int x = (int)(node % M), y = (int)((node / M) % M), z = (int)(node / ((int64_t)M * M)) + 1;
        int cn = cnt_xy(x, N) * cnt_xy(y, N) * cnt_z(z, N);
        int64_t before = (int64_t)pre_z(z, N) * W * W + (int64_t)cnt_z(z, N) * ((int64_t)pre_xy(y) * W + (int64_t)cnt_xy(y, N) * pre_xy(x));
        int64_t base = k * nnz1 + 9 * before + (int64_t)c * 3 * cn;
        rowptr[gi] = (int32_t)base;
        if (gi == total - 1) rowptr[total] = (int32_t)(nb * nnz1);
        const double *Ek = E + k * (int64_t)N * N * N;
        int64_t off = k * n1;
        int64_t pos = base;
        for (int dz = -1; dz <= 1; ++dz) {
            int qz = z + dz;
            if (qz < 1 || qz > N) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int qy = y + dy;
                if (qy < 0 || qy > N) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = x + dx;
                    if (qx < 0 || qx > N) continue;
                    int64_t qnode = qx + (int64_t)M * (qy + (int64_t)M * (qz - 1));
                    double v[3] = {0.0, 0.0, 0.0};
                    // elements holding both nodes, ascending ez, ey, ex
                    for (int ez = max(z, qz) - 1; ez <= min(z, qz); ++ez) {
                        if (ez < 0 || ez >= N) continue;
                        for (int ey = max(y, qy) - 1; ey <= min(y, qy); ++ey) {
                            if (ey < 0 || ey >= N) continue;
                            for (int ex = max(x, qx) - 1; ex <= min(x, qx); ++ex) {
                                if (ex < 0 || ex >= N) continue;
                                double Ee = Ek[ex + (int64_t)N * (ey + (int64_t)N * ez)];
                                int la = (x - ex) + 2 * (y - ey) + 4 * (z - ez);
                                int lb = (qx - ex) + 2 * (qy - ey) + 4 * (qz - ez);
                                const double *row = Ke + (3 * la + c) * 24 + 3 * lb;
                                v[0] += Ee * row[0];
                                v[1] += Ee * row[1];
                                v[2] += Ee * row[2];
                            }
                        }
                    }
                    for (int d = 0; d < 3; ++d) {
                        col[pos] = (int32_t)(off + 3 * qnode + d);
                        val[pos] = v[d];
                        ++pos;
                    }
                }
            }
        }
    }
}

}  // namespace gic

using namespace gic;

extern "C" {

int gic_fem_hex_sizes(int N, int64_t *n, int64_t *nnz)
{
    if (N < 1 || N > 100000 || !n || !nnz) return GIC_ERR_INVALID_ARG;
    int64_t nn = 3 * (int64_t)N * (N + 1) * (N + 1);
    int64_t w = 3 * (int64_t)N + 1;
    int64_t nz = (N == 1) ? 9 * 4 * 4 * 1 : 9 * w * w * (3 * (int64_t)N - 2);
    *n = nn;
    *nnz = nz;
    return GIC_OK;
}

int gic_fem_hex_assemble(gic_handle *h, int N, double nu, int nb, const double *E, int32_t *rowptr, int32_t *col,
                         double *val)
{
    GIC_TRY(check_handle(h));
    int64_t n1, nnz1;
    GIC_TRY(gic_fem_hex_sizes(N, &n1, &nnz1));
    if (nb < 1 || !E || !rowptr || !col || !val || !(nu > -1.0 && nu < 0.5)) return GIC_ERR_INVALID_ARG;
    if (nnz1 * nb >= (1ll << 31)) return GIC_ERR_TOO_LARGE;
    double *Ke = (double *)h->dev_small;
    ++h->launches;
    k_element_matrix<<<1, 576, 0, h->stream>>>(nu, 1.0 / N, Ke);
    int64_t rows = n1 * nb;
    int64_t blocks = (rows + 255) / 256;
    if (blocks > (int64_t)h->num_sms * 32) blocks = (int64_t)h->num_sms * 32;
    ++h->launches;
    k_assemble<<<(unsigned)blocks, 256, 0, h->stream>>>(N, nb, E, Ke, rowptr, col, val, n1, nnz1);
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

}  // extern "C"
