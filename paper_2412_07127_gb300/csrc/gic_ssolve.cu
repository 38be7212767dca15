// gic_ssolve.cu -- A7b: level-sliced sync-free triangular solves, one lane per
// row, for patterns the warp-specialised schedule admits (row groups of at
// most 3 rows with at most QCOL - 3 external columns).
//
// The rows of a group are solved in the premultiplied form of the
// warp-specialised kernels (Eq. (11) read as forward substitution, with the
// group's dense diagonal block D inverted once per factor, M = D^-1):
//     forward   y_g = M r_g - (M L_ext) y_ext,
//     backward  z_g = M^T y_g - (M^T U_ext) z_ext,
// so every row is an independent dot product over the group's external
// columns. Here those dot products are spread one row per lane: the groups
// of a sweep are sorted by level (forward: the level of their first row,
// ascending; backward: of their last row, descending) and cut into slices of
// whole groups with at most 32 rows that never span two levels, so the rows
// of a slice never depend on each other. A slice's coefficients are stored
// step by step (step k: one value per lane, 32 consecutive words), its
// columns step by step per group (the rows of a group share them), each
// group's list front-padded to the slice's width so that the columns
// finished last (the nearest levels) come last for every lane.
//
// Why a second kernel family: an FP64 warp instruction occupies this GPU's
// FP64 pipe for ~17 cycles however few of its lanes are active. The
// warp-specialised kernels spend ~20 FP64 warp instructions per 3-row group
// (lane-parallel products, a cross-lane reduction, a finisher on 12 lanes);
// on large systems, where thousands of groups are ready at once, that issue
// cost is the bound. Lane-per-row slices spend one FP64 instruction per
// column step for 30 rows and need no reduction. On small systems, where the
// dependency chain rather than the throughput sets the time, the
// warp-specialised kernels stay faster.
//
// Warps take slices round-robin in sweep order (every warp of the grid is
// resident: cooperative launch), so the first unfinished slice can always
// run; readiness is the solution word itself (the sentinel until written)
// and every wait is bounded.
#include <algorithm>
#include <vector>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int SBLOCK = 256;        // threads per block of the sliced solves
constexpr int SBATCH = 10;         // early column steps whose loads are in flight together
constexpr int SLATE = QLATE + 3;   // late + previous-group steps of a slice, loaded at once
constexpr int SNEAR = 9;           // of which the last ones, summed after the others

// Kernel view of one sweep's slice schedule.
struct SliceView {
    int32_t nsl;
    const int32_t *w, *we, *ng;
    const int64_t *kv, *kc;
    const int2 *lane;
    const int32_t *col;
};

static SliceView view_of(const SliceSched &S)
{
    return SliceView{S.nsl, S.w, S.we, S.ng, S.kv, S.kc, S.lane, S.col};
}

// FWD: L y = r (x = y, rhs = r). Backward: L^T z = y (x = z, rhs = y); with
// PCG it also resets y to the sentinel for the next forward sweep and forms
// r^T z in FP64, then beta = r_k^T z_k / r_{k-1}^T z_{k-1} (Algorithm 1) in
// the last warp to finish. x must hold the sentinel. kval: step-major
// coefficients (-K), 32 per step; mval: 3 x 32 in-group coefficients per
// slice (forward M_tu, backward M_ut, zero where unused).
template <typename T, bool FWD, bool PCG>
__global__ void __launch_bounds__(SBLOCK, 2) k_ssolve(SliceView S, const T *__restrict__ kval, const T *__restrict__ mval,
                                                   const T *rhs, T *x, T *yreset, const double *__restrict__ rd,
                                                   double *partials, unsigned *err, int poll, Scalars *sc)
{
    if (sc && sc->done) return;
    __shared__ __align__(16) T s_klate[SBLOCK / 32][SLATE * 32]; // each warp's late coefficients
    const int lane = threadIdx.x & 31;
    T *klate = s_klate[threadIdx.x >> 5];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned sleep_ns = (unsigned)(poll & 0xffff);
    double dot = 0.0;
    // the next slice's header is loaded while the current one runs, and a
    // slice's own right-hand side, in-group coefficients and (PCG) r values
    // are requested before its first wait and consumed after its last, so no
    // warp stalls on a load that does not depend on another row
    int64_t sl = gw;
    int hW = 0, hWe = 0, hng = 0;
    int64_t hkv = 0, hkc = 0;
    int2 hd = make_int2(-1, 0);
    if (sl < S.nsl) {
        hW = S.w[sl], hWe = S.we[sl], hng = S.ng[sl];
        hkv = S.kv[sl], hkc = S.kc[sl];
        hd = S.lane[sl * 32 + lane];
    }
    for (; sl < S.nsl; sl += nw) {
        const int W = hW, We = hWe, Wl = W - We, ng = hng;
        const int64_t kv0 = hkv, kc0 = hkc;
        const int2 d = hd;
        const int32_t row = d.x;
        const int slot = d.y & 255, t = (d.y >> 8) & 255, G = (d.y >> 16) & 255;
        const bool act = row >= 0;
        const int32_t s = row - t;
        T mv[3], rv[3];
        double rdv = 0.0;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            mv[u] = (act && u < G) ? mval[sl * 96 + u * 32 + lane] : (T)0;
            rv[u] = (act && u < G) ? rhs[s + u] : (T)0;
        }
        if (PCG && act) rdv = rd[row];
        const int64_t sn = sl + nw;
        if (sn < S.nsl) {
            hW = S.w[sn], hWe = S.we[sn], hng = S.ng[sn];
            hkv = S.kv[sn], hkc = S.kc[sn];
            hd = S.lane[sn * 32 + lane];
        }
        T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
        const int32_t *cp = S.col + kc0 + slot;
        const T *kp = kval + kv0 * 32 + lane;
        for (int b = 0; b < Wl; ++b) cp_async_t(&klate[b * 32 + lane], kp + (int64_t)(We + b) * 32);
        cp_async_commit();
        // early section (columns finished well before the slice's level): in
        // batches, the next batch's columns and coefficients loaded while one
        // waits; the warp stays converged (one wait loop per batch)
        int32_t c[SBATCH];
        T kv[SBATCH];
#pragma unroll
        for (int b = 0; b < SBATCH; ++b) {
            c[b] = (act && b < We) ? cp[(int64_t)b * ng] : -1;
            kv[b] = (b < We) ? kp[(int64_t)b * 32] : (T)0;
        }
        for (int k0 = 0; k0 < We; k0 += SBATCH) {
            T v[SBATCH];
#pragma unroll
            for (int b = 0; b < SBATCH; ++b) v[b] = (c[b] >= 0) ? ld_relaxed(x + c[b]) : (T)0;
            int32_t cn[SBATCH];
            T kn[SBATCH];
#pragma unroll
            for (int b = 0; b < SBATCH; ++b) {
                const int k = k0 + SBATCH + b;
                cn[b] = (act && k < We) ? cp[(int64_t)k * ng] : -1;
                kn[b] = (k < We) ? kp[(int64_t)k * 32] : (T)0;
            }
            slice_wait<T, SBATCH>(x, c, v, err, sleep_ns, lane);
#pragma unroll
            for (int b = 0; b < SBATCH; ++b) {
                if (k0 + b < We) { // uniform over the warp
                    if (b & 1) acc1 = fma(kv[b], v[b], acc1);
                    else acc0 = fma(kv[b], v[b], acc0);
                }
            }
#pragma unroll
            for (int b = 0; b < SBATCH; ++b) {
                c[b] = cn[b];
                kv[b] = kn[b];
            }
        }
        // the group's own right-hand side M r (zero where unused), off the
        // chain that follows the late values
#pragma unroll
        for (int u = 0; u < 3; ++u) acc1 = fma(mv[u], rv[u], acc1);
        // late section (the nearest levels and the previous group of the
        // chunk): every value is requested at once, then summed in two waves,
        // the last SNEAR steps (for hex elasticity: the level just before)
        // after the others, so that once the last value lands a single poll
        // round and a few FMAs remain. Its coefficients were copied into the
        // warp's shared memory at the start of the slice.
        {
            constexpr int SFAR = SLATE - SNEAR;
            const int Wn = Wl < SNEAR ? Wl : SNEAR, Wf = Wl - Wn;
            int32_t cf[SFAR], cn2[SNEAR];
            T vf[SFAR], vn[SNEAR];
#pragma unroll
            for (int b = 0; b < SFAR; ++b) cf[b] = (act && b < Wf) ? cp[(int64_t)(We + b) * ng] : -1;
#pragma unroll
            for (int b = 0; b < SNEAR; ++b) cn2[b] = (act && b < Wn) ? cp[(int64_t)(We + Wf + b) * ng] : -1;
#pragma unroll
            for (int b = 0; b < SFAR; ++b) vf[b] = (cf[b] >= 0) ? ld_relaxed(x + cf[b]) : (T)0;
#pragma unroll
            for (int b = 0; b < SNEAR; ++b) vn[b] = (cn2[b] >= 0) ? ld_relaxed(x + cn2[b]) : (T)0;
            cp_async_wait<0>(); // this lane's late coefficients are in shared memory
            slice_wait<T, SFAR>(x, cf, vf, err, sleep_ns, lane);
#pragma unroll
            for (int b = 0; b < SFAR; ++b) {
                if (b < Wf) { // uniform over the warp
                    const T kb = klate[b * 32 + lane];
                    if ((b & 3) == 0) acc0 = fma(kb, vf[b], acc0);
                    else if ((b & 3) == 1) acc1 = fma(kb, vf[b], acc1);
                    else if ((b & 3) == 2) acc2 = fma(kb, vf[b], acc2);
                    else acc3 = fma(kb, vf[b], acc3);
                }
            }
            slice_wait<T, SNEAR>(x, cn2, vn, err, sleep_ns, lane);
#pragma unroll
            for (int b = 0; b < SNEAR; ++b) {
                if (b < Wn) {
                    const T kb = klate[(Wf + b) * 32 + lane];
                    if (b % 3 == 0) acc0 = fma(kb, vn[b], acc0);
                    else if (b % 3 == 1) acc2 = fma(kb, vn[b], acc2);
                    else acc3 = fma(kb, vn[b], acc3);
                }
            }
        }
        const T y = (acc0 + acc1) + (acc2 + acc3);
        // the rows of a group (its own slice, this warp) read their right-hand
        // side before any lane resets it; the warp enters the next slice together
        __syncwarp();
        if (act) {
            st_relaxed(x + row, y);
            if (PCG) {
                yreset[row] = sentinel_of<T>();
                dot = fma(rdv, (double)y, dot);
            }
        }
    }
    if (PCG) {
        dot = warp_sum(dot);
        if (lane == 0) partials[gw] = dot;
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence();
            last = (atomicAdd(&sc->counter, 1u) == (unsigned)nw - 1u);
        }
        last = __shfl_sync(0xffffffffu, last, 0);
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

// Coefficients of a factor in the slice layout, one thread per lane of a
// slice, computed in FP64 and stored in TL: the group's diagonal block D
// (lower, dense), M = D^-1, then forward K_t = sum_{u<=t} M_tu L_ext(s+u)
// over the group's columns in the schedule order (qf_pos: position of each
// column in the rows' external part), backward K_t = sum_{u>=t} M_ut
// U_ext(s+u) (qb_pos, U values through tperm). Padding and idle lanes get 0.
template <typename TL, bool FWD>
__global__ void k_ssetup(SliceView S, const int32_t *__restrict__ Lrowptr, const int32_t *__restrict__ Urowptr,
                         const int32_t *__restrict__ tperm, const uint8_t *__restrict__ qpos,
                         const TL *__restrict__ Lval, TL *__restrict__ kval, TL *__restrict__ mval)
{
    const int64_t total = (int64_t)S.nsl * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i >> 5;
        const int l = (int)(i & 31);
        const int W = S.w[sl];
        const int64_t kv0 = S.kv[sl];
        const int2 d = S.lane[i];
        const int32_t row = d.x;
        TL *kp = kval + kv0 * 32 + l;
        if (row < 0) {
            for (int k = 0; k < W; ++k) kp[(int64_t)k * 32] = (TL)0;
            for (int u = 0; u < 3; ++u) mval[sl * 96 + u * 32 + l] = (TL)0;
            continue;
        }
        const int t = (d.y >> 8) & 255, G = (d.y >> 16) & 255;
        const int32_t s = row - t, e = s + G - 1;
        const int64_t b0 = Lrowptr[s];
        const int m = (int)(Lrowptr[s + 1] - b0 - 1); // external columns of the group's rows
        double D[3][3] = {}, M[3][3] = {};
        for (int a = 0; a < G; ++a)
            for (int u = 0; u <= a; ++u) D[a][u] = (double)Lval[Lrowptr[s + a] + m + u];
        for (int a = 0; a < G; ++a) {
            M[a][a] = 1.0 / D[a][a];
            for (int u = 0; u < a; ++u) {
                double acc = 0.0;
                for (int v = u; v < a; ++v) acc = fma(D[a][v], M[v][u], acc);
                M[a][u] = -acc * M[a][a];
            }
        }
        // schedule position of step k: the early part front-padded to We,
        // the late part front-padded to W - We
        const int We = S.we[sl], ne = (d.y >> 24) & 255;
        auto pos_of = [&](int k, int mm) {
            if (k < We) return k - (We - ne);
            return ne + (k - We) - ((W - We) - (mm - ne));
        };
        if (FWD) {
            for (int k = 0; k < W; ++k) {
                const int q = pos_of(k, m);
                double acc = 0.0;
                if ((k < We) ? (q >= 0) : (q >= ne)) { // else padding
                    const int j = qpos[b0 + q];
                    for (int u = 0; u <= t; ++u) acc = fma(M[t][u], (double)Lval[Lrowptr[s + u] + j], acc);
                }
                kp[(int64_t)k * 32] = (TL)(-acc);
            }
            for (int u = 0; u < 3; ++u) mval[sl * 96 + u * 32 + l] = (TL)((u <= t && u < G) ? M[t][u] : 0.0);
        } else {
            const int64_t bu = Urowptr[s];
            const int mu = (int)(Urowptr[e + 1] - Urowptr[e] - 1);
            for (int k = 0; k < W; ++k) {
                const int q = pos_of(k, mu);
                double acc = 0.0;
                if ((k < We) ? (q >= 0) : (q >= ne)) { // else padding
                    const int j = qpos[bu + q];
                    for (int u = t; u < G; ++u)
                        acc = fma(M[u][t], (double)Lval[tperm[Urowptr[s + u] + (G - u) + j]], acc);
                }
                kp[(int64_t)k * 32] = (TL)(-acc);
            }
            for (int u = 0; u < 3; ++u) mval[sl * 96 + u * 32 + l] = (TL)((u >= t && u < G) ? M[u][t] : 0.0);
        }
    }
}

// Column lists of the slices: the first lane of every group writes the
// group's columns at its slot, the early ones (schedule order) front-padded
// with -1 to the slice's early width, then the late and previous-group ones
// front-padded to the rest of the width.
__global__ void k_scols(SliceView S, const int32_t *__restrict__ Xrowptr, const int32_t *__restrict__ qcol,
                        const int32_t *__restrict__ qcnt, const int32_t *__restrict__ rowgrp_id, int32_t *col)
{
    const int64_t total = (int64_t)S.nsl * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 d = S.lane[i];
        if (d.x < 0 || ((d.y >> 8) & 255) != 0) continue;
        const int64_t sl = i >> 5;
        const int W = S.w[sl], We = S.we[sl], ng = S.ng[sl], slot = d.y & 255;
        const int32_t s = d.x;
        const int32_t cw = qcnt[rowgrp_id[s]];
        const int ne = cw & 255, nlp = ((cw >> 8) & 255) + ((cw >> 16) & 255);
        const int pe = We - ne, pl = (W - We) - nlp;
        const int64_t b0 = Xrowptr[s];
        int32_t *cp = col + S.kc[sl] + slot;
        for (int k = 0; k < We; ++k) cp[(int64_t)k * ng] = (k < pe) ? -1 : qcol[b0 + k - pe];
        for (int k = 0; k < W - We; ++k) cp[(int64_t)(We + k) * ng] = (k < pl) ? -1 : qcol[b0 + ne + k - pl];
    }
}

// group index of every group's first row (only first rows are written)
__global__ void k_group_index(int32_t ngroups, const int32_t *grp, int32_t *gid)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
        gid[grp[g]] = (int32_t)g;
}

// sort keys of the groups: level of the first row (forward) and last row (backward)
__global__ void k_group_keys(int32_t ngroups, const int32_t *grp, const int32_t *level, int32_t *kf, int32_t *kb)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        kf[g] = level[grp[g]];
        kb[g] = level[grp[g + 1] - 1];
    }
}

static unsigned grid_for(gic_handle *h, int64_t items)
{
    int64_t b = (items + 255) / 256, cap = (int64_t)h->num_sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

void free_ssched(SliceSched &S)
{
    cudaFree(S.w);
    cudaFree(S.we);
    cudaFree(S.ng);
    cudaFree(S.kv);
    cudaFree(S.kc);
    cudaFree(S.lane);
    cudaFree(S.col);
    S = SliceSched();
}

// Host part of one sweep's schedule: order the groups by key (ascending;
// the backward keys arrive negated), then by external column count
// (descending, so that slices of equal width form) and by index in the
// sweep's direction (ascending forward, descending backward: a level's
// slices are then taken in the order in which the level before them
// finishes); cut slices.
static int plan_slices(gic_handle *h, int32_t ngroups, const std::vector<int32_t> &grp, const std::vector<int32_t> &key,
                       const std::vector<int32_t> &cnt, bool forward, SliceSched &S)
{
    auto early = [&](int32_t g) { return cnt[g] & 255; };
    auto late = [&](int32_t g) { return ((cnt[g] >> 8) & 255) + ((cnt[g] >> 16) & 255); };
    int32_t kmin = 0, kmax = 0;
    for (int32_t g = 0; g < ngroups; ++g) {
        if (g == 0 || key[g] < kmin) kmin = key[g];
        if (g == 0 || key[g] > kmax) kmax = key[g];
    }
    // two stable counting sorts (by descending width, then by key) of the
    // groups visited in index order in the sweep's direction: sorted by key,
    // then width, then that index order
    constexpr int WMAX = 2 * QCOL; // early + late widths are each < QCOL
    const int64_t nk = (int64_t)kmax - kmin + 1;
    std::vector<int32_t> byw(ngroups), order(ngroups);
    {
        std::vector<int64_t> c(WMAX + 1, 0);
        for (int32_t g = 0; g < ngroups; ++g) ++c[WMAX - (early(g) + late(g))];
        for (int k = 0; k < WMAX; ++k) c[k + 1] += c[k];
        for (int32_t q = 0; q < ngroups; ++q) {
            const int32_t g = forward ? q : ngroups - 1 - q;
            byw[c[WMAX - 1 - (early(g) + late(g))]++] = g;
        }
    }
    std::vector<int64_t> start(nk + 1, 0);
    for (int32_t g = 0; g < ngroups; ++g) ++start[key[g] - kmin + 1];
    for (int64_t k = 0; k < nk; ++k) start[k + 1] += start[k];
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int32_t q = 0; q < ngroups; ++q) order[fill[key[byw[q]] - kmin]++] = byw[q];
    }
    std::vector<int32_t> w, we, ng;
    std::vector<int64_t> kv, kc;
    std::vector<int2> lane;
    int64_t steps = 0, ncol = 0;
    for (int64_t k = 0; k < nk; ++k) {
        int64_t p = start[k];
        while (p < start[k + 1]) {
            int rows = 0, groups = 0, E = 0, Lt = 0;
            const size_t l0 = lane.size();
            lane.resize(l0 + 32, make_int2(-1, 0));
            while (p < start[k + 1] && groups < 32) {
                const int32_t g = order[p];
                const int G = grp[g + 1] - grp[g];
                if (rows + G > 32) break;
                for (int t = 0; t < G; ++t)
                    lane[l0 + rows + t] = make_int2(grp[g] + t, groups | (t << 8) | (G << 16) | (early(g) << 24));
                rows += G;
                E = std::max(E, early(g));
                Lt = std::max(Lt, late(g));
                ++groups;
                ++p;
            }
            if (Lt > SLATE) return GIC_ERR_UNSUPPORTED; // the kernel holds at most SLATE late steps
            w.push_back(E + Lt);
            we.push_back(E);
            ng.push_back(groups);
            kv.push_back(steps);
            kc.push_back(ncol);
            steps += E + Lt;
            ncol += (int64_t)(E + Lt) * groups;
        }
    }
    S.nsl = (int32_t)w.size();
    S.steps = steps;
    S.ncol = ncol;
    const size_t ns = (size_t)S.nsl;
    GIC_CUDA_TRY(cudaMalloc(&S.w, 4 * ns));
    GIC_CUDA_TRY(cudaMalloc(&S.we, 4 * ns));
    GIC_CUDA_TRY(cudaMalloc(&S.ng, 4 * ns));
    GIC_CUDA_TRY(cudaMalloc(&S.kv, 8 * ns));
    GIC_CUDA_TRY(cudaMalloc(&S.kc, 8 * ns));
    GIC_CUDA_TRY(cudaMalloc(&S.lane, sizeof(int2) * 32 * ns));
    GIC_CUDA_TRY(cudaMalloc(&S.col, 4 * (size_t)(ncol > 0 ? ncol : 1)));
    GIC_CUDA_TRY(cudaMemcpyAsync(S.w, w.data(), 4 * ns, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(S.we, we.data(), 4 * ns, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(S.ng, ng.data(), 4 * ns, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(S.kv, kv.data(), 8 * ns, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(S.kc, kc.data(), 8 * ns, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(S.lane, lane.data(), sizeof(int2) * 32 * ns, cudaMemcpyHostToDevice, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream)); // the host vectors go out of scope
    return GIC_OK;
}

static int build_ssched_impl(gic_handle *h, Pattern &P, int32_t *tmp)
{
    const int32_t ng = P.ngroups;
    int32_t *kf = tmp, *kb = tmp + ng, *gid = tmp + 2 * (size_t)ng;
    ++h->launches;
    k_group_keys<<<grid_for(h, ng), 256, 0, h->stream>>>(ng, P.grp, P.level, kf, kb);
    ++h->launches;
    k_group_index<<<grid_for(h, ng), 256, 0, h->stream>>>(ng, P.grp, gid);
    GIC_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hgrp(ng + 1), hkf(ng), hkb(ng), hcf(ng), hcb(ng);
    GIC_CUDA_TRY(cudaMemcpyAsync(hgrp.data(), P.grp, 4 * (size_t)(ng + 1), cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(hkf.data(), kf, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(hkb.data(), kb, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(hcf.data(), P.qf_cnt, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(hcb.data(), P.qb_cnt, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int32_t g = 0; g < ng; ++g) hkb[g] = -hkb[g]; // backward: descending level
    GIC_TRY(plan_slices(h, ng, hgrp, hkf, hcf, true, P.sf));
    GIC_TRY(plan_slices(h, ng, hgrp, hkb, hcb, false, P.sb));
    ++h->launches;
    k_scols<<<grid_for(h, (int64_t)P.sf.nsl * 32), 256, 0, h->stream>>>(view_of(P.sf), P.Lrowptr, P.qf_col, P.qf_cnt,
                                                                        gid, P.sf.col);
    ++h->launches;
    k_scols<<<grid_for(h, (int64_t)P.sb.nsl * 32), 256, 0, h->stream>>>(view_of(P.sb), P.Urowptr, P.qb_col, P.qb_cnt,
                                                                        gid, P.sb.col);
    GIC_CUDA_TRY(cudaGetLastError());
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return GIC_OK;
}

int build_ssched(gic_handle *h, Pattern &P)
{
    P.sready = 0;
    if (!P.qready || P.ngroups == 0) return GIC_OK;
    int32_t *tmp = nullptr;
    GIC_CUDA_TRY(cudaMalloc(&tmp, 4 * (2 * (size_t)P.ngroups + (size_t)P.n)));
    int rc = build_ssched_impl(h, P, tmp);
    cudaFree(tmp);
    if (rc != GIC_OK) {
        free_ssched(P.sf);
        free_ssched(P.sb);
        return rc == GIC_ERR_UNSUPPORTED ? GIC_OK : rc; // the pattern runs the other solves
    }
    P.sready = 1;
    return GIC_OK;
}

size_t s_values_bytes(const SliceSched &S, size_t es)
{
    return es * (32 * (size_t)S.steps + 96 * (size_t)S.nsl);
}

int s_setup(gic_handle *h, const Pattern &P, bool f32, const void *Lval, void *Sf, void *Sb)
{
    if (!P.sready) return GIC_ERR_UNSUPPORTED;
    const size_t es = f32 ? 4 : 8;
    char *mf = (char *)Sf + es * 32 * (size_t)P.sf.steps, *mb = (char *)Sb + es * 32 * (size_t)P.sb.steps;
    const unsigned gf = grid_for(h, (int64_t)P.sf.nsl * 32), gb = grid_for(h, (int64_t)P.sb.nsl * 32);
    h->launches += 2;
    if (f32) {
        k_ssetup<float, true><<<gf, 256, 0, h->stream>>>(view_of(P.sf), P.Lrowptr, P.Urowptr, P.tperm, P.qf_pos,
                                                         (const float *)Lval, (float *)Sf, (float *)mf);
        k_ssetup<float, false><<<gb, 256, 0, h->stream>>>(view_of(P.sb), P.Lrowptr, P.Urowptr, P.tperm, P.qb_pos,
                                                          (const float *)Lval, (float *)Sb, (float *)mb);
    } else {
        k_ssetup<double, true><<<gf, 256, 0, h->stream>>>(view_of(P.sf), P.Lrowptr, P.Urowptr, P.tperm, P.qf_pos,
                                                          (const double *)Lval, (double *)Sf, (double *)mf);
        k_ssetup<double, false><<<gb, 256, 0, h->stream>>>(view_of(P.sb), P.Lrowptr, P.Urowptr, P.tperm, P.qb_pos,
                                                           (const double *)Lval, (double *)Sb, (double *)mb);
    }
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

template <typename T, bool FWD, bool PCG>
static int s_launch(gic_handle *h, const Pattern &P, const void *vals, const T *rhs, T *x, T *yreset,
                    const double *rd, double *partials, Scalars *sc)
{
    if (!P.sready) return GIC_ERR_UNSUPPORTED;
    const SliceSched &SS = FWD ? P.sf : P.sb;
    SliceView S = view_of(SS);
    const T *kval = (const T *)vals;
    const T *mval = kval + 32 * (size_t)SS.steps;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&S, &kval, &mval, &rhs, &x, &yreset, &rd, &partials, &er, &poll, &sc};
    // warps: every slice could run at once, but waiting warps take issue
    // slots from working ones, so residency is capped per SM (tunable)
    int64_t need = SS.nsl;
    int per_sm = h->tune_solve_warps_per_sm;
    if (per_sm <= 0) per_sm = 32;
    if (need > (int64_t)per_sm * h->num_sms) need = (int64_t)per_sm * h->num_sms;
    if (PCG && need > MAX_PARTIALS) need = MAX_PARTIALS; // grid warps <= partial slots
    return launch_persistent(h, (const void *)k_ssolve<T, FWD, PCG>, SBLOCK, 0, need, args);
}

int s_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Sf, const void *r, void *y, const Scalars *sc)
{
    Scalars *s = const_cast<Scalars *>(sc);
    if (f32)
        return s_launch<float, true, false>(h, P, Sf, (const float *)r, (float *)y, nullptr, nullptr, nullptr, s);
    return s_launch<double, true, false>(h, P, Sf, (const double *)r, (double *)y, nullptr, nullptr, nullptr, s);
}

int s_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Sb, void *y, void *z,
              const double *rd, double *partials, Scalars *sc)
{
    if (f32) {
        if (pcg)
            return s_launch<float, false, true>(h, P, Sb, (const float *)y, (float *)z, (float *)y, rd, partials, sc);
        return s_launch<float, false, false>(h, P, Sb, (const float *)y, (float *)z, nullptr, nullptr, nullptr, sc);
    }
    if (pcg)
        return s_launch<double, false, true>(h, P, Sb, (const double *)y, (double *)z, (double *)y, rd, partials, sc);
    return s_launch<double, false, false>(h, P, Sb, (const double *)y, (double *)z, nullptr, nullptr, nullptr, sc);
}

}  // namespace gic
