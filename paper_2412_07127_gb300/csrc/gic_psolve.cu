// gic_psolve.cu -- A7c: pair-sliced sync-free triangular solves: the
// level-sliced solves (gic_ssolve.cu) with the number of dependency hops
// halved, for patterns of row groups of at most 3 rows.
//
// Every group is solved in the premultiplied form (Eq. (11) read as forward
// substitution, M = D^-1 of the group's diagonal block):
//     forward   y_g = M_g r_g + sum_j K_g(:, j) y_j,     K_g = -M_g L_ext(g)
// (backward: the same with U and M^T, over z and rhs y). A sweep that takes
// the groups level by level pays one cross-SM hand-off (a store, seen by a
// poll on another SM) per level; on this GPU that hand-off, not the
// arithmetic, sets the time of large sweeps. Here the group levels are taken
// two at a time (a "pair"): a group at the second level of a pair reads rows
// of groups at the first level of the same pair, and those reads are
// substituted by the rows' own formulas,
//     y_e = M_e r_e + sum_k K_e(:, k) y_k        for every such group e,
// which is exact algebra; the substituted group then reads only rows of
// earlier pairs, its column list is the union of its other columns and the
// columns of the groups e, and its right-hand side gains the rows of e:
//     y_g = M_g r_g + sum_e (K_g(:, e) M_e) r_e
//           + sum_{j not in e} K_g(:, j) y_j + sum_e K_g(:, e) K_e y.
// Both levels of a pair then depend only on earlier pairs, so one hand-off
// serves two levels. The price is arithmetic and bytes: for hex elasticity
// a second-level group reads 32 nodes (96 columns) instead of 13.
//
// Lanes: two per row (lane 2i + h: row i of the slice, half h), each half
// taking every other column of each part of the group's list, summed across
// the pair of lanes at the end. That halves the per-lane registers the
// longer lists need and the FP64 instructions between a slice's last
// dependency landing and its store (this GPU's FP64 warp instructions
// occupy the pipe for ~17 cycles however few lanes are active).
//
// A group's column list is kept in three parts: early (every column of a
// level older than the far level, ordered so the most recent come last),
// far (the first level of the previous pair's pair of levels to finish) and
// near (the last one): forward, pair p holds levels 2p and 2p + 1 and the
// previous pair's second level 2p - 1 finishes last (its groups carry the
// substitution), so near = level 2p - 1 and far = level 2p - 2; backward,
// pairs run in descending order, the substituted groups are the even
// levels, near = 2p + 2 and far = 2p + 3.
#include <algorithm>
#include <vector>

#include "gic_internal.cuh"
#include "gic_solve.cuh"

namespace gic {

constexpr int PBLOCK = 128;  // threads per block of the pair-sliced solves (4 blocks of 4 warps per SM)
constexpr int PBATCH = 10;   // early steps per lane whose loads are in flight together
constexpr int PFAR = 10;     // far steps per lane, loaded at once
constexpr int PNEAR = 9;     // near steps per lane, loaded at once, summed last
constexpr int PRHS = 6;      // right-hand-side steps per lane
constexpr int PEMAX = 3;     // substituted groups per group
constexpr int PRECENT = 2;   // levels before the far one kept at the end of the early part

struct PairView {
    int32_t nsl;
    const int32_t *w, *we, *wf, *wr, *ng;
    const int64_t *kv, *kc, *kr, *krc;
    const int2 *lane;
    const int32_t *col, *rcol;
};

static PairView pview_of(const PairSched &S)
{
    return PairView{S.nsl, S.w, S.we, S.wf, S.wr, S.ng, S.kv, S.kc, S.kr, S.krc, S.lane, S.col, S.rcol};
}

// ------------------------------------------------------------ analysis
// A group's dependency list: forward the external lower columns of its
// first row, backward the external upper columns of its last row (both
// ascending; the group's rows share them).
template <bool FWD>
__device__ __forceinline__ void dep_list(int32_t s, int32_t e, const int32_t *Lrowptr, const int32_t *Lcol,
                                         const int32_t *Urowptr, const int32_t *Ucol, const int32_t *&d, int &m)
{
    if (FWD) {
        d = Lcol + Lrowptr[s];
        m = Lrowptr[s + 1] - Lrowptr[s] - 1;
    } else {
        d = Ucol + Urowptr[e] + 1;
        m = Urowptr[e + 1] - Urowptr[e] - 1;
    }
}

// Classes of a column of group g's composite list, by the column's group
// level: 0 old early, 1 recent early, 2 far, 3 near; 4 = not in an earlier
// pair (the schedule would be invalid).
template <bool FWD>
__device__ __forceinline__ int col_class(int32_t lv, int32_t nl)
{
    const int32_t d = FWD ? nl - lv : lv - nl; // 0 near, 1 far, 2.. older
    if (d < 0) return 4;
    if (d == 0) return 3;
    if (d == 1) return 2;
    return d <= 1 + PRECENT ? 1 : 0;
}

// One thread per group. PASS 0 counts the group's composite columns per
// class and its right-hand-side rows: cnt[g] = n_old | n_recent << 8 |
// n_far << 16 | n_near << 24, rcnt[g] = rows; errors (more than PEMAX
// substituted groups: bit 0; a column outside the earlier pairs: 1; far,
// near, right-hand-side or early lists too long for the kernel: 2-5) are
// or-ed into *flag. PASS 1 writes the list at
// off[g] (old, recent, far, near; ascending within each) and the
// right-hand-side rows at roff[g] (the group's own rows, then each
// substituted group's rows). Lists are merged from the group's own
// dependencies (without the substituted rows) and those of the substituted
// groups, ascending, without repeats.
template <bool FWD, int PASS>
__global__ void k_pcomp(int64_t n, int32_t ngroups, int paired, const int32_t *__restrict__ grp, const int32_t *__restrict__ rowgrp,
                        const int32_t *__restrict__ glev, const int32_t *__restrict__ Lrowptr,
                        const int32_t *__restrict__ Lcol, const int32_t *__restrict__ Urowptr,
                        const int32_t *__restrict__ Ucol, int32_t *cnt, int32_t *rcnt, const int64_t *off,
                        const int64_t *roff, int32_t *list, int32_t *rlist, unsigned *flag)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = grp[g], e = grp[g + 1] - 1, G = e - s + 1;
        const int32_t L = glev[s];
        // the pair's near level and whether this group is substituted
        int32_t nl;
        bool sub;
        if (paired) {
            const int32_t p = L >> 1;
            nl = FWD ? 2 * p - 1 : 2 * p + 2;
            sub = FWD ? (L & 1) != 0 : (L & 1) == 0;
        } else {
            nl = FWD ? L - 1 : L + 1;
            sub = false;
        }
        const int32_t sl = FWD ? L - 1 : L + 1; // level of the substituted groups
        const int32_t *d0;
        int m0;
        dep_list<FWD>(s, e, Lrowptr, Lcol, Urowptr, Ucol, d0, m0);
        // substituted groups: the groups of the columns at level sl
        const int32_t *dl[1 + PEMAX];
        int ml[1 + PEMAX], pos[1 + PEMAX];
        int32_t es[PEMAX], eG[PEMAX];
        int ne = 0;
        unsigned bad = 0;
        dl[0] = d0;
        ml[0] = m0;
        if (sub) {
            for (int k = 0; k < m0; ++k) {
                const int32_t j = d0[k];
                if (glev[j] != sl) continue;
                const int32_t f = rowgrp[j];
                if (ne > 0 && es[ne - 1] == f) continue;
                if (ne == PEMAX) { bad |= 1u; break; }
                es[ne++] = f;
            }
        }
        for (int q = 0; q < ne; ++q) {
            const int32_t f = es[q];
            int32_t l = f;
            while (l + 1 < n && rowgrp[l + 1] == f) ++l;
            eG[q] = l - f + 1;
            dep_list<FWD>(f, l, Lrowptr, Lcol, Urowptr, Ucol, dl[1 + q], ml[1 + q]);
        }
        const int nlists = 1 + ne;
        for (int q = 0; q < nlists; ++q) pos[q] = 0;
        // merge: classes counted (PASS 0) or written (PASS 1)
        int c[4] = {0, 0, 0, 0};
        int64_t base[4] = {0, 0, 0, 0};
        if (PASS == 1) {
            const int32_t k = cnt[g];
            base[0] = off[g];
            base[1] = base[0] + (k & 255);
            base[2] = base[1] + ((k >> 8) & 255);
            base[3] = base[2] + ((k >> 16) & 255);
        }
        int32_t last = -1;
        while (!bad) {
            int32_t best = 0x7fffffff;
            int bq = -1;
            for (int q = 0; q < nlists; ++q) {
                // the own list skips the substituted rows
                while (q == 0 && sub && pos[0] < ml[0] && glev[dl[0][pos[0]]] == sl) ++pos[0];
                if (pos[q] < ml[q] && dl[q][pos[q]] < best) { best = dl[q][pos[q]]; bq = q; }
            }
            if (bq < 0) break;
            ++pos[bq];
            if (best == last) continue;
            last = best;
            const int cl = col_class<FWD>(glev[best], nl);
            if (cl == 4) { bad |= 2u; break; }
            if (PASS == 1) list[base[cl] + c[cl]] = best;
            ++c[cl];
        }
        // the old part holds the columns two or more levels before the far
        // one in ascending column order; "recent" (the PRECENT levels before
        // far) follow it, so an early batch that waits holds the latest ones
        int nR = G;
        for (int q = 0; q < ne; ++q) nR += eG[q];
        if ((c[2] + 1) / 2 > PFAR) bad |= 4u;
        if ((c[3] + 1) / 2 > PNEAR) bad |= 8u;
        if ((nR + 1) / 2 > PRHS) bad |= 16u;
        if (c[0] > 255 || c[1] > 255) bad |= 32u;
        if (bad) {
            if (PASS == 0) atomicOr(flag, bad);
            continue;
        }
        if (PASS == 0) {
            cnt[g] = c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24);
            rcnt[g] = nR;
        } else {
            int32_t *rp = rlist + roff[g];
            int k = 0;
            for (int u = 0; u < G; ++u) rp[k++] = s + u;
            for (int q = 0; q < ne; ++q)
                for (int u = 0; u < eG[q]; ++u) rp[k++] = es[q] + u;
        }
    }
}

__global__ void k_pgid(int32_t ngroups, const int32_t *grp, const int32_t *glev, int32_t *gid, int32_t *gl)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x) {
        gid[grp[g]] = (int32_t)g;
        gl[g] = glev[grp[g]];
    }
}

// Column words of the slices: the first lane of every group writes the
// group's list split between the two halves (entry i of a part goes to half
// i & 1), each part front-padded with -1 to the slice's width of that part
// (early, far, near), and its right-hand-side rows, padded at the end.
__global__ void k_pcols(PairView S, const int32_t *__restrict__ gid, const int32_t *__restrict__ cnt,
                        const int32_t *__restrict__ rcnt, const int64_t *__restrict__ off,
                        const int64_t *__restrict__ roff, const int32_t *__restrict__ list,
                        const int32_t *__restrict__ rlist, int32_t *col, int32_t *rcol)
{
    const int64_t total = (int64_t)S.nsl * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 d = S.lane[i];
        if (d.x < 0 || (d.y & 0x0100ff00) != 0) continue; // first row, half 0 only
        const int64_t sl = i >> 5;
        const int ng = S.ng[sl], slot = d.y & 255;
        const int W = S.w[sl], We = S.we[sl], Wf = S.wf[sl], Wn = W - We - Wf, Wr = S.wr[sl];
        const int32_t g = gid[d.x];
        const int32_t k = cnt[g];
        const int ce = (k & 255) + ((k >> 8) & 255), cf = (k >> 16) & 255, cn = (k >> 24) & 255;
        const int32_t *src = list + off[g];
        int32_t *cp = col + S.kc[sl] + 2 * slot;
        const int parts[3][3] = {{0, We, ce}, {We, Wf, cf}, {We + Wf, Wn, cn}};
        int from = 0;
        for (int pt = 0; pt < 3; ++pt) {
            const int b = parts[pt][0], wp = parts[pt][1], c = parts[pt][2];
            for (int h = 0; h < 2; ++h) {
                const int ch = (c + 1 - h) / 2, pad = wp - ch;
                for (int q = 0; q < wp; ++q)
                    cp[(int64_t)(b + q) * 2 * ng + h] = (q < pad) ? -1 : src[from + 2 * (q - pad) + h];
            }
            from += c;
        }
        const int nr = rcnt[g];
        const int32_t *rs = rlist + roff[g];
        int32_t *rp = rcol + S.krc[sl] + 2 * slot;
        for (int q = 0; q < Wr; ++q)
            for (int h = 0; h < 2; ++h) rp[(int64_t)q * 2 * ng + h] = (2 * q + h < nr) ? rs[2 * q + h] : -1;
    }
}

static unsigned pgrid(gic_handle *h, int64_t items)
{
    int64_t b = (items + 255) / 256, cap = (int64_t)h->num_sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

void free_psched(PairSched &S)
{
    cudaFree(S.w);
    cudaFree(S.we);
    cudaFree(S.wf);
    cudaFree(S.wr);
    cudaFree(S.ng);
    cudaFree(S.kv);
    cudaFree(S.kc);
    cudaFree(S.kr);
    cudaFree(S.krc);
    cudaFree(S.lane);
    cudaFree(S.col);
    cudaFree(S.rcol);
    S = PairSched();
}

template <typename T>
static int to_device(gic_handle *h, T **d, const std::vector<T> &v)
{
    GIC_CUDA_TRY(cudaMalloc(d, sizeof(T) * (v.empty() ? 1 : v.size())));
    if (!v.empty())
        GIC_CUDA_TRY(cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->stream));
    return GIC_OK;
}

// Host part of one sweep's schedule: order the groups by pair (forward
// ascending, backward descending), then by width (descending, so slices of
// equal width form) and by index in the sweep's direction; cut slices of
// whole groups with at most 16 rows inside one pair.
static int plan_pslices(gic_handle *h, int32_t ngroups, bool forward, int paired, const std::vector<int32_t> &grp,
                        const std::vector<int32_t> &gl, const std::vector<int32_t> &cnt,
                        const std::vector<int32_t> &rcnt, PairSched &S)
{
    auto we_of = [&](int32_t g) { return ((cnt[g] & 255) + ((cnt[g] >> 8) & 255) + 1) / 2; };
    auto wf_of = [&](int32_t g) { return (((cnt[g] >> 16) & 255) + 1) / 2; };
    auto wn_of = [&](int32_t g) { return (((cnt[g] >> 24) & 255) + 1) / 2; };
    auto key_of = [&](int32_t g) { const int32_t p = paired ? gl[g] >> 1 : gl[g]; return forward ? p : -p; };
    int32_t kmin = 0, kmax = 0;
    int wmax = 0;
    for (int32_t g = 0; g < ngroups; ++g) {
        const int32_t k = key_of(g);
        if (g == 0 || k < kmin) kmin = k;
        if (g == 0 || k > kmax) kmax = k;
        wmax = std::max(wmax, we_of(g) + wf_of(g) + wn_of(g));
    }
    const int64_t nk = (int64_t)kmax - kmin + 1;
    std::vector<int32_t> byw(ngroups), order(ngroups);
    {
        std::vector<int64_t> c(wmax + 2, 0);
        for (int32_t g = 0; g < ngroups; ++g) ++c[wmax - (we_of(g) + wf_of(g) + wn_of(g)) + 1];
        for (int k = 0; k <= wmax; ++k) c[k + 1] += c[k];
        for (int32_t q = 0; q < ngroups; ++q) {
            const int32_t g = forward ? q : ngroups - 1 - q;
            byw[c[wmax - (we_of(g) + wf_of(g) + wn_of(g))]++] = g;
        }
    }
    std::vector<int64_t> start(nk + 1, 0);
    for (int32_t g = 0; g < ngroups; ++g) ++start[key_of(g) - kmin + 1];
    for (int64_t k = 0; k < nk; ++k) start[k + 1] += start[k];
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int32_t q = 0; q < ngroups; ++q) order[fill[key_of(byw[q]) - kmin]++] = byw[q];
    }
    std::vector<int32_t> w, we, wf, wr, ng;
    std::vector<int64_t> kv, kc, kr, krc;
    std::vector<int2> lane;
    int64_t steps = 0, ncol = 0, rsteps = 0, nrcol = 0;
    for (int64_t k = 0; k < nk; ++k) {
        int64_t p = start[k];
        while (p < start[k + 1]) {
            int rows = 0, groups = 0, E = 0, F = 0, Nn = 0, R = 0;
            const size_t l0 = lane.size();
            lane.resize(l0 + 32, make_int2(-1, 0));
            while (p < start[k + 1] && groups < 16) {
                const int32_t g = order[p];
                const int G = grp[g + 1] - grp[g];
                if (rows + G > 16) break;
                for (int t = 0; t < G; ++t)
                    for (int hh = 0; hh < 2; ++hh)
                        lane[l0 + 2 * (rows + t) + hh] = make_int2(grp[g] + t, groups | (t << 8) | (G << 16) | (hh << 24));
                rows += G;
                E = std::max(E, we_of(g));
                F = std::max(F, wf_of(g));
                Nn = std::max(Nn, wn_of(g));
                R = std::max(R, (rcnt[g] + 1) / 2);
                ++groups;
                ++p;
            }
            if (groups == 0) return GIC_ERR_UNSUPPORTED; // cannot happen: groups have at most 3 rows
            w.push_back(E + F + Nn);
            we.push_back(E);
            wf.push_back(F);
            wr.push_back(R);
            ng.push_back(groups);
            kv.push_back(steps);
            kc.push_back(ncol);
            kr.push_back(rsteps);
            krc.push_back(nrcol);
            steps += E + F + Nn;
            ncol += (int64_t)(E + F + Nn) * groups * 2;
            rsteps += R;
            nrcol += (int64_t)R * groups * 2;
        }
    }
    S.nsl = (int32_t)w.size();
    S.steps = steps;
    S.ncol = ncol;
    S.rsteps = rsteps;
    S.nrcol = nrcol;
    GIC_TRY(to_device(h, &S.w, w));
    GIC_TRY(to_device(h, &S.we, we));
    GIC_TRY(to_device(h, &S.wf, wf));
    GIC_TRY(to_device(h, &S.wr, wr));
    GIC_TRY(to_device(h, &S.ng, ng));
    GIC_TRY(to_device(h, &S.kv, kv));
    GIC_TRY(to_device(h, &S.kc, kc));
    GIC_TRY(to_device(h, &S.kr, kr));
    GIC_TRY(to_device(h, &S.krc, krc));
    GIC_TRY(to_device(h, &S.lane, lane));
    GIC_CUDA_TRY(cudaMalloc(&S.col, 4 * (size_t)(ncol > 0 ? ncol : 1)));
    GIC_CUDA_TRY(cudaMalloc(&S.rcol, 4 * (size_t)(nrcol > 0 ? nrcol : 1)));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream)); // the host vectors go out of scope
    return GIC_OK;
}

// One sweep: composite lists (two passes), plan, column words.
template <bool FWD>
static int build_pdir(gic_handle *h, Pattern &P, int paired, const std::vector<int32_t> &hgrp,
                      const std::vector<int32_t> &hgl, const int32_t *gid, int32_t *dcnt, int32_t *drcnt,
                      unsigned *dflag, PairSched &S)
{
    const int32_t ng = P.ngroups;
    const unsigned gr = pgrid(h, ng);
    int64_t *doff = nullptr, *droff = nullptr;
    int32_t *list = nullptr, *rlist = nullptr;
    // the body returns early on any error; the temporaries are freed after it
    const int rc = [&]() -> int {
        GIC_CUDA_TRY(cudaMemsetAsync(dflag, 0, sizeof(unsigned), h->stream));
        ++h->launches;
        k_pcomp<FWD, 0><<<gr, 256, 0, h->stream>>>(P.n, ng, paired, P.grp, P.rowgrp, P.glev, P.Lrowptr, P.Lcol,
                                                   P.Urowptr, P.Ucol, dcnt, drcnt, nullptr, nullptr, nullptr,
                                                   nullptr, dflag);
        GIC_CUDA_TRY(cudaGetLastError());
        std::vector<int32_t> cnt(ng), rcnt(ng);
        unsigned flag = 0;
        GIC_CUDA_TRY(cudaMemcpyAsync(cnt.data(), dcnt, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
        GIC_CUDA_TRY(cudaMemcpyAsync(rcnt.data(), drcnt, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
        GIC_CUDA_TRY(cudaMemcpyAsync(&flag, dflag, sizeof flag, cudaMemcpyDeviceToHost, h->stream));
        GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
        if (flag) {
            P.pwhy |= (int)flag;
            return GIC_ERR_UNSUPPORTED;
        }
        std::vector<int64_t> off(ng), roff(ng);
        int64_t tot = 0, rtot = 0;
        for (int32_t g = 0; g < ng; ++g) {
            const int32_t k = cnt[g];
            off[g] = tot;
            roff[g] = rtot;
            tot += (k & 255) + ((k >> 8) & 255) + ((k >> 16) & 255) + ((k >> 24) & 255);
            rtot += rcnt[g];
        }
        GIC_TRY(to_device(h, &doff, off));
        GIC_TRY(to_device(h, &droff, roff));
        GIC_CUDA_TRY(cudaMalloc(&list, 4 * (size_t)(tot > 0 ? tot : 1)));
        GIC_CUDA_TRY(cudaMalloc(&rlist, 4 * (size_t)(rtot > 0 ? rtot : 1)));
        ++h->launches;
        k_pcomp<FWD, 1><<<gr, 256, 0, h->stream>>>(P.n, ng, paired, P.grp, P.rowgrp, P.glev, P.Lrowptr, P.Lcol,
                                                   P.Urowptr, P.Ucol, dcnt, drcnt, doff, droff, list, rlist,
                                                   dflag);
        GIC_CUDA_TRY(cudaGetLastError());
        GIC_TRY(plan_pslices(h, ng, FWD, paired, hgrp, hgl, cnt, rcnt, S));
        ++h->launches;
        k_pcols<<<pgrid(h, (int64_t)S.nsl * 32), 256, 0, h->stream>>>(pview_of(S), gid, dcnt, drcnt, doff, droff, list,
                                                                      rlist, S.col, S.rcol);
        GIC_CUDA_TRY(cudaGetLastError());
        GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
        return GIC_OK;
    }();
    cudaFree(doff);
    cudaFree(droff);
    cudaFree(list);
    cudaFree(rlist);
    return rc;
}

static int build_psched_impl(gic_handle *h, Pattern &P, int paired, int32_t *tmp)
{
    const int32_t ng = P.ngroups;
    int32_t *gid = tmp, *gl = tmp + P.n, *dcnt = gl + ng, *drcnt = dcnt + ng;
    unsigned *dflag = (unsigned *)(drcnt + ng);
    ++h->launches;
    k_pgid<<<pgrid(h, ng), 256, 0, h->stream>>>(ng, P.grp, P.glev, gid, gl);
    GIC_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hgrp(ng + 1), hgl(ng);
    GIC_CUDA_TRY(cudaMemcpyAsync(hgrp.data(), P.grp, 4 * (size_t)(ng + 1), cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaMemcpyAsync(hgl.data(), gl, 4 * (size_t)ng, cudaMemcpyDeviceToHost, h->stream));
    GIC_CUDA_TRY(cudaStreamSynchronize(h->stream));
    GIC_TRY(build_pdir<true>(h, P, paired, hgrp, hgl, gid, dcnt, drcnt, dflag, P.pf));
    GIC_TRY(build_pdir<false>(h, P, paired, hgrp, hgl, gid, dcnt, drcnt, dflag, P.pb));
    return GIC_OK;
}

int build_psched(gic_handle *h, Pattern &P)
{
    P.pready = 0;
    P.pwhy = 0;
    if (P.max_group > 3) P.pwhy = 128;
    if (P.ngroups == 0 || P.max_group > 3 || !P.glev) return GIC_OK;
    // built when asked for, or when the automatic choice would take it
    const int64_t c = P.nchunks, sms = h->num_sms;
    const bool autosel = (h->tune_pipeline == 4 || h->tune_pipeline > 5) && c >= (int64_t)SLICED_CHUNKS_PER_SM * sms &&
                         c < (int64_t)PAIRED_CHUNKS_PER_SM * sms;
    if (h->tune_pipeline != 5 && !autosel) {
        P.pwhy = 256;
        return GIC_OK;
    }
    int32_t *tmp = nullptr;
    GIC_CUDA_TRY(cudaMalloc(&tmp, 4 * ((size_t)P.n + 3 * (size_t)P.ngroups + 1)));
    const int paired = h->tune_pair_levels == 0 ? 1 : 0;
    int rc = build_psched_impl(h, P, paired, tmp);
    cudaFree(tmp);
    if (rc != GIC_OK) {
        free_psched(P.pf);
        free_psched(P.pb);
        return rc == GIC_ERR_UNSUPPORTED ? GIC_OK : rc; // the pattern runs the other solves
    }
    P.pready = paired ? 1 : 2;
    return GIC_OK;
}

// ------------------------------------------------------------ coefficients
__device__ __forceinline__ int bsearch_col(const int32_t *d, int m, int32_t c)
{
    int lo = 0, hi = m - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = d[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// M = D^-1 of a group's lower diagonal block (rows s.., G <= 3; mL = the
// first row's external lower count)
template <typename TL>
__device__ __forceinline__ void group_inverse(int32_t s, int G, const int32_t *Lrowptr, const TL *Lval,
                                              double (&M)[3][3])
{
    const int32_t mL = Lrowptr[s + 1] - Lrowptr[s] - 1;
    double D[3][3] = {};
    for (int a = 0; a < 3; ++a)
        for (int u = 0; u < 3; ++u) M[a][u] = 0.0;
    for (int a = 0; a < G; ++a)
        for (int u = 0; u <= a; ++u) D[a][u] = (double)Lval[Lrowptr[s + a] + mL + u];
    for (int a = 0; a < G; ++a) {
        M[a][a] = 1.0 / D[a][a];
        for (int u = 0; u < a; ++u) {
            double acc = 0.0;
            for (int v = u; v < a; ++v) acc = fma(D[a][v], M[v][u], acc);
            M[a][u] = -acc * M[a][a];
        }
    }
}

// K_t(c) of a group (rows s.., G rows, dependency list d/m): forward
// -sum_{u<=t} M_tu L(s+u, c), backward -sum_{u>=t} M_ut U(s+u, c); 0 if c
// is not in the list
template <typename TL, bool FWD>
__device__ __forceinline__ double kappa(int32_t s, int G, int t, const double (&M)[3][3], const int32_t *d, int m,
                                        int32_t c, const int32_t *Lrowptr, const int32_t *Urowptr,
                                        const int32_t *tperm, const TL *Lval)
{
    const int p = bsearch_col(d, m, c);
    if (p < 0) return 0.0;
    double acc = 0.0;
    if (FWD) {
        for (int u = 0; u <= t; ++u) acc = fma(M[t][u], (double)Lval[Lrowptr[s + u] + p], acc);
    } else {
        for (int u = t; u < G; ++u) acc = fma(M[u][t], (double)Lval[tperm[Urowptr[s + u] + (G - u) + p]], acc);
    }
    return -acc;
}

// The coefficients of a factor in the pair-slice layout, one thread per lane,
// in FP64, stored in TL: for every column word of the lane's half the
// composite coefficient K_g(t, c) + sum_e sum_u K_g(t, e_u) K_e(u, c), for
// every right-hand-side row the own M_g entry or sum_u K_g(t, e_u) M_e(u, v)
// (forward; backward with M^T). Idle lanes and padding get 0.
template <typename TL, bool FWD>
__global__ void k_psetup(PairView S, const int32_t *__restrict__ Lrowptr, const int32_t *__restrict__ Lcol,
                         const int32_t *__restrict__ Urowptr, const int32_t *__restrict__ Ucol,
                         const int32_t *__restrict__ tperm, const int32_t *__restrict__ rowgrp,
                         const TL *__restrict__ Lval, TL *__restrict__ kval, TL *__restrict__ rkval)
{
    const int64_t total = (int64_t)S.nsl * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = i >> 5;
        const int l = (int)(i & 31);
        const int W = S.w[sl], Wr = S.wr[sl], ng = S.ng[sl];
        TL *kp = kval + S.kv[sl] * 32 + l;
        TL *rp = rkval + S.kr[sl] * 32 + l;
        const int2 d = S.lane[i];
        const int32_t row = d.x;
        if (row < 0) {
            for (int k = 0; k < W; ++k) kp[(int64_t)k * 32] = (TL)0;
            for (int k = 0; k < Wr; ++k) rp[(int64_t)k * 32] = (TL)0;
            continue;
        }
        const int slot = d.y & 255, t = (d.y >> 8) & 255, G = (d.y >> 16) & 255, h = (d.y >> 24) & 1;
        const int32_t s = row - t;
        double M[3][3];
        group_inverse<TL>(s, G, Lrowptr, Lval, M);
        const int32_t *dg;
        int mg;
        dep_list<FWD>(s, s + G - 1, Lrowptr, Lcol, Urowptr, Ucol, dg, mg);
        // substituted groups from the right-hand-side list (own rows first)
        const int32_t *rc = S.rcol + S.krc[sl] + 2 * slot;
        int ne = 0;
        int32_t sE[PEMAX] = {0, 0, 0};
        int GE[PEMAX] = {0, 0, 0};
        double a[PEMAX][3] = {};
        for (int q = G; q < 2 * Wr; ++q) {
            const int32_t r = rc[(int64_t)(q >> 1) * 2 * ng + (q & 1)];
            if (r < 0) break;
            const int32_t f = rowgrp[r];
            if (ne == 0 || sE[ne - 1] != f) {
                if (ne == PEMAX) break; // cannot happen: the analysis caps it
                sE[ne] = f;
                GE[ne] = 0;
                ++ne;
            }
            ++GE[ne - 1];
            a[ne - 1][r - f] = kappa<TL, FWD>(s, G, t, M, dg, mg, r, Lrowptr, Urowptr, tperm, Lval);
        }
        double ME[PEMAX][3][3];
        const int32_t *de[PEMAX];
        int me[PEMAX];
        for (int q = 0; q < ne; ++q) {
            group_inverse<TL>(sE[q], GE[q], Lrowptr, Lval, ME[q]);
            dep_list<FWD>(sE[q], sE[q] + GE[q] - 1, Lrowptr, Lcol, Urowptr, Ucol, de[q], me[q]);
        }
        const int32_t *cp = S.col + S.kc[sl] + 2 * slot + h;
        for (int k = 0; k < W; ++k) {
            const int32_t c = cp[(int64_t)k * 2 * ng];
            double v = 0.0;
            if (c >= 0) {
                v = kappa<TL, FWD>(s, G, t, M, dg, mg, c, Lrowptr, Urowptr, tperm, Lval);
                for (int q = 0; q < ne; ++q)
                    for (int u = 0; u < GE[q]; ++u)
                        if (a[q][u] != 0.0)
                            v = fma(a[q][u], kappa<TL, FWD>(sE[q], GE[q], u, ME[q], de[q], me[q], c, Lrowptr,
                                                             Urowptr, tperm, Lval), v);
            }
            kp[(int64_t)k * 32] = (TL)v;
        }
        for (int k = 0; k < Wr; ++k) {
            const int q2 = 2 * k + h;
            const int32_t r = rc[(int64_t)k * 2 * ng + h];
            double v = 0.0;
            if (r >= 0 && q2 < G) {
                const int u = r - s;
                v = FWD ? (u <= t ? M[t][u] : 0.0) : (u >= t ? M[u][t] : 0.0);
            } else if (r >= 0) {
                int q = 0;
                while (q + 1 < ne && sE[q] != rowgrp[r]) ++q;
                const int vv = r - sE[q];
                for (int u = 0; u < GE[q]; ++u)
                    if (FWD ? u >= vv : u <= vv) v = fma(a[q][u], FWD ? ME[q][u][vv] : ME[q][vv][u], v);
            }
            rp[(int64_t)k * 32] = (TL)v;
        }
    }
}

// ------------------------------------------------------------ solve
// FWD: L y = r (x = y, rhs = r). Backward: L^T z = y (x = z, rhs = y); with
// PCG it also forms r^T z in FP64 and beta = r_k^T z_k / r_{k-1}^T z_{k-1}
// (Algorithm 1) in the last warp to finish. x must hold the sentinel; the
// right-hand side is only read (a substituted group reads other groups'
// right-hand-side rows, so the PCG driver resets y elsewhere). kval:
// step-major coefficients, 32 per step; rkval: right-hand-side coefficients.
template <typename T, bool FWD, bool PCG>
__global__ void __launch_bounds__(PBLOCK, 4) k_psolve(PairView S, const T *__restrict__ kval,
                                                   const T *__restrict__ rkval, const T *rhs, T *x,
                                                   const double *__restrict__ rd, double *partials, unsigned *err,
                                                   int poll, Scalars *sc)
{
    if (sc && sc->done) return;
    constexpr int PLATE = PFAR + PNEAR;
    // each warp's far and near coefficients and column words, right-hand-side
    // coefficients and rows
    __shared__ __align__(16) T s_klate[PBLOCK / 32][PLATE * 32];
    __shared__ __align__(16) T s_rk[PBLOCK / 32][PRHS * 32];
    __shared__ __align__(16) int32_t s_lidx[PBLOCK / 32][PLATE * 32];
    __shared__ __align__(16) int32_t s_ridx[PBLOCK / 32][PRHS * 32];
    const int lane = threadIdx.x & 31;
    T *klate = s_klate[threadIdx.x >> 5], *rkw = s_rk[threadIdx.x >> 5];
    int32_t *lidx = s_lidx[threadIdx.x >> 5], *ridx = s_ridx[threadIdx.x >> 5];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned sleep_ns = (unsigned)(poll & 0xffff);
    double dot = 0.0;
    int64_t sl = gw;
    int hW = 0, hWe = 0, hWf = 0, hWr = 0, hng = 0;
    int64_t hkv = 0, hkc = 0, hkr = 0, hkrc = 0;
    int2 hd = make_int2(-1, 0);
    if (sl < S.nsl) {
        hW = S.w[sl], hWe = S.we[sl], hWf = S.wf[sl], hWr = S.wr[sl], hng = S.ng[sl];
        hkv = S.kv[sl], hkc = S.kc[sl], hkr = S.kr[sl], hkrc = S.krc[sl];
        hd = S.lane[sl * 32 + lane];
    }
    for (; sl < S.nsl; sl += nw) {
        const int W = hW, We = hWe, Wf = hWf, Wn = W - We - Wf, Wr = hWr, ng = hng;
        const int64_t kv0 = hkv, kc0 = hkc, kr0 = hkr, krc0 = hkrc;
        const int2 d = hd;
        const int32_t row = d.x;
        const int slot = d.y & 255, h = (d.y >> 24) & 1;
        const bool act = row >= 0;
        double rdv = 0.0;
        if (PCG && act && h == 0) rdv = rd[row];
        const int64_t sn = sl + nw;
        if (sn < S.nsl) {
            hW = S.w[sn], hWe = S.we[sn], hWf = S.wf[sn], hWr = S.wr[sn], hng = S.ng[sn];
            hkv = S.kv[sn], hkc = S.kc[sn], hkr = S.kr[sn], hkrc = S.krc[sn];
            hd = S.lane[sn * 32 + lane];
        }
        T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
        const int32_t *cp = S.col + kc0 + 2 * slot + h;
        const int64_t cs = 2 * (int64_t)ng; // column words per step
        const T *kp = kval + kv0 * 32 + lane;
        // the far and near coefficients and column words and the right-hand
        // side's coefficients and rows go to the warp's shared memory in one
        // asynchronous group, in flight with the first early batch's words
        {
            const int32_t *rcp = S.rcol + krc0 + 2 * slot + h;
            const T *rkp = rkval + kr0 * 32 + lane;
            for (int b = 0; b < W - We; ++b) {
                cp_async_t(&klate[b * 32 + lane], kp + (int64_t)(We + b) * 32);
                cp_async_t(&lidx[b * 32 + lane], cp + (int64_t)(We + b) * cs);
            }
            for (int b = 0; b < Wr; ++b) {
                cp_async_t(&rkw[b * 32 + lane], rkp + (int64_t)b * 32);
                cp_async_t(&ridx[b * 32 + lane], rcp + (int64_t)b * cs);
            }
            cp_async_commit();
        }
        int32_t c[PBATCH];
        T kv[PBATCH];
#pragma unroll
        for (int b = 0; b < PBATCH; ++b) {
            c[b] = (act && b < We) ? cp[(int64_t)b * cs] : -1;
            kv[b] = (b < We) ? kp[(int64_t)b * 32] : (T)0;
        }
        cp_async_wait<0>(); // this lane's copies are in shared memory
        // right-hand side (never waited on): the group's own rows and, for a
        // substituted group, the rows of the groups it substitutes; its values
        // are requested with the first early batch and summed after it
        T rv[PRHS];
#pragma unroll
        for (int b = 0; b < PRHS; ++b) {
            const int32_t r = (act && b < Wr) ? ridx[b * 32 + lane] : -1;
            rv[b] = (r >= 0) ? rhs[r] : (T)0;
        }
        // early section in batches (the next batch's columns and
        // coefficients loaded while one waits); the warp stays converged
        for (int k0 = 0; k0 < We; k0 += PBATCH) {
            T v[PBATCH];
#pragma unroll
            for (int b = 0; b < PBATCH; ++b) v[b] = (c[b] >= 0) ? ld_relaxed(x + c[b]) : (T)0;
            int32_t cn[PBATCH];
            T kn[PBATCH];
#pragma unroll
            for (int b = 0; b < PBATCH; ++b) {
                const int k = k0 + PBATCH + b;
                cn[b] = (act && k < We) ? cp[(int64_t)k * cs] : -1;
                kn[b] = (k < We) ? kp[(int64_t)k * 32] : (T)0;
            }
            slice_wait<T, PBATCH>(x, c, v, err, sleep_ns, lane);
            if (k0 == 0) {
#pragma unroll
                for (int b = 0; b < PRHS; ++b)
                    if (b < Wr) acc1 = fma(rkw[b * 32 + lane], rv[b], acc1);
            }
#pragma unroll
            for (int b = 0; b < PBATCH; ++b) {
                if (k0 + b < We) { // uniform over the warp
                    if (b & 1) acc1 = fma(kv[b], v[b], acc1);
                    else acc0 = fma(kv[b], v[b], acc0);
                }
            }
#pragma unroll
            for (int b = 0; b < PBATCH; ++b) {
                c[b] = cn[b];
                kv[b] = kn[b];
            }
        }
        if (We == 0) {
#pragma unroll
            for (int b = 0; b < PRHS; ++b)
                if (b < Wr) acc1 = fma(rkw[b * 32 + lane], rv[b], acc1);
        }
        // far and near waves: every value requested at once, the far ones
        // summed first; once the last near value lands a poll round and a few
        // FMAs remain
        {
            int32_t cf[PFAR], cq[PNEAR];
            T vf[PFAR], vq[PNEAR];
#pragma unroll
            for (int b = 0; b < PFAR; ++b) cf[b] = (act && b < Wf) ? lidx[b * 32 + lane] : -1;
#pragma unroll
            for (int b = 0; b < PNEAR; ++b) cq[b] = (act && b < Wn) ? lidx[(Wf + b) * 32 + lane] : -1;
#pragma unroll
            for (int b = 0; b < PFAR; ++b) vf[b] = (cf[b] >= 0) ? ld_relaxed(x + cf[b]) : (T)0;
#pragma unroll
            for (int b = 0; b < PNEAR; ++b) vq[b] = (cq[b] >= 0) ? ld_relaxed(x + cq[b]) : (T)0;
            slice_wait<T, PFAR>(x, cf, vf, err, sleep_ns, lane);
#pragma unroll
            for (int b = 0; b < PFAR; ++b) {
                if (b < Wf) { // uniform over the warp
                    const T kb = klate[b * 32 + lane];
                    if ((b & 3) == 0) acc0 = fma(kb, vf[b], acc0);
                    else if ((b & 3) == 1) acc1 = fma(kb, vf[b], acc1);
                    else if ((b & 3) == 2) acc2 = fma(kb, vf[b], acc2);
                    else acc3 = fma(kb, vf[b], acc3);
                }
            }
            slice_wait<T, PNEAR>(x, cq, vq, err, sleep_ns, lane);
#pragma unroll
            for (int b = 0; b < PNEAR; ++b) {
                if (b < Wn) {
                    const T kb = klate[(Wf + b) * 32 + lane];
                    if (b % 3 == 0) acc0 = fma(kb, vq[b], acc0);
                    else if (b % 3 == 1) acc2 = fma(kb, vq[b], acc2);
                    else acc3 = fma(kb, vq[b], acc3);
                }
            }
        }
        const T yh = (acc0 + acc1) + (acc2 + acc3);
        const T y = yh + __shfl_xor_sync(0xffffffffu, yh, 1); // the two halves of the row
        __syncwarp(); // every lane's shared-memory reads precede the next slice's copies
        if (act && h == 0) {
            st_relaxed(x + row, y);
            if (PCG) dot = fma(rdv, (double)y, dot);
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

// ------------------------------------------------------------ host
size_t p_values_bytes(const PairSched &S, size_t es)
{
    return es * 32 * ((size_t)S.steps + (size_t)S.rsteps);
}

int p_setup(gic_handle *h, const Pattern &P, bool f32, const void *Lval, void *Vf, void *Vb)
{
    if (!P.pready) return GIC_ERR_UNSUPPORTED;
    const size_t es = f32 ? 4 : 8;
    char *rf = (char *)Vf + es * 32 * (size_t)P.pf.steps, *rb = (char *)Vb + es * 32 * (size_t)P.pb.steps;
    const unsigned gf = pgrid(h, (int64_t)P.pf.nsl * 32), gb = pgrid(h, (int64_t)P.pb.nsl * 32);
    h->launches += 2;
    if (f32) {
        k_psetup<float, true><<<gf, 256, 0, h->stream>>>(pview_of(P.pf), P.Lrowptr, P.Lcol, P.Urowptr, P.Ucol, P.tperm,
                                                         P.rowgrp, (const float *)Lval, (float *)Vf, (float *)rf);
        k_psetup<float, false><<<gb, 256, 0, h->stream>>>(pview_of(P.pb), P.Lrowptr, P.Lcol, P.Urowptr, P.Ucol,
                                                          P.tperm, P.rowgrp, (const float *)Lval, (float *)Vb,
                                                          (float *)rb);
    } else {
        k_psetup<double, true><<<gf, 256, 0, h->stream>>>(pview_of(P.pf), P.Lrowptr, P.Lcol, P.Urowptr, P.Ucol,
                                                          P.tperm, P.rowgrp, (const double *)Lval, (double *)Vf,
                                                          (double *)rf);
        k_psetup<double, false><<<gb, 256, 0, h->stream>>>(pview_of(P.pb), P.Lrowptr, P.Lcol, P.Urowptr, P.Ucol,
                                                           P.tperm, P.rowgrp, (const double *)Lval, (double *)Vb,
                                                           (double *)rb);
    }
    GIC_CUDA_TRY(cudaGetLastError());
    return GIC_OK;
}

template <typename T, bool FWD, bool PCG>
static int p_launch(gic_handle *h, const Pattern &P, const void *vals, const T *rhs, T *x, const double *rd,
                    double *partials, Scalars *sc)
{
    if (!P.pready) return GIC_ERR_UNSUPPORTED;
    const PairSched &SS = FWD ? P.pf : P.pb;
    PairView S = pview_of(SS);
    const T *kval = (const T *)vals;
    const T *rkval = kval + 32 * (size_t)SS.steps;
    unsigned *er = h->dev_err;
    int poll = h->tune_poll;
    void *args[] = {&S, &kval, &rkval, &rhs, &x, &rd, &partials, &er, &poll, &sc};
    int64_t need = SS.nsl;
    int per_sm = h->tune_solve_warps_per_sm;
    if (per_sm <= 0) per_sm = 32;
    if (need > (int64_t)per_sm * h->num_sms) need = (int64_t)per_sm * h->num_sms;
    if (PCG && need > MAX_PARTIALS) need = MAX_PARTIALS; // grid warps <= partial slots
    return launch_persistent(h, (const void *)k_psolve<T, FWD, PCG>, PBLOCK, 0, need, args);
}

int p_lsolve(gic_handle *h, const Pattern &P, bool f32, const void *Vf, const void *r, void *y, const Scalars *sc)
{
    Scalars *s = const_cast<Scalars *>(sc);
    if (f32) return p_launch<float, true, false>(h, P, Vf, (const float *)r, (float *)y, nullptr, nullptr, s);
    return p_launch<double, true, false>(h, P, Vf, (const double *)r, (double *)y, nullptr, nullptr, s);
}

int p_ltsolve(gic_handle *h, const Pattern &P, bool f32, bool pcg, const void *Vb, const void *y, void *z,
              const double *rd, double *partials, Scalars *sc)
{
    if (f32) {
        if (pcg) return p_launch<float, false, true>(h, P, Vb, (const float *)y, (float *)z, rd, partials, sc);
        return p_launch<float, false, false>(h, P, Vb, (const float *)y, (float *)z, nullptr, nullptr, sc);
    }
    if (pcg) return p_launch<double, false, true>(h, P, Vb, (const double *)y, (double *)z, rd, partials, sc);
    return p_launch<double, false, false>(h, P, Vb, (const double *)y, (double *)z, nullptr, nullptr, sc);
}

}  // namespace gic
