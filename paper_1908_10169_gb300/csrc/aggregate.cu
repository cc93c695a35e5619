// Progressive aggregation (Sec. 3.5): consecutive blocks of the finished factor merged into
// larger ones.
//
// A merge only rewrites finished blocks.  For a group G of consecutive blocks merged into one,
// with L_GG the unit lower part of L inside the group and T_GG its upper part (the pivot blocks
// P_m on the diagonal, U-breve inside the group above them),
//   L-hat = L_{:,G} L_GG^{-1},  U-hat = L_GG U-breve_{G,:},  P-hat = L_GG T_GG,
//   D-hat = P-hat^{-1} = T_GG^{-1} L_GG^{-1}
// leave the product of the factors unchanged (two blocks at a time this is the rewrite of
// Sec. 3.5; a group is that rewrite applied to each of its blocks in turn).  The later blocks of
// the factorization therefore receive the same updates whether or not the earlier ones were
// merged -- up to rounding: a row of a merged block meets a column only through the common
// pattern when both of their own products are zero, and then the two terms of the merged
// product cancel exactly in exact arithmetic -- so their candidates, drop decisions and kept
// patterns, which the merge test reads, are those of the unmerged factorization.  The merges are
// therefore taken here, after the factorization, walking the blocks in order with the merge
// test on the finished patterns: the same decisions, block after block, as merging inside the
// factorization loop, on any schedule.  The factorization's own arrays stay as they are (the
// next bilu_factor starts again from the analysis partition); the merged copy is what the
// sweeps, the solves and the export read (factor_view).
//
// Host: the merge decisions and the merged patterns (sorted unions of the members' rows and
// columns beyond the group), the block offsets, the row -> block map and the sweeps' producer
// lists -- integer work on the finished patterns.  Device: the merged values, one CTA per group.
#include <algorithm>
#include <chrono>
#include <vector>

#include "dev_common.cuh"

namespace {

constexpr int AGT = 256;                 // threads per CTA
constexpr int AGW = AGT / 32;
constexpr int QS = BILU_MAX_BLOCK + 1;   // padded row stride of the shared w x w matrices
constexpr int AG_SMEM = 5 * BILU_MAX_BLOCK * QS * (int)sizeof(double);

struct AggArgs {
    // the factorization's arrays (analysis blocks)
    const int32_t *bstart, *Lrow, *Ucol;
    const int64_t *Lptr, *Lvptr, *Uptr, *Uvptr, *Dptr;
    const void *Lval, *Uval, *Uhval;
    const double *Dinv, *Pblk;
    // the merged copy
    const int32_t *grp;  // per group: its first and last block
    const int32_t *oLrow, *oUcol;
    const int64_t *oLptr, *oLvptr, *oUptr, *oUvptr, *oDptr;
    void *oLval, *oUval, *oUhval;
    double *oDinv, *oPblk;
};

template <class TS> __device__ __forceinline__ TS to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) {
    return __float2bfloat16((float)v);
}

// first position in sorted a[lo, hi) with a[pos] >= key
__device__ __forceinline__ int64_t lower_pos(const int32_t *a, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One CTA per group of blocks [k0, k1] (the merged block takes index k1; k0 .. k1-1 are void).
// A group of one block is copied unchanged.
template <class TS>
__global__ void __launch_bounds__(AGT) agg_values_kernel(AggArgs a) {
    extern __shared__ double sm[];
    const int g = blockIdx.x;
    const int k0 = a.grp[2 * g], k1 = a.grp[2 * g + 1];
    const int sG = a.bstart[k0], eG = a.bstart[k1 + 1], w = eG - sG;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TS *Lv = (const TS *)a.Lval, *Uv = (const TS *)a.Uval, *Uhv = (const TS *)a.Uhval;
    TS *oLv = (TS *)a.oLval, *oUv = (TS *)a.oUval, *oUhv = (TS *)a.oUhval;
    const int64_t dL = a.oLptr[k1], nR = a.oLptr[k1 + 1] - dL, dLv = a.oLvptr[k1];
    const int64_t dU = a.oUptr[k1], nC = a.oUptr[k1 + 1] - dU, dUv = a.oUvptr[k1];
    const int64_t dD = a.oDptr[k1];
    if (k0 == k1) {
        const int64_t sLv = a.Lvptr[k1], sUv = a.Uvptr[k1], sD = a.Dptr[k1];
        for (int64_t e = tid; e < nR * w; e += AGT) oLv[dLv + e] = Lv[sLv + e];
        for (int64_t e = tid; e < nC * w; e += AGT) {
            oUv[dUv + e] = Uv[sUv + e];
            oUhv[dUv + e] = Uhv[sUv + e];
        }
        for (int e = tid; e < w * w; e += AGT) {
            a.oDinv[dD + e] = a.Dinv[sD + e];
            a.oPblk[dD + e] = a.Pblk[sD + e];
        }
        return;
    }
    double *Lg = sm;                         // L_GG (unit lower)
    double *Tg = Lg + BILU_MAX_BLOCK * QS;   // T_GG (pivot blocks, U-breve above them)
    double *Li = Tg + BILU_MAX_BLOCK * QS;   // L_GG^{-1}
    double *X = Li + BILU_MAX_BLOCK * QS;    // T_GG^{-1}
    double *Y = X + BILU_MAX_BLOCK * QS;     // scratch, then D-hat
    for (int e = tid; e < w * w; e += AGT) {
        const int r = e / w, c = e - r * w;
        Lg[r * QS + c] = r == c ? 1.0 : 0.0;
        Tg[r * QS + c] = 0.0;
        X[r * QS + c] = 0.0;
    }
    __syncthreads();
    for (int m = k0; m <= k1; ++m) {
        const int om = a.bstart[m] - sG, bm = a.bstart[m + 1] - a.bstart[m];
        const double *P = a.Pblk + a.Dptr[m];
        for (int e = tid; e < bm * bm; e += AGT) {
            const int r = e / bm, c = e - r * bm;
            Tg[(om + r) * QS + om + c] = P[e];
        }
        // the member's rows (columns) inside the group come first: they are sorted
        const int64_t l0 = a.Lptr[m], lin = lower_pos(a.Lrow, l0, a.Lptr[m + 1], eG) - l0;
        const TS *lv = Lv + a.Lvptr[m];
        for (int64_t e = tid; e < lin * bm; e += AGT) {
            const int64_t ir = e / bm;
            const int c = (int)(e - ir * bm);
            Lg[(a.Lrow[l0 + ir] - sG) * QS + om + c] = dval(lv[e]);
        }
        const int64_t u0 = a.Uptr[m], uin = lower_pos(a.Ucol, u0, a.Uptr[m + 1], eG) - u0;
        const TS *uv = Uv + a.Uvptr[m];
        for (int64_t e = tid; e < uin * bm; e += AGT) {
            const int64_t iq = e / bm;
            const int c = (int)(e - iq * bm);
            Tg[(om + c) * QS + (a.Ucol[u0 + iq] - sG)] = dval(uv[e]);
        }
    }
    __syncthreads();
    // L_GG^{-1}: thread c forms column c by forward substitution
    if (tid < w) {
        const int c = tid;
        for (int i = 0; i < w; ++i) Li[i * QS + c] = i == c ? 1.0 : 0.0;
        for (int i = c + 1; i < w; ++i) {
            double s = 0.0;
            for (int k = c; k < i; ++k) s = fma(Lg[i * QS + k], Li[k * QS + c], s);
            Li[i * QS + c] = -s;
        }
    }
    // T_GG^{-1} by block back substitution, members from the last to the first:
    // X[m rows, :] = D_m (E_m - T_GG[m rows, later columns] X[later rows, :])
    for (int m = k1; m >= k0; --m) {
        const int om = a.bstart[m] - sG, bm = a.bstart[m + 1] - a.bstart[m], oe = om + bm;
        __syncthreads();
        for (int e = tid; e < bm * w; e += AGT) {
            const int r = e / w, c = e - r * w;
            double s = om + r == c ? 1.0 : 0.0;
            for (int k = oe; k < w; ++k) s = fma(-Tg[(om + r) * QS + k], X[k * QS + c], s);
            Y[r * QS + c] = s;
        }
        __syncthreads();
        const double *D = a.Dinv + a.Dptr[m];
        for (int e = tid; e < bm * w; e += AGT) {
            const int r = e / w, c = e - r * w;
            double s = 0.0;
            for (int k = 0; k < bm; ++k) s = fma(D[r * bm + k], Y[k * QS + c], s);
            X[(om + r) * QS + c] = s;
        }
    }
    __syncthreads();
    // D-hat = T_GG^{-1} L_GG^{-1} (kept in Y for the columns below), P-hat = L_GG T_GG
    for (int e = tid; e < w * w; e += AGT) {
        const int r = e / w, c = e - r * w;
        double s = 0.0;
        for (int k = c; k < w; ++k) s = fma(X[r * QS + k], Li[k * QS + c], s);
        Y[r * QS + c] = s;
        a.oDinv[dD + e] = s;
        double p = 0.0;
        for (int k = 0; k <= r; ++k) p = fma(Lg[r * QS + k], Tg[k * QS + c], p);
        a.oPblk[dD + e] = p;
    }
    __syncthreads();
    // merged rows l-hat_i = [L_{i,m}]_m L_GG^{-1}: a warp per row, lanes own columns lane, lane+32
    for (int64_t e = warp; e < nR; e += AGW) {
        const int32_t i = a.oLrow[dL + e];
        double x0 = 0.0, x1 = 0.0;
        for (int m = k0; m <= k1; ++m) {
            const int om = a.bstart[m] - sG, bm = a.bstart[m + 1] - a.bstart[m];
            const int64_t l0 = a.Lptr[m], l1 = a.Lptr[m + 1], pos = lower_pos(a.Lrow, l0, l1, i);
            if (pos < l1 && a.Lrow[pos] == i) {
                const TS *row = Lv + a.Lvptr[m] + (pos - l0) * bm;
                if (lane >= om && lane < om + bm) x0 = dval(row[lane - om]);
                if (lane + 32 >= om && lane + 32 < om + bm) x1 = dval(row[lane + 32 - om]);
            }
        }
        double o0 = 0.0, o1 = 0.0;
        for (int k = 0; k < w; ++k) {
            const double xk = __shfl_sync(FULL_MASK, k < 32 ? x0 : x1, k & 31);
            if (lane <= k) o0 = fma(xk, Li[k * QS + lane], o0);
            if (lane + 32 <= k) o1 = fma(xk, Li[k * QS + lane + 32], o1);
        }
        TS *out = oLv + dLv + e * w;
        if (lane < w) out[lane] = to_store<TS>(o0);
        if (lane + 32 < w) out[lane + 32] = to_store<TS>(o1);
    }
    // merged columns u-hat_j = L_GG [U-breve_{m,j}]_m, and D-hat u-hat_j for the backward sweep
    for (int64_t e = warp; e < nC; e += AGW) {
        const int32_t j = a.oUcol[dU + e];
        double y0 = 0.0, y1 = 0.0;
        for (int m = k0; m <= k1; ++m) {
            const int om = a.bstart[m] - sG, bm = a.bstart[m + 1] - a.bstart[m];
            const int64_t u0 = a.Uptr[m], u1 = a.Uptr[m + 1], pos = lower_pos(a.Ucol, u0, u1, j);
            if (pos < u1 && a.Ucol[pos] == j) {
                const TS *col = Uv + a.Uvptr[m] + (pos - u0) * bm;
                if (lane >= om && lane < om + bm) y0 = dval(col[lane - om]);
                if (lane + 32 >= om && lane + 32 < om + bm) y1 = dval(col[lane + 32 - om]);
            }
        }
        double v0 = 0.0, v1 = 0.0;
        for (int k = 0; k < w; ++k) {
            const double yk = __shfl_sync(FULL_MASK, k < 32 ? y0 : y1, k & 31);
            if (lane >= k && lane < w) v0 = fma(Lg[lane * QS + k], yk, v0);
            if (lane + 32 >= k && lane + 32 < w) v1 = fma(Lg[(lane + 32) * QS + k], yk, v1);
        }
        double h0 = 0.0, h1 = 0.0;
        for (int k = 0; k < w; ++k) {
            const double vk = __shfl_sync(FULL_MASK, k < 32 ? v0 : v1, k & 31);
            if (lane < w) h0 = fma(Y[lane * QS + k], vk, h0);
            if (lane + 32 < w) h1 = fma(Y[(lane + 32) * QS + k], vk, h1);
        }
        TS *ou = oUv + dUv + e * w, *oh = oUhv + dUv + e * w;
        if (lane < w) {
            ou[lane] = to_store<TS>(v0);
            oh[lane] = to_store<TS>(h0);
        }
        if (lane + 32 < w) {
            ou[lane + 32] = to_store<TS>(v1);
            oh[lane + 32] = to_store<TS>(h1);
        }
    }
}

// Sec. 3.5 merge test: mu values stored before the merge, nu after it (the diagonal block
// dense); merge iff nu <= 1.2 mu (compared exactly as 5 nu <= 6 mu) or nu <= mu + 2 (p + q).
bool merge_test(int64_t p, int64_t q, int64_t r, int64_t s, int64_t rp, int64_t sp, int64_t t, int64_t tp,
                int64_t u, int64_t v) {
    const int64_t mu = p * (p + r + s + rp + sp) + q * (q + t + tp);
    const int64_t nu = (p + q) * (p + q + u + v);
    return 5 * nu <= 6 * mu || nu <= mu + 2 * (p + q);
}

int64_t union_size(const int32_t *a, int64_t na, const int32_t *b, int64_t nb) {
    int64_t i = 0, j = 0, m = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (b[j] < a[i]) ++j;
        else { ++i; ++j; }
        ++m;
    }
    return m + (na - i) + (nb - j);
}

struct Plan {
    std::vector<int32_t> bstart, blkof, Lrow, Ucol, grp, prodU, prodUcnt;
    std::vector<int64_t> ptr;  // Lptr, Lvptr, Uptr, Uvptr, Dptr, each nb + 1
    int32_t merges = 0, bmax = 0, prodcap = 1;
};

// The merge decisions in block order and the merged copy's integer structure.
void make_plan(const std::vector<int32_t> &bs, const std::vector<int64_t> &Lp, const std::vector<int32_t> &Lr,
               const std::vector<int64_t> &Up, const std::vector<int32_t> &Uc, int amax, Plan &pl) {
    const int32_t nb = (int32_t)bs.size() - 1;
    const int64_t n = bs[nb];
    pl.bstart = bs;
    std::vector<int64_t> nL(nb, 0), nU(nb, 0), wd(nb, 0);
    std::vector<int32_t> R, C, tmp;
    int32_t k0 = 0;
    R.assign(Lr.begin() + Lp[0], Lr.begin() + Lp[1]);
    C.assign(Uc.begin() + Up[0], Uc.begin() + Up[1]);
    auto close = [&](int32_t k1) {
        pl.grp.push_back(k0);
        pl.grp.push_back(k1);
        for (int32_t k = k0; k <= k1; ++k) pl.bstart[k] = bs[k0];
        nL[k1] = (int64_t)R.size();
        nU[k1] = (int64_t)C.size();
        wd[k1] = bs[k1 + 1] - bs[k0];
        pl.bmax = std::max<int32_t>(pl.bmax, (int32_t)wd[k1]);
        pl.Lrow.insert(pl.Lrow.end(), R.begin(), R.end());
        pl.Ucol.insert(pl.Ucol.end(), C.begin(), C.end());
    };
    for (int32_t K = 1; K < nb; ++K) {
        const int64_t s0 = bs[K], s1 = bs[K + 1], p = s0 - bs[k0], q = s1 - s0;
        const int32_t *rK = Lr.data() + Lp[K], *cK = Uc.data() + Up[K];
        const int64_t t = Lp[K + 1] - Lp[K], tp = Up[K + 1] - Up[K];
        // the group's rows (columns) inside B_K come first
        const int64_t r = std::lower_bound(R.begin(), R.end(), (int32_t)s1) - R.begin(), s = (int64_t)R.size() - r;
        const int64_t rp = std::lower_bound(C.begin(), C.end(), (int32_t)s1) - C.begin(), sp = (int64_t)C.size() - rp;
        bool merge = p + q <= amax;
        if (merge) {
            const int64_t u = union_size(R.data() + r, s, rK, t), v = union_size(C.data() + rp, sp, cK, tp);
            merge = merge_test(p, q, r, s, rp, sp, t, tp, u, v);
        }
        if (merge) {
            tmp.clear();
            std::set_union(R.begin() + r, R.end(), rK, rK + t, std::back_inserter(tmp));
            R.swap(tmp);
            tmp.clear();
            std::set_union(C.begin() + rp, C.end(), cK, cK + tp, std::back_inserter(tmp));
            C.swap(tmp);
            pl.merges += 1;
        } else {
            close(K - 1);
            k0 = K;
            R.assign(rK, rK + t);
            C.assign(cK, cK + tp);
        }
    }
    close(nb - 1);
    pl.ptr.assign(5 * (size_t)(nb + 1), 0);
    int64_t *Lptr = pl.ptr.data(), *Lvptr = Lptr + nb + 1, *Uptr = Lvptr + nb + 1, *Uvptr = Uptr + nb + 1,
            *Dptr = Uvptr + nb + 1;
    for (int32_t k = 0; k < nb; ++k) {
        Lptr[k + 1] = Lptr[k] + nL[k];
        Lvptr[k + 1] = Lvptr[k] + nL[k] * wd[k];
        Uptr[k + 1] = Uptr[k] + nU[k];
        Uvptr[k + 1] = Uvptr[k] + nU[k] * wd[k];
        Dptr[k + 1] = Dptr[k] + wd[k] * wd[k];
    }
    pl.blkof.assign((size_t)n, 0);
    const int32_t ng = (int32_t)pl.grp.size() / 2;
    for (int32_t g = 0; g < ng; ++g)
        for (int32_t i = bs[pl.grp[2 * g]]; i < bs[pl.grp[2 * g + 1] + 1]; ++i) pl.blkof[i] = pl.grp[2 * g + 1];
    // producer lists of the forward sweep: for block K, the blocks with kept rows of L inside
    // B_K, ascending (groups are visited in order)
    std::vector<std::vector<int32_t>> lists((size_t)nb);
    for (int32_t g = 0; g < ng; ++g) {
        const int32_t k1 = pl.grp[2 * g + 1];
        int32_t last = -1;
        for (int64_t e = Lptr[k1]; e < Lptr[k1 + 1]; ++e) {
            const int32_t tb = pl.blkof[pl.Lrow[e]];
            if (tb != last) {
                lists[tb].push_back(k1);
                last = tb;
            }
        }
    }
    pl.prodcap = 1;
    for (const auto &l : lists) pl.prodcap = std::max<int32_t>(pl.prodcap, (int32_t)l.size());
    pl.prodU.assign((size_t)nb * pl.prodcap, 0);
    pl.prodUcnt.assign((size_t)nb, 0);
    for (int32_t k = 0; k < nb; ++k) {
        pl.prodUcnt[k] = (int32_t)lists[k].size();
        std::copy(lists[k].begin(), lists[k].end(), pl.prodU.begin() + (int64_t)k * pl.prodcap);
    }
}

template <class T>
cudaError_t grow(T *&p, int64_t &cap, int64_t need) {
    if (p && need <= cap) return cudaSuccess;
    dev_free(p);
    cap = 0;
    const int64_t nc = std::max<int64_t>(need + need / 8, 1);
    cudaError_t e = dev_alloc(&p, nc);
    if (e == cudaSuccess) cap = nc;
    return e;
}

template <class T>
cudaError_t h2d(T *dst, const std::vector<T> &src, cudaStream_t st) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

template <class TS>
cudaError_t launch_values(const AggArgs &a, int ng, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(agg_values_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, AG_SMEM);
    if (e != cudaSuccess) return e;
    agg_values_kernel<TS><<<ng, AGT, AG_SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

void aggregate_free(bilu_ctx *c) {
    dev_free(c->d_ag_bstart); dev_free(c->d_ag_blkof); dev_free(c->d_ag_Lrow); dev_free(c->d_ag_Ucol);
    dev_free(c->d_ag_prodU); dev_free(c->d_ag_prodUcnt); dev_free(c->d_ag_grp); dev_free(c->d_ag_ptr);
    char *lv = (char *)c->d_ag_Lval, *uv = (char *)c->d_ag_Uval, *uh = (char *)c->d_ag_Uhval;
    dev_free(lv); dev_free(uv); dev_free(uh);
    c->d_ag_Lval = c->d_ag_Uval = c->d_ag_Uhval = nullptr;
    dev_free(c->d_ag_Dinv); dev_free(c->d_ag_Pblk);
    for (auto &v : c->ag_cap) v = 0;
    c->agg_merges = 0;
    c->h_ag_bstart.clear();
}

FactorView factor_view(const bilu_ctx *c) {
    FactorView v;
    v.nb = c->nb;
    if (c->agg_merges > 0) {
        const int64_t nb1 = c->nb + 1;
        v.prodcap = c->agg_prodcap;
        v.bstart = c->d_ag_bstart; v.blkof = c->d_ag_blkof; v.Lrow = c->d_ag_Lrow; v.Ucol = c->d_ag_Ucol;
        v.prodU = c->d_ag_prodU; v.prodUcnt = c->d_ag_prodUcnt;
        v.Lptr = c->d_ag_ptr; v.Lvptr = c->d_ag_ptr + nb1; v.Uptr = c->d_ag_ptr + 2 * nb1;
        v.Uvptr = c->d_ag_ptr + 3 * nb1; v.Dptr = c->d_ag_ptr + 4 * nb1;
        v.Lval = c->d_ag_Lval; v.Uval = c->d_ag_Uval; v.Uhval = c->d_ag_Uhval;
        v.Dinv = c->d_ag_Dinv; v.Pblk = c->d_ag_Pblk;
        v.kept_rows = c->agg_rows; v.kept_cols = c->agg_cols;
        v.nnz_l = c->agg_nnz_l; v.nnz_u = c->agg_nnz_u; v.nnz_d = c->agg_nnz_d;
    } else {
        v.prodcap = c->prodcap;
        v.bstart = c->d_bstart; v.blkof = c->d_blkof; v.Lrow = c->d_Lrow; v.Ucol = c->d_Ucol;
        v.prodU = c->d_prodU; v.prodUcnt = c->d_prodUcnt;
        v.Lptr = c->d_Lptr; v.Lvptr = c->d_Lvptr; v.Uptr = c->d_Uptr; v.Uvptr = c->d_Uvptr; v.Dptr = c->d_Dptr;
        v.Lval = c->d_Lval; v.Uval = c->d_Uval; v.Uhval = c->d_Uhval;
        v.Dinv = c->d_Dinv; v.Pblk = c->d_Pblk;
        v.kept_rows = c->kept_rows; v.kept_cols = c->kept_cols;
        v.nnz_l = c->nnz_l; v.nnz_u = c->nnz_u; v.nnz_d = c->h_Dptr.empty() ? 0 : c->h_Dptr.back();
    }
    return v;
}

bilu_status aggregate_run(bilu_ctx *c) {
    c->agg_merges = 0;
    c->t_aggregate_ms = 0.0;
    if (c->p.aggregate_max < 2 || c->nb < 2) return BILU_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const int32_t nb = c->nb;
    std::vector<int64_t> Lp(nb + 1), Up(nb + 1);
    std::vector<int32_t> Lr((size_t)c->kept_rows), Uc((size_t)c->kept_cols);
    BILU_CUDA(c, cudaMemcpyAsync(Lp.data(), c->d_Lptr, (nb + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    BILU_CUDA(c, cudaMemcpyAsync(Up.data(), c->d_Uptr, (nb + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    if (!Lr.empty())
        BILU_CUDA(c, cudaMemcpyAsync(Lr.data(), c->d_Lrow, Lr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    if (!Uc.empty())
        BILU_CUDA(c, cudaMemcpyAsync(Uc.data(), c->d_Ucol, Uc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    if (Lp[nb] != c->kept_rows || Up[nb] != c->kept_cols)
        return set_err(c, BILU_ERR_STATE, "aggregation: factor offsets disagree with the kept counts");
    Plan pl;
    make_plan(c->h_bstart, Lp, Lr, Up, Uc, c->p.aggregate_max, pl);
    if (pl.merges == 0) {
        c->t_aggregate_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return BILU_OK;
    }
    const int64_t nb1 = nb + 1;
    const int64_t *P = pl.ptr.data();
    const int64_t nnz_l = P[nb1 + nb], nnz_u = P[3 * nb1 + nb], nnz_d = P[4 * nb1 + nb];
    const size_t es = c->p.precision == BILU_PREC_FP64 ? 8 : c->p.precision == BILU_PREC_FP32 ? 4 : 2;
    const int ng = (int)pl.grp.size() / 2;
    char *lv = (char *)c->d_ag_Lval, *uv = (char *)c->d_ag_Uval, *uh = (char *)c->d_ag_Uhval;
    cudaError_t e;
    if ((e = grow(c->d_ag_bstart, c->ag_cap[0], nb1)) != cudaSuccess ||
        (e = grow(c->d_ag_blkof, c->ag_cap[1], c->n)) != cudaSuccess ||
        (e = grow(c->d_ag_ptr, c->ag_cap[2], 5 * nb1)) != cudaSuccess ||
        (e = grow(c->d_ag_prodUcnt, c->ag_cap[3], nb)) != cudaSuccess ||
        (e = grow(c->d_ag_prodU, c->ag_cap[4], (int64_t)pl.prodU.size())) != cudaSuccess ||
        (e = grow(c->d_ag_Lrow, c->ag_cap[5], (int64_t)pl.Lrow.size())) != cudaSuccess ||
        (e = grow(c->d_ag_Ucol, c->ag_cap[6], (int64_t)pl.Ucol.size())) != cudaSuccess ||
        (e = grow(c->d_ag_grp, c->ag_cap[7], (int64_t)pl.grp.size())) != cudaSuccess ||
        (e = grow(c->d_ag_Dinv, c->ag_cap[8], nnz_d)) != cudaSuccess ||
        (e = grow(c->d_ag_Pblk, c->ag_cap[9], nnz_d)) != cudaSuccess) {
        aggregate_free(c);
        return set_err(c, BILU_ERR_OOM, "aggregation: allocation failed");
    }
    // value buffers in bytes; capacity slot 10 holds the bytes of each
    const int64_t need = std::max<int64_t>(nnz_l, nnz_u) * (int64_t)es;
    if (!lv || !uv || !uh || need > c->ag_cap[10]) {
        dev_free(lv); dev_free(uv); dev_free(uh);
        c->ag_cap[10] = 0;
        const int64_t nc = std::max<int64_t>(need + need / 8, 16);
        if (dev_alloc(&lv, nc) != cudaSuccess || dev_alloc(&uv, nc) != cudaSuccess || dev_alloc(&uh, nc) != cudaSuccess) {
            dev_free(lv); dev_free(uv); dev_free(uh);
            c->d_ag_Lval = c->d_ag_Uval = c->d_ag_Uhval = nullptr;
            aggregate_free(c);
            return set_err(c, BILU_ERR_OOM, "aggregation: allocation failed");
        }
        c->ag_cap[10] = nc;
    }
    c->d_ag_Lval = lv;
    c->d_ag_Uval = uv;
    c->d_ag_Uhval = uh;
    BILU_CUDA(c, h2d(c->d_ag_bstart, pl.bstart, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_blkof, pl.blkof, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_ptr, pl.ptr, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_prodUcnt, pl.prodUcnt, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_prodU, pl.prodU, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_Lrow, pl.Lrow, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_Ucol, pl.Ucol, c->stream));
    BILU_CUDA(c, h2d(c->d_ag_grp, pl.grp, c->stream));
    AggArgs a{};
    a.bstart = c->d_bstart; a.Lrow = c->d_Lrow; a.Ucol = c->d_Ucol;
    a.Lptr = c->d_Lptr; a.Lvptr = c->d_Lvptr; a.Uptr = c->d_Uptr; a.Uvptr = c->d_Uvptr; a.Dptr = c->d_Dptr;
    a.Lval = c->d_Lval; a.Uval = c->d_Uval; a.Uhval = c->d_Uhval; a.Dinv = c->d_Dinv; a.Pblk = c->d_Pblk;
    a.grp = c->d_ag_grp; a.oLrow = c->d_ag_Lrow; a.oUcol = c->d_ag_Ucol;
    a.oLptr = c->d_ag_ptr; a.oLvptr = c->d_ag_ptr + nb1; a.oUptr = c->d_ag_ptr + 2 * nb1;
    a.oUvptr = c->d_ag_ptr + 3 * nb1; a.oDptr = c->d_ag_ptr + 4 * nb1;
    a.oLval = lv; a.oUval = uv; a.oUhval = uh; a.oDinv = c->d_ag_Dinv; a.oPblk = c->d_ag_Pblk;
    if (c->p.precision == BILU_PREC_FP64) e = launch_values<double>(a, ng, c->stream);
    else if (c->p.precision == BILU_PREC_FP32) e = launch_values<float>(a, ng, c->stream);
    else e = launch_values<__nv_bfloat16>(a, ng, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "aggregation values kernel");
    c->launches += 1;
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    c->agg_merges = pl.merges;
    c->agg_bmax = pl.bmax;
    c->agg_prodcap = pl.prodcap;
    c->agg_rows = (int64_t)pl.Lrow.size();
    c->agg_cols = (int64_t)pl.Ucol.size();
    c->agg_nnz_l = nnz_l;
    c->agg_nnz_u = nnz_u;
    c->agg_nnz_d = nnz_d;
    c->h_ag_bstart = pl.bstart;
    c->t_aggregate_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return BILU_OK;
}
