// Numeric Crout-type block ILU on the GPU (Algorithm 1 with blocks, Sec. 2.2).
//
// One cooperative persistent kernel walks the diagonal blocks K = 0..nb-1 in order.  For
// each block all CTAs cooperate through five phases separated by a bounded grid barrier:
//   A  candidate sets: the rows of the block column of L and the columns of the block row
//      of U that can be nonzero (A's pattern plus the kept rows / columns of the earlier
//      blocks that update this one), sorted via a bitmap; per-producer update plans.
//   B  accumulation: tiles of candidate rows (and columns) are loaded from A and updated
//      by every producer block J in increasing J: dense products of the producer's kept
//      L rows and U-breve columns, scattered into the tile (gather / GEMM / scatter).
//   C  the pivot block P_K: LU with partial pivoting inside the block (first index of the
//      largest |.|), perturbation of singular blocks (Sec. 3.6).
//   C2 D_K = P_K^{-1}, one column per warp, from the LU factors.
//   D  l_i = T_L[i,:] D_K for candidate rows and u^_j = D_K T_U[:,j] for candidate columns,
//      Euclidean norms, keep iff norm > tau (drop when <= tau, Algorithm 1).
//   E  compaction of the kept rows / columns into the L / U-breve pools (sorted), and
//      producer-list appends for the later blocks they hit (the role of L_head/L_list
//      and U_head/U_list of Sec. 2.1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_bf16.h>

#include "dev_common.cuh"
#include "mlp.cuh"

namespace {

// Value types of one kernel instance: TS stores the L / U-breve values, TA accumulates the
// updates and the scaling.  FP64: double/double; FP32: float/float; BF16: bf16 storage with
// FP32 accumulation.  The pivot LU, the inverse D_K and the drop norms are always FP64.
template <class TS> struct Prec;
template <> struct Prec<double> { using TA = double; };
template <> struct Prec<float> { using TA = float; };
template <> struct Prec<__nv_bfloat16> { using TA = float; };

__device__ __forceinline__ double to_acc_d(double v) { return v; }
__device__ __forceinline__ float to_acc_f(float v) { return v; }
__device__ __forceinline__ float to_acc_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class TA, class TS> __device__ __forceinline__ TA acc_of(TS v);
template <> __device__ __forceinline__ double acc_of<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float acc_of<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float acc_of<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class TS> __device__ __forceinline__ TS store_of(double v);
template <> __device__ __forceinline__ double store_of<double>(double v) { return v; }
template <> __device__ __forceinline__ float store_of<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_of<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }

// L2 loads of data written by other CTAs during the launch, for every value type
__device__ __forceinline__ double ldv(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ldv(const float *p) { return __ldcg(p); }
__device__ __forceinline__ __nv_bfloat16 ldv(const __nv_bfloat16 *p) {
    return __ushort_as_bfloat16(__ldcg((const unsigned short *)p));
}

constexpr int NT = 512;          // threads per CTA
constexpr int NW = NT / 32;      // warps per CTA
static_assert(NW == 16, "the pivot LU's trailing update maps 12 of the 16 warps");
constexpr int TRMAX = 16;        // max candidate slots per accumulation tile
constexpr int PS = BILU_MAX_BLOCK + 1;  // padded row stride (doubles) of staged panels
constexpr int PMAX = 1024;       // max producers per block handled by the kernel
constexpr int SMEM_BYTES = 160 * 1024;  // dynamic shared memory of the factor kernels (one CTA per SM)
constexpr int TRP = 2;           // rows per pivot-row tile
// Producer slices per pivot-row tile: the pivot rows' updates are on the critical path (the LU
// waits for them), so each tile's producer list is split into PPART slices computed side by
// side and summed in slice order when the LU loads the pivot block.
constexpr int PPART = 4;

struct FactorArgs {
    int32_t n, nb, G, perturb;
    double tau, alpha, pert_tau, pert_rho;
    long long spin_limit;
    const int32_t *rowptr, *colind, *colptr, *rowind, *bstart, *blkof;
    const double *val, *cval;
    const int64_t *Dptr;
    int64_t *Lptr, *Lvptr, *Uptr, *Uvptr;
    int32_t *Lrow, *Ucol;
    void *Lval, *Uval;           // factor values, storage type TS of the kernel instance
    void *Uhval;                 // D_K U-breve_K (the normalised columns), layout of Uval, for the sweeps
    double *Dinv, *Pblk;
    int64_t capLrow, capLval, capUcol, capUval;
    int32_t prodcap;
    int32_t *prodL, *prodLcnt, *prodU, *prodUcnt, *lastL, *lastU;
    void *TL, *TU;               // candidate accumulators, type TA of the kernel instance
    void *TUh;                   // per candidate column: u^_j = D_K T_U[:,j] (type TA)
    void *TLP;                   // pivot rows: PPART partial accumulators of b x b (type TA)
    int32_t *rowsL, *rowsU, *keepL, *keepU;
    uint32_t *bmL, *bmU;
    int32_t *wbL, *wbU;          // bitmap word prefix counts
    int32_t *xslotL, *xslotU;    // candidate slot of every producer X entry
    int64_t capXS;
    int64_t *pinfoL, *pinfoU;    // PIS int64 per producer
    int64_t capT;
    double *LU;
    int32_t *perm;
    int32_t *kst;                // [0] mL, [1] mU, [2] pcntL, [3] pcntU
    int32_t *status;
    int64_t *info;
    uint32_t *bar;
    int32_t debug_extra_cta;     // test hook: the barrier waits for one CTA that never comes
    volatile int32_t *trace;     // test hook (tree schedule): per CTA [mode, block, last barrier
                                 // site, CTA-0 wait site, wait heartbeat], mapped host memory, or null
    int64_t *timeline;           // test hook (tree schedule): per block 8 words: group, then the
                                 // clock at its start and after phases A, B+C, C2, (Bs,) D, E
    int32_t trcap;               // most candidate rows per accumulation tile (4..TRMAX)
    int32_t tc;                  // 1: BF16 update tiles on the tensor cores (tcgen05, TMEM)
    int32_t skip_bound;          // 1: skip candidates that the norm bound proves dropped
    int32_t sym;                 // 1: BILDL (symmetric A): the L side only; U-breve's columns
                                 // are L's rows, the pivot block and D_K symmetric
    double *Lnrm, *Unrm;         // per kept row of L: ||l_i||; per kept column of U-breve: ||u_j||
    double *dcolsq;              // squared column norms of D_K (b entries)
    uint32_t *pivdone;           // pivot-row tiles finished for the current block
    double *nrmL, *nrmU;         // per candidate slot: ||l_i|| and ||T_U[:,j]|| (phase D -> E)
    // learned skip: classifier (FP32 normalisation, FP16 weights) and its logit threshold
    int32_t learned;
    float zhi;
    const float *mlp_norm;
    const __half *mlp_w;
    // sample recording: features per candidate slot of the current block (phase B -> D),
    // the sample arrays and their fill count
    int32_t record;
    uint32_t rec_thresh;
    uint64_t rec_seed;
    long long rec_cap;
    float *featL, *featU;
    float *rec_x, *rec_y;
    long long *rec_tag;
    unsigned long long *rec_count;
    // end of block K's kept rows of L / columns of U-breve (chain schedule: Lptr + 1, Uptr + 1)
    int64_t *Lend, *Uend;
    // tree schedule: blocks of different subtrees finish in any order, so the pools are filled
    // from per-group chunks (arena) and the producer lists are sorted before use
    int32_t arena, sortprod;
    int64_t *gcur;               // this group's chunk cursors: [cur, end] for L rows, L values,
                                 // U columns, U values, then the current block's four bases
    unsigned long long *acur;    // global cursors of the four pools
    int64_t chunkR, chunkV;      // chunk sizes (rows / columns, values)
};

// (always PPART: the factor must not depend on the launch configuration, so that a batched
// factorization equals the one-by-one factorization bit for bit)
__device__ __forceinline__ int pivot_parts(int W, int npt) { return PPART; }

// pinfo layout (per producer t of the current block)
enum { PI_J = 0, PI_BJ, PI_XCNT, PI_YCNT, PI_OFF, PI_XPOS, PI_XVAL, PI_YVAL, PI_YPOS, PI_YF, PIS };

// Rank of this CTA inside its group of a.G CTAs (the whole grid for one matrix; a slice of
// the grid when a batch of matrices is factored in one launch).
__device__ __forceinline__ int crank(const FactorArgs &a) { return (int)(blockIdx.x % (unsigned)a.G); }

__device__ __forceinline__ double perturbed(double d, double ptau, double prho, double alpha) {
    // Sec. 3.6: d (1 + rho beta_j) + sign(d) tau alpha with beta_j := 1 and sign(0) := +1
    return d * (1.0 + prho) + (d >= 0.0 ? 1.0 : -1.0) * ptau * alpha;
}

// ---------------------------------------------------------------- phase A
// Candidate set and update plan of one side (L: rows of the block column, U: columns of
// the block row) of block K; executed by one whole CTA.  All loops over the producers'
// entries are flat (one pass over every entry of every producer) so that the global
// loads are issued together instead of one producer after another.
__device__ __forceinline__ int find_owner(const int32_t *off, int pcnt, int f) {
    // largest t with off[t] <= f (off is the exclusive prefix of the producers' counts)
    int lo = 0, hi = pcnt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// BILDL has no row-block pass, whose phase A sorts the list of blocks with kept L rows in B_K;
// the forward sweep folds those producers in list order, so under the tree schedule (appends
// in any order) the list is sorted here instead.  Shared scratch: 2 PMAX ints.
__device__ void sort_row_producers(const FactorArgs &a, int K, char *smem) {
    int32_t *plist = a.prodU + (int64_t)K * a.prodcap;
    const int pcnt = min(min(ldcg(a.prodUcnt + K), a.prodcap), PMAX);  // an overflow is phase A's to report
    if (pcnt < 2) return;
    int32_t *sl = (int32_t *)smem, *st = sl + PMAX;
    for (int t = threadIdx.x; t < pcnt; t += NT) sl[t] = ldcg(plist + t);
    __syncthreads();
    for (int t = threadIdx.x; t < pcnt; t += NT) {  // rank sort: the entries are distinct
        const int v = sl[t];
        int r = 0;
        for (int u = 0; u < pcnt; ++u) r += sl[u] < v;
        st[r] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < pcnt; t += NT) plist[t] = st[t];
    __syncthreads();
}

__device__ void phase_A(const FactorArgs &a, int K, bool Lside, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    int32_t *xcnt = (int32_t *)smem;            // PMAX
    int32_t *off = xcnt + PMAX;                  // PMAX + 1
    int32_t *xposs = off + PMAX + 1;             // PMAX
    int32_t *ws = xposs + PMAX;                  // 40
    int32_t *lohi = ws + 40;                     // 2
    int32_t *slist = lohi + 2;                   // PMAX: the producer list
    int32_t *stmp = slist + PMAX;                // PMAX: sort buffer

    int32_t *plist = (Lside ? a.prodL : a.prodU) + (int64_t)K * a.prodcap;
    int pcnt = ldcg((Lside ? a.prodLcnt : a.prodUcnt) + K);
    // until the sets are complete the step's counts say "pivot rows only, no producers", so
    // that the later phases of a step that ends early (an overflow) stay within their buffers
    if (tid == 0) {
        a.kst[Lside ? 0 : 1] = Lside ? b : 0;
        a.kst[Lside ? 2 : 3] = 0;
    }
    if (pcnt > a.prodcap || pcnt > PMAX) {
        if (tid == 0) set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
        pcnt = 0;
    }
    for (int t = tid; t < pcnt; t += NT) slist[t] = ldcg(plist + t);
    __syncthreads();
    if (a.sortprod && pcnt > 1) {
        // blocks of different subtrees append to the list in any order: a rank sort (the
        // entries are distinct) restores increasing J, written back for the later readers
        for (int t = tid; t < pcnt; t += NT) {
            const int v = slist[t];
            int r = 0;
            for (int u = 0; u < pcnt; ++u) r += slist[u] < v;
            stmp[r] = v;
        }
        __syncthreads();
        for (int t = tid; t < pcnt; t += NT) {
            slist[t] = stmp[t];
            plist[t] = stmp[t];
        }
        __syncthreads();
    }
    int64_t *pinfo = Lside ? a.pinfoL : a.pinfoU;
    uint32_t *bm = Lside ? a.bmL : a.bmU;
    int32_t *wb = Lside ? a.wbL : a.wbU;
    int32_t *xslot = Lside ? a.xslotL : a.xslotU;
    int32_t *rows = Lside ? a.rowsL : a.rowsU;
    if (tid == 0) { lohi[0] = INT32_MAX; lohi[1] = -1; }

    // producer ranges: warp per producer
    for (int t = warp; t < pcnt; t += NW) {
        const int J = slist[t];
        const int bJ = a.bstart[J + 1] - a.bstart[J];
        const int l0 = (int)ldcg(a.Lptr + J), l1 = (int)ldcg(a.Lend + J);
        const int u0 = (int)ldcg(a.Uptr + J), u1 = (int)ldcg(a.Uend + J);
        const int64_t lv = ldcg(a.Lvptr + J), uv = ldcg(a.Uvptr + J);
        int xbeg, xend, ybeg, yend;
        int64_t xval, yval;
        if (Lside) {  // X: L_J rows >= s0, Y: U-breve_J columns in [s0, s1)
            xbeg = warp_lower_bound(a.Lrow, l0, l1, s0);
            xend = l1;
            ybeg = warp_lower_bound(a.Ucol, u0, u1, s0);
            yend = warp_lower_bound(a.Ucol, ybeg, u1, s1);
            xval = lv + (int64_t)(xbeg - l0) * bJ;
            yval = uv + (int64_t)(ybeg - u0) * bJ;
        } else {      // X: U-breve_J columns >= s1, Y: L_J rows in [s0, s1)
            xbeg = warp_lower_bound(a.Ucol, u0, u1, s1);
            xend = u1;
            ybeg = warp_lower_bound(a.Lrow, l0, l1, s0);
            yend = warp_lower_bound(a.Lrow, ybeg, l1, s1);
            xval = uv + (int64_t)(xbeg - u0) * bJ;
            yval = lv + (int64_t)(ybeg - l0) * bJ;
        }
        double yf = 0.0;  // Frobenius norm of the producer's Y block (norm-bound skip, features)
        if (a.skip_bound || a.learned || a.record) {
            const double *nrm = Lside ? a.Unrm : a.Lnrm;
            double acc = 0.0;
            for (int y = ybeg + lane; y < yend; y += 32) {
                const double v = ldcg(nrm + y);
                acc = fma(v, v, acc);
            }
            yf = sqrt(warp_sum(acc));
        }
        if (lane == 0) {
            int64_t *pi = pinfo + PIS * t;
            pi[PI_YF] = __double_as_longlong(yf);
            pi[PI_J] = J;
            pi[PI_BJ] = bJ;
            pi[PI_XCNT] = xend - xbeg;
            pi[PI_YCNT] = yend - ybeg;
            pi[PI_XPOS] = xbeg;
            pi[PI_XVAL] = xval;
            pi[PI_YVAL] = yval;
            pi[PI_YPOS] = ybeg;
            xcnt[t] = xend - xbeg;
            xposs[t] = xbeg;
        }
    }
    __syncthreads();
    // exclusive prefix of the producers' X counts
    {
        int carry = 0;
        for (int c0 = 0; c0 < pcnt; c0 += NT) {
            const int t = c0 + tid;
            int tot;
            const int ex = block_excl_scan(t < pcnt ? xcnt[t] : 0, ws, &tot);
            if (t < pcnt) off[t] = carry + ex;
            carry += tot;
        }
        if (tid == 0) off[pcnt] = carry;
        __syncthreads();
    }
    const int total = off[pcnt];
    if ((int64_t)total > a.capXS) {
        if (tid == 0) set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
        return;
    }
    for (int t = tid; t < pcnt; t += NT) pinfo[PIS * t + PI_OFF] = off[t];

    // mark candidates >= s1 in the bitmap: entries of A, then every producer X entry
    int lo = INT32_MAX, hi = -1;
    {
        const int e0 = Lside ? a.colptr[s0] : a.rowptr[s0];
        const int e1 = Lside ? a.colptr[s1] : a.rowptr[s1];
        const int32_t *ind = Lside ? a.rowind : a.colind;
        for (int e = e0 + tid; e < e1; e += NT) {
            const int i = ind[e];
            if (i >= s1) { atomicOr(bm + (i >> 5), 1u << (i & 31)); lo = min(lo, i); hi = max(hi, i); }
        }
    }
    const int32_t *Xidx = Lside ? a.Lrow : a.Ucol;
    for (int f = tid; f < total; f += NT) {
        const int t = find_owner(off, pcnt, f);
        const int i = ldcg(Xidx + xposs[t] + (f - off[t]));
        if (i >= s1) { atomicOr(bm + (i >> 5), 1u << (i & 31)); lo = min(lo, i); hi = max(hi, i); }
    }
    lo = __reduce_min_sync(FULL_MASK, lo);
    hi = __reduce_max_sync(FULL_MASK, hi);
    if (lane == 0) { atomicMin(lohi, lo); atomicMax(lohi + 1, hi); }
    __syncthreads();
    const int glo = lohi[0], ghi = lohi[1];
    const int pre = Lside ? b : 0;  // L: the b pivot rows come first
    int count = 0;
    if (ghi >= 0) {
        const int wlo = glo >> 5, whi = ghi >> 5;
        int carry = 0;
        for (int w0 = wlo; w0 <= whi; w0 += NT) {
            const int w = w0 + tid;
            const uint32_t word = (w <= whi) ? ldcg(bm + w) : 0u;
            int tot;
            const int ex = block_excl_scan(__popc(word), ws, &tot);
            if (w <= whi) {
                wb[w - wlo] = carry + ex;
                uint32_t m = word;
                int k = 0;
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const int64_t pos = (int64_t)pre + carry + ex + k;
                    if (pos < a.capT) rows[pos] = w * 32 + bit;
                    ++k;
                }
            }
            carry += tot;
        }
        count = carry;
    }
    if (Lside)
        for (int r = tid; r < b; r += NT) rows[r] = s0 + r;
    if ((int64_t)pre + count > a.capT) {
        if (tid == 0) set_status(a.status, DEV_INTERNAL, a.info, K);
        return;
    }
    __syncthreads();

    // candidate slot of every producer X entry (monotone in the index)
    const int wlo = glo >> 5;
    for (int f = tid; f < total; f += NT) {
        const int t = find_owner(off, pcnt, f);
        const int i = ldcg(Xidx + xposs[t] + (f - off[t]));
        int slot;
        if (i < s1) {
            slot = i - s0;  // pivot rows (L side only)
        } else {
            const uint32_t word = ldcg(bm + (i >> 5));
            slot = pre + ldcg(wb + ((i >> 5) - wlo)) + __popc(word & ((1u << (i & 31)) - 1u));
        }
        xslot[f] = slot;
    }
    __syncthreads();
    if (ghi >= 0)
        for (int w = (glo >> 5) + tid; w <= (ghi >> 5); w += NT) bm[w] = 0u;
    if (tid == 0) {
        a.kst[Lside ? 0 : 1] = pre + count;
        a.kst[Lside ? 2 : 3] = pcnt;
    }
}

// ---------------------------------------------------------------- phase B
// One tile: candidate slots [sa, sa + cnt) of one side, accumulated in shared memory.
// The producers are processed in increasing J (fixed summation order); while producer t
// is multiplied, the X rows and Y rows of producer t+1 are already loading into registers.
constexpr int PF = (TRMAX * BILU_MAX_BLOCK + BILU_MAX_BLOCK * BILU_MAX_BLOCK + NT - 1) / NT;

template <class TA>
struct ProdStage {
    int nx, ny, bJ;
    TA v[PF];
    int xl, yc;
};

template <class TS>
__device__ __forceinline__ void prefetch_producer(const FactorArgs &a, bool Lside, int t, int sa, int cnt, int s0,
                                                  int b, const int32_t *sxs, const int32_t *sxe,
                                                  const int32_t *pbJ, const int32_t *pny, const int32_t *poff,
                                                  const int64_t *pxv, const int64_t *pyv, const int32_t *pyp,
                                                  ProdStage<typename Prec<TS>::TA> &st) {
    using TA = typename Prec<TS>::TA;
    const int tid = threadIdx.x;
    st.nx = sxe[t] - sxs[t];
    st.ny = pny[t];
    st.bJ = pbJ[t];
    if (st.nx <= 0 || st.ny <= 0) { st.nx = 0; return; }
    const TS *Xpool = (const TS *)(Lside ? a.Lval : a.Uval);
    const TS *Ypool = (const TS *)(Lside ? a.Uval : a.Lval);
    const int32_t *Yidx = Lside ? a.Ucol : a.Lrow;
    const int32_t *xslot = Lside ? a.xslotL : a.xslotU;
    const int nxv = st.nx * st.bJ, tot = nxv + st.ny * st.bJ;
    const int64_t xval = pxv[t] + (int64_t)sxs[t] * st.bJ, yval = pyv[t];
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int e = tid + k * NT;
        st.v[k] = e < nxv ? acc_of<TA, TS>(ldv(Xpool + xval + e))
                          : (e < tot ? acc_of<TA, TS>(ldv(Ypool + yval + (e - nxv))) : TA(0));
    }
    st.xl = tid < st.nx ? ldcg(xslot + poff[t] + sxs[t] + tid) - sa : 0;
    st.yc = (tid >= 64 && tid - 64 < st.ny) ? ldcg(Yidx + pyp[t] + (tid - 64)) - s0 : 0;
}

// bound = true (norm-bound skip, after D_K is known): every candidate row of the tile first
// gets an upper bound of ||T[i,:]||: ||A part|| + sum_J ||X row of J|| * ||Y block of J||_F.
// Rows with bound * ||D_K||_F <= tau (1 - 1e-10) are provably dropped (||l_i|| <= ||T[i,:]||
// ||D_K||_2): their products and scaling are skipped and their keep flag is set to -1.
// feat = true (candidate tiles with the learned skip or sample recording): the tile's rows get
// their classifier features (written out when recording); with the learned skip, rows whose
// logit reaches the threshold are skipped the same way.
// log10(max(x, 1e-30)) in FP32 (x rounded to FP32 first, then clamped)
__device__ __forceinline__ float lg30f(double x) { return log10f(fmaxf((float)x, 1e-30f)); }

// Features of the tile's candidate rows (learned skip, recording) and, with the learned skip,
// the classifier's decisions.  Kept out of line so that it adds no register pressure to the
// update loop of the tile.
__device__ __noinline__ void tile_features(const FactorArgs &a, int K, bool Lside, int sa, int cnt, int b, int s1,
                                           int pcnt, const int32_t *xslot, const int32_t *poff, const int32_t *sxs,
                                           const int32_t *sxe, const int32_t *pxp, const int32_t *pbJ,
                                           const double *pyf, const int32_t *g, const double *bnd, const double *sdf,
                                           const int32_t *sina, double *pn, float *sfeat, float *sh1, float *sh2,
                                           int32_t *act, int32_t *sskip) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // per tile row, over its producers in a fixed order (chunks of 32 producers, lane t of
    // a chunk takes producer c0 + t, lanes combined by a butterfly): sum, max and count of
    // ||X row of J|| ||Y block of J||_F and the sum of b_J
    const double *Xn = Lside ? a.Lnrm : a.Unrm;
    double Sl = 0.0, Ml = 0.0;
    int Cl = 0, Bl = 0;
    for (int c0 = 0; c0 < pcnt; c0 += 32) {
        for (int e = tid; e < TRMAX * 32; e += NT) pn[e] = -1.0;
        __syncthreads();
        for (int t = c0 + warp; t < min(pcnt, c0 + 32); t += NW) {
            const int nx = sxe[t] - sxs[t];
            for (int x = lane; x < nx; x += 32) {
                const int r = ldcg(xslot + poff[t] + sxs[t] + x) - sa;
                if (r >= 0 && r < cnt) pn[r * 32 + (t - c0)] = ldcg(Xn + pxp[t] + sxs[t] + x) * pyf[t];
            }
        }
        __syncthreads();
        if (warp < cnt) {
            const double v = pn[warp * 32 + lane];
            if (v >= 0.0) {
                Sl += v;
                Ml = fmax(Ml, v);
                ++Cl;
                Bl += pbJ[c0 + lane];
            }
        }
        __syncthreads();
    }
    if (warp < cnt) {
        const double S = warp_sum(Sl);
        double M = Ml;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(FULL_MASK, M, o));
        const int C = warp_sum_i(Cl), SB = warp_sum_i(Bl);
        // lane k forms feature k; the logarithms in FP32 (FP64 transcendentals are slow here)
        const int r = warp;
        const double av = bnd[r], d = sdf[1];
        float f = 0.f;
        switch (lane) {
            case 0: f = lg30f(av); break;
            case 1: f = sina[r] ? 1.f : 0.f; break;
            case 2: f = lg30f(S); break;
            case 3: f = lg30f(M); break;
            case 4: f = log2f(1.f + (float)C); break;
            case 5: f = lg30f(d); break;
            case 6: f = lg30f((av + S) * d); break;
            case 7: f = lg30f(a.tau); break;
            case 8: f = (float)b / 64.f; break;
            case 9: f = C > 0 ? (float)SB / (float)C / 64.f : 0.f; break;
            case 10: f = log2f(1.f + (float)max(0, g[r] - s1) / 64.f); break;
            case 11: f = Lside ? 0.f : 1.f; break;
            default: break;
        }
        if (lane < MF) sfeat[r * MF + lane] = f;
    }
    __syncthreads();
    if (a.record) {
        float *fo = (Lside ? a.featL : a.featU) + (int64_t)sa * MF;
        for (int e = tid; e < cnt * MF; e += NT) fo[e] = sfeat[e];
    }
    if (a.learned) {
        // the classifier, in the summation order of the sequential inference
        for (int e = tid; e < cnt * MF; e += NT) sfeat[e] = mlp_std(a.mlp_norm, e % MF, sfeat[e]);
        __syncthreads();
        for (int e = tid; e < cnt * MH; e += NT) {
            const int r = e / MH, u = e - r * MH;
            float acc = mlp_w(a.mlp_w, MO_B1 + u);
            for (int k = 0; k < MF; ++k) acc = fmaf(mlp_w(a.mlp_w, MO_W1 + u * MF + k), sfeat[r * MF + k], acc);
            sh1[e] = fmaxf(acc, 0.f);
        }
        __syncthreads();
        for (int e = tid; e < cnt * MH; e += NT) {
            const int r = e / MH, u = e - r * MH;
            float acc = mlp_w(a.mlp_w, MO_B2 + u);
            for (int k = 0; k < MH; ++k) acc = fmaf(mlp_w(a.mlp_w, MO_W2 + u * MH + k), sh1[r * MH + k], acc);
            sh2[e] = fmaxf(acc, 0.f);
        }
        __syncthreads();
        int32_t *kp = Lside ? a.keepL : a.keepU;
        for (int r = tid; r < cnt; r += NT) {
            float z = mlp_w(a.mlp_w, MO_B3);
            for (int u = 0; u < MH; ++u) z = fmaf(mlp_w(a.mlp_w, MO_W3 + u), sh2[r * MH + u], z);
            const bool pivot_row = Lside && sa + r < b;
            const bool drop = !pivot_row && z >= a.zhi;
            act[r] = drop ? 0 : 1;
            kp[sa + r] = drop ? -1 : 0;
            if (drop) atomicAdd(sskip, 1);
        }
        __syncthreads();
    }
    }

// ---------------------------------------------------------------- tensor-core update tiles
// BF16 storage: the Schur updates of a tile, T[r, c] = A_part[r, c] - sum_J X_J[r, :] Y_J[c, :]
// (L side: X_J the tile's rows of L_J, Y_J the columns of U-breve_J inside B_K; U side: X_J
// the tile's columns of U-breve_J, Y_J the rows of L_J inside B_K), run on the 5th-generation
// tensor cores: per producer J (increasing J) the tile's X rows are placed at their tile slots
// in a zero 128 x 64 BF16 operand and the Y rows at their B_K columns in a zero 64 x 64 one,
// both in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix), and
// ceil(b_J / 16) MMAs of 128 x 64 x 16 accumulate X_J Y_J^T in FP32 in tensor memory (TMEM,
// 128 lanes = tile rows, 64 columns).  The products of BF16 values are exact in FP32; the
// accumulation is FP32.  One thread issues the MMAs; their completion arrives on an mbarrier
// that the CTA waits on (bounded) before the operands are overwritten.  The producers' panel
// ranges (contiguous per producer) and their slot / column indices are copied into shared
// memory by cp.async one producer ahead, so their loads overlap the placement and the MMAs of
// the producer before.
constexpr int TC_ROWS = 128;             // tile rows (MMA M)
constexpr int TC_COLS = BILU_MAX_BLOCK;  // B_K columns (MMA N) and TMEM columns allocated
constexpr uint32_t TC_IDESC = (1u << 4)                    // accumulator FP32
                            | (1u << 7) | (1u << 10)       // A and B BF16, both K-major
                            | ((uint32_t)(TC_COLS >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);

__shared__ uint32_t s_tc_tmem;   // TMEM address of the CTA's accumulator
__shared__ __align__(8) uint64_t s_tc_bar;
__shared__ uint32_t s_tc_phase;  // parity of the mbarrier phase the next commit completes

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte step between core matrices
// along K, sbo = along M (N)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// element offset of (row, k) in the core-matrix layout of a rows x 64 K-major BF16 operand
__device__ __forceinline__ int tc_off(int row, int k) {
    return ((row >> 3) * (BILU_MAX_BLOCK / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// 4-byte asynchronous copy global -> shared (both 4-byte aligned), and its group fences
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <class TS> __device__ __forceinline__ bool tc_on(const FactorArgs &a) { return false; }
template <> __device__ __forceinline__ bool tc_on<__nv_bfloat16>(const FactorArgs &a) { return a.tc != 0; }

// TMEM for the CTA's accumulator and the MMA mbarrier, at kernel start (all threads call)
template <class TS>
__device__ void tc_begin(bool on) {
    if (!on) return;
    if (threadIdx.x < 32)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
                     "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
                     ::"r"(smem_addr(&s_tc_tmem)), "r"((uint32_t)TC_COLS) : "memory");
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_tc_bar)) : "memory");
        s_tc_phase = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// releases the TMEM at kernel end (all threads call, after their last tile)
template <class TS>
__device__ void tc_end(bool on) {
    if (!on) return;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tc_tmem), "r"((uint32_t)TC_COLS)
                     : "memory");
}

// waits (thread 0, bounded) for the MMAs of the last commit; the CTA then goes on together.
// False on timeout (status set).
__device__ __forceinline__ bool tc_wait(const FactorArgs &a, int K) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const uint32_t par = s_tc_phase;
        uint32_t done = 0;
        for (long long it = 0; !done; ++it) {
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(smem_addr(&s_tc_bar)), "r"(par) : "memory");
            if (!done && it > a.spin_limit) break;
        }
        if (done) {
            s_tc_phase = par ^ 1u;
        } else if (atomicCAS(a.status, 0, DEV_TIMEOUT) == 0) {
            a.info[INFO_TIMEOUT_SITE] = 9;
            a.info[INFO_FAIL_BLOCK] = K;
        }
        s_ok = done ? 1 : 0;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return s_ok != 0;
}

// part >= 0: the pivot rows [0, b) of the L side over one of nparts slices of the producer list
// (A's values only in part 0), written to the part's pivot accumulator, which the LU sums in
// part order -- as the FP32-unit pivot-row tiles do, with all rows in one tile.
__device__ void phase_B_tile_tc(const FactorArgs &a, int K, bool Lside, int sa, int cnt, char *smem, int part = -1,
                                int nparts = 1) {
    using TS = __nv_bfloat16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    // shared memory: the tile's A part, the two operands, the producer metadata
    float *Ain = (float *)smem;                              // TC_ROWS x 64
    TS *sA = (TS *)(Ain + TC_ROWS * BILU_MAX_BLOCK);         // TC_ROWS x 64, core-matrix layout
    TS *sB = sA + TC_ROWS * BILU_MAX_BLOCK;                  // 64 x 64, core-matrix layout
    int64_t *pxv = (int64_t *)(sB + BILU_MAX_BLOCK * BILU_MAX_BLOCK);
    int64_t *pyv = pxv + PMAX;
    int32_t *sxs = (int32_t *)(pyv + PMAX), *sxe = sxs + PMAX, *pbJ = sxe + PMAX, *pny = pbJ + PMAX;
    int32_t *poff = pny + PMAX, *pyp = poff + PMAX, *pxc = pyp + PMAX;
    int32_t *g = pxc + PMAX;                                 // TC_ROWS
    int32_t *ws = g + TC_ROWS;                               // 33 (scan scratch)
    if (cnt > TC_ROWS) {
        if (tid == 0) set_status(a.status, DEV_INTERNAL, a.info, K);
        return;
    }
    const int32_t *rows = Lside ? a.rowsL : a.rowsU;
    const int pcnt = ldcg(a.kst + (Lside ? 2 : 3));
    const int64_t *pinfo = Lside ? a.pinfoL : a.pinfoU;
    for (int r = tid; r < cnt; r += NT) g[r] = ldcg(rows + sa + r);
    for (int e = tid; e < TC_ROWS * BILU_MAX_BLOCK; e += NT) Ain[e] = 0.f;
    for (int t = tid; t < pcnt; t += NT) {
        const int64_t *pi = pinfo + PIS * t;
        pbJ[t] = (int)ldcg(pi + PI_BJ);
        pny[t] = (int)ldcg(pi + PI_YCNT);
        poff[t] = (int)ldcg(pi + PI_OFF);
        pyp[t] = (int)ldcg(pi + PI_YPOS);
        pxc[t] = (int)ldcg(pi + PI_XCNT);
        pxv[t] = ldcg(pi + PI_XVAL);
        pyv[t] = ldcg(pi + PI_YVAL);
    }
    __syncthreads();
    // A restricted to B_K: rows i (L side) or columns j (U side) of the tile
    for (int r = warp; r < (part > 0 ? 0 : cnt); r += NW) {
        const int idx = g[r];
        if (Lside) {
            for (int e = a.rowptr[idx] + lane; e < a.rowptr[idx + 1]; e += 32) {
                const int c = a.colind[e];
                if (c >= s0 && c < s1) Ain[r * BILU_MAX_BLOCK + (c - s0)] = (float)a.val[e];
            }
        } else {
            for (int e = a.colptr[idx] + lane; e < a.colptr[idx + 1]; e += 32) {
                const int rr = a.rowind[e];
                if (rr >= s0 && rr < s1) Ain[r * BILU_MAX_BLOCK + (rr - s0)] = (float)a.cval[e];
            }
        }
    }
    const int32_t *xslot = Lside ? a.xslotL : a.xslotU;
    for (int t = warp; t < pcnt; t += NW) {
        const int xs = warp_lower_bound(xslot + poff[t], 0, pxc[t], sa);
        const int xe = warp_lower_bound(xslot + poff[t], xs, pxc[t], sa + cnt);
        if (lane == 0) { sxs[t] = xs; sxe[t] = xe; }
    }
    __syncthreads();
    // the producers with entries in this tile (of the part's slice), increasing
    int32_t *tl = pxc;
    int ntl = 0;
    const int tbeg = part >= 0 ? pcnt * part / nparts : 0;
    const int tend = part >= 0 ? pcnt * (part + 1) / nparts : pcnt;
    for (int c0 = tbeg; c0 < tend; c0 += NT) {
        const int t = c0 + tid;
        const int hit = (t < tend && sxe[t] > sxs[t] && pny[t] > 0) ? 1 : 0;
        int tot;
        const int ex = block_excl_scan(hit, ws, &tot);
        if (hit) tl[ntl + ex] = t;
        ntl += tot;
    }
    __syncthreads();
    const TS *Xpool = (const TS *)(Lside ? a.Lval : a.Uval);
    const TS *Ypool = (const TS *)(Lside ? a.Uval : a.Lval);
    const int32_t *Yidx = Lside ? a.Ucol : a.Lrow;
    // raw panel ranges of two producers in flight (cp.async, 4-byte words): the next producer's
    // X rows, Y rows and their slot / column indices load while the current one is placed and
    // multiplied
    constexpr int RAWX = TC_ROWS * BILU_MAX_BLOCK / 2 + 2, RAWY = BILU_MAX_BLOCK * BILU_MAX_BLOCK / 2 + 2;
    uint32_t *raw = (uint32_t *)(ws + 40);                 // 2 stages: X words, Y words, X slots, Y columns
    const int stage_words = RAWX + RAWY + TC_ROWS + BILU_MAX_BLOCK;
    auto prefetch = [&](int i) {
        const int t = tl[i];
        const int nx = sxe[t] - sxs[t], ny = pny[t], bJ = pbJ[t];
        uint32_t *st = raw + (i & 1) * stage_words;
        const int64_t xval = pxv[t] + (int64_t)sxs[t] * bJ, yval = pyv[t];
        const int64_t xw0 = xval >> 1, yw0 = yval >> 1;
        const int nxw = (int)(((xval + (int64_t)nx * bJ + 1) >> 1) - xw0);
        const int nyw = (int)(((yval + (int64_t)ny * bJ + 1) >> 1) - yw0);
        if (nx <= cnt && ny <= BILU_MAX_BLOCK && bJ <= BILU_MAX_BLOCK && nxw <= RAWX && nyw <= RAWY) {
            const uint32_t *gx = (const uint32_t *)Xpool + xw0, *gy = (const uint32_t *)Ypool + yw0;
            for (int e = tid; e < nxw; e += NT) cp_async4(st + e, gx + e);
            for (int e = tid; e < nyw; e += NT) cp_async4(st + RAWX + e, gy + e);
            for (int e = tid; e < nx; e += NT) cp_async4(st + RAWX + RAWY + e, xslot + poff[t] + sxs[t] + e);
            for (int e = tid; e < ny; e += NT) cp_async4(st + RAWX + RAWY + TC_ROWS + e, Yidx + pyp[t] + e);
        }
        cp_async_commit();
    };
    long long flops = 0;
    bool ok = true;
    if (ntl > 0) prefetch(0);
    for (int i = 0; i < ntl && ok; ++i) {
        const int t = tl[i];
        const int nx = sxe[t] - sxs[t], ny = pny[t], bJ = pbJ[t];
        if (nx > cnt || ny > b || bJ > BILU_MAX_BLOCK) {
            if (tid == 0) set_status(a.status, DEV_INTERNAL, a.info, K);
            ok = false;
            break;
        }
        flops += 2LL * nx * ny * bJ;
        if (i + 1 < ntl) {
            prefetch(i + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // producer i's words are in shared memory for every thread
        if (i > 0 && !tc_wait(a, K)) { ok = false; break; }
        // zero both operands (K padding and absent rows stay zero), then place the values
        {
            uint4 *z = (uint4 *)sA;
            const int nz = (TC_ROWS + BILU_MAX_BLOCK) * BILU_MAX_BLOCK * (int)sizeof(TS) / 16;
            for (int e = tid; e < nz; e += NT) z[e] = make_uint4(0, 0, 0, 0);
        }
        __syncthreads();
        const uint32_t *st = raw + (i & 1) * stage_words;
        const TS *rx = (const TS *)st + ((pxv[t] + (int64_t)sxs[t] * bJ) & 1);
        const TS *ry = (const TS *)(st + RAWX) + (pyv[t] & 1);
        const int32_t *rxs = (const int32_t *)(st + RAWX + RAWY), *ryc = rxs + TC_ROWS;
        const int nxv = nx * bJ, tot = nxv + ny * bJ;
        // row of element e: floor((e + 1/2) / bJ) in FP32 is exact here (e < 2^14, bJ <= 64: the
        // quotient stays at least 1/128 from an integer, far above the FP32 rounding)
        const float rb = 1.0f / (float)bJ;
        for (int e = tid; e < tot; e += NT) {
            if (e < nxv) {
                const int x = (int)(((float)e + 0.5f) * rb), kk = e - x * bJ, r = rxs[x] - sa;
                if (r >= 0 && r < cnt) sA[tc_off(r, kk)] = rx[e];
                else set_status(a.status, DEV_INTERNAL, a.info, K);
            } else {
                const int ee = e - nxv, y = (int)(((float)ee + 0.5f) * rb), kk = ee - y * bJ, c = ryc[y] - s0;
                if (c >= 0 && c < b) sB[tc_off(c, kk)] = ry[ee];
                else set_status(a.status, DEV_INTERNAL, a.info, K);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
            const int ks = (bJ + 15) >> 4;
            for (int s = 0; s < ks; ++s) {
                const uint64_t da = tc_desc(a0 + s * 256, 128, (BILU_MAX_BLOCK / 8) * 128);
                const uint64_t db = tc_desc(b0 + s * 256, 128, (BILU_MAX_BLOCK / 8) * 128);
                const uint32_t accum = (i > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(s_tc_tmem), "l"(da), "l"(db), "r"(TC_IDESC), "r"(accum) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_addr(&s_tc_bar)) : "memory");
        }
    }
    cp_async_wait<0>();  // nothing left in flight when the tile ends early
    if (ok && ntl > 0 && !tc_wait(a, K)) ok = false;
    if (ok) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows), columns 16 (w / 4) ..
        float *out = part >= 0 ? (float *)a.TLP + (int64_t)part * BILU_MAX_BLOCK * BILU_MAX_BLOCK + (int64_t)sa * b
                               : (float *)(Lside ? a.TL : a.TU) + (int64_t)sa * b;
        const int r = (warp & 3) * 32 + lane, c0 = (warp >> 2) * 16;
        uint32_t d[16];
        if (ntl > 0) {
            const uint32_t taddr = s_tc_tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
                           "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]),
                           "=r"(d[14]), "=r"(d[15])
                         : "r"(taddr) : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) d[j] = 0u;
        }
        if (r < cnt) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = c0 + j;
                if (c < b) out[(int64_t)r * b + c] = Ain[r * BILU_MAX_BLOCK + c] - __uint_as_float(d[j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    // the products computed (the algorithmic count, as the FFMA tiles count it)
    {
        long long f = tid == 0 ? flops : 0;
        if (tid == 0 && f) atomicAdd((unsigned long long *)(a.info + (Lside ? INFO_FLOP_UPD_L : INFO_FLOP_UPD_U)),
                                     (unsigned long long)f);
    }
}

template <class TS>
__device__ void phase_B_tile(const FactorArgs &a, int K, bool Lside, int sa, int cnt, char *smem, bool bound,
                             bool feat = false, int part = -1, int nparts = 1) {
    // part >= 0: one of nparts slices of the producer list of pivot-row tile rows [sa, sa+cnt):
    // producers [pcnt * part / nparts, pcnt * (part + 1) / nparts), A's values only in part 0,
    // the partial accumulator written to the pivot-part buffer (summed in part order by the LU)
    static_assert(TRMAX <= NW, "one warp per tile row in the feature pass");
    using TA = typename Prec<TS>::TA;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    TA *T = (TA *)smem;                          // TRMAX * 64
    TA *Xs = T + TRMAX * BILU_MAX_BLOCK;         // TRMAX * PS
    TA *Ys = Xs + TRMAX * PS;                    // 64 * PS
    int64_t *pxv = (int64_t *)(Ys + BILU_MAX_BLOCK * PS);  // PMAX: X value offset
    int64_t *pyv = pxv + PMAX;                   // PMAX: Y value offset
    int32_t *g = (int32_t *)(pyv + PMAX);        // TRMAX
    int32_t *xl = g + TRMAX;                     // TRMAX: local slot of staged X rows
    int32_t *yc = xl + TRMAX;                    // 64: column of staged Y rows
    int32_t *sxs = yc + BILU_MAX_BLOCK;          // PMAX
    int32_t *sxe = sxs + PMAX;                   // PMAX
    int32_t *pbJ = sxe + PMAX;                   // PMAX
    int32_t *pny = pbJ + PMAX;                   // PMAX
    int32_t *poff = pny + PMAX;                  // PMAX
    int32_t *pyp = poff + PMAX;                  // PMAX
    int32_t *pxc = pyp + PMAX;                   // PMAX
    int32_t *pxp = pxc + PMAX;                   // PMAX: X index position
    int32_t *act = pxp + PMAX;                   // TRMAX: row active (not provably dropped)
    double *pyf = (double *)(act + TRMAX);       // PMAX: Frobenius norm of the Y block
    double *bnd = pyf + PMAX;                    // TRMAX: bound of ||T[i,:]||
    double *sdf = bnd + TRMAX;                   // [0] ||D_K||_F, [1] ||D_{K-1}||_F
    int32_t *sskip = (int32_t *)(sdf + 2);       // [0] skipped rows of the tile
    double *pn = sdf + 4;                        // TRMAX x 32: ||X|| ||Y||_F per (row, producer of a chunk)
    float *sfeat = (float *)(pn + TRMAX * 32);   // TRMAX x MF features
    float *sh1 = sfeat + TRMAX * MF;             // TRMAX x MH hidden layer 1
    float *sh2 = sh1 + TRMAX * MH;               // TRMAX x MH hidden layer 2
    int32_t *sina = (int32_t *)(sh2 + TRMAX * MH);  // TRMAX: A has an entry in the row's part
    const bool useact = bound || (feat && a.learned);

    const int32_t *rows = Lside ? a.rowsL : a.rowsU;
    const int pcnt = ldcg(a.kst + (Lside ? 2 : 3));
    const int64_t *pinfo = Lside ? a.pinfoL : a.pinfoU;
    for (int r = tid; r < cnt; r += NT) g[r] = ldcg(rows + sa + r);
    for (int e = tid; e < cnt * b; e += NT) T[e] = 0.0;
    for (int t = tid; t < pcnt; t += NT) {
        const int64_t *pi = pinfo + PIS * t;
        pbJ[t] = (int)ldcg(pi + PI_BJ);
        pny[t] = (int)ldcg(pi + PI_YCNT);
        poff[t] = (int)ldcg(pi + PI_OFF);
        pyp[t] = (int)ldcg(pi + PI_YPOS);
        pxc[t] = (int)ldcg(pi + PI_XCNT);
        pxv[t] = ldcg(pi + PI_XVAL);
        pyv[t] = ldcg(pi + PI_YVAL);
        pxp[t] = (int)ldcg(pi + PI_XPOS);
        pyf[t] = __longlong_as_double(ldcg(pi + PI_YF));
    }
    if (useact || feat) {
        for (int r = tid; r < cnt; r += NT) { act[r] = 1; bnd[r] = 0.0; }
        if (warp == 0) {
            double acc = 0.0;
            if (bound) {
                for (int c = lane; c < b; c += 32) acc += ldcg(a.dcolsq + c);
                acc = warp_sum(acc);
            }
            if (lane == 0) { sdf[0] = sqrt(acc); sskip[0] = 0; }
        }
        if (feat && warp == 1) {  // ||D_{K-1}||_F from the column norms of the previous inverse
            double acc = 0.0;
            if (K > 0) {
                const int bp = a.bstart[K] - a.bstart[K - 1];
                for (int c = lane; c < bp; c += 32) acc += ldcg(a.dcolsq + c);
                acc = warp_sum(acc);
            }
            if (lane == 0) sdf[1] = K > 0 ? sqrt(acc) : (a.alpha > 0.0 ? 1.0 / a.alpha : 1.0);
        }
    }
    __syncthreads();
    // load A: L side rows i of A restricted to columns B_K; U side columns j restricted to rows B_K
    for (int r = warp; r < (part > 0 ? 0 : cnt); r += NW) {
        const int idx = g[r];
        double sq = 0.0;
        bool found = false;
        if (Lside) {
            for (int e = a.rowptr[idx] + lane; e < a.rowptr[idx + 1]; e += 32) {
                const int c = a.colind[e];
                if (c >= s0 && c < s1) {
                    const double v = a.val[e];
                    T[r * b + (c - s0)] = (TA)v;
                    sq = fma(v, v, sq);
                    found = true;
                }
            }
        } else {
            for (int e = a.colptr[idx] + lane; e < a.colptr[idx + 1]; e += 32) {
                const int rr = a.rowind[e];
                if (rr >= s0 && rr < s1) {
                    const double v = a.cval[e];
                    T[r * b + (rr - s0)] = (TA)v;
                    sq = fma(v, v, sq);
                    found = true;
                }
            }
        }
        if (bound || feat) {
            sq = warp_sum(sq);
            const bool any = __any_sync(FULL_MASK, found);
            if (lane == 0) {
                bnd[r] = sqrt(sq);
                sina[r] = any ? 1 : 0;
            }
        }
    }
    // X entries of each producer that fall into this tile (slots are sorted)
    const int32_t *xslot = Lside ? a.xslotL : a.xslotU;
    for (int t = warp; t < pcnt; t += NW) {
        const int xs = warp_lower_bound(xslot + poff[t], 0, pxc[t], sa);
        const int xe = warp_lower_bound(xslot + poff[t], xs, pxc[t], sa + cnt);
        if (lane == 0) { sxs[t] = xs; sxe[t] = xe; }
    }
    __syncthreads();
    if (feat)
        tile_features(a, K, Lside, sa, cnt, b, s1, pcnt, xslot, poff, sxs, sxe, pxp, pbJ, pyf, g, bnd, sdf, sina, pn,
                      sfeat, sh1, sh2, act, sskip);
    if (bound) {
        // bound of ||T[i,:]||; the order of the additions does not matter: rows with a bound
        // near the threshold are kept (margin 1e-10), the exact test then decides
        const double *Xn = Lside ? a.Lnrm : a.Unrm;
        for (int t = 0; t < pcnt; ++t) {
            const int nx = sxe[t] - sxs[t];
            for (int x = tid; x < nx; x += NT) {
                const int r = ldcg(xslot + poff[t] + sxs[t] + x) - sa;
                if (r >= 0 && r < cnt) atomicAdd(bnd + r, ldcg(Xn + pxp[t] + sxs[t] + x) * pyf[t]);
            }
        }
        __syncthreads();
        int32_t *kp = Lside ? a.keepL : a.keepU;
        for (int r = tid; r < cnt; r += NT) {
            const bool pivot_row = Lside && sa + r < b;
            const bool drop = !pivot_row && bnd[r] * sdf[0] <= a.tau * (1.0 - 1e-10);
            act[r] = drop ? 0 : 1;
            kp[sa + r] = drop ? -1 : 0;
            if (drop) atomicAdd(sskip, 1);
        }
        __syncthreads();
    }
    long long flops = 0;
    ProdStage<TA> st;
    const int tbeg = part >= 0 ? pcnt * part / nparts : 0;
    const int tend = part >= 0 ? pcnt * (part + 1) / nparts : pcnt;
    // the producers with entries in this tile, in increasing order (the others add nothing to
    // it, so leaving them out keeps the sums and their order)
    int32_t *tl = pxc;             // free after the searches above
    int32_t *ws = (int32_t *)pn;   // scan scratch (pn is free after the feature pass)
    int ntl = 0;
    for (int c0 = tbeg; c0 < tend; c0 += NT) {
        const int t = c0 + tid;
        const int hit = (t < tend && sxe[t] > sxs[t] && pny[t] > 0) ? 1 : 0;
        int tot;
        const int ex = block_excl_scan(hit, ws, &tot);
        if (hit) tl[ntl + ex] = t;
        ntl += tot;
    }
    __syncthreads();
    if (ntl > 0) prefetch_producer<TS>(a, Lside, tl[0], sa, cnt, s0, b, sxs, sxe, pbJ, pny, poff, pxv, pyv, pyp, st);
    for (int i = 0; i < ntl; ++i) {
        const int nx = st.nx, ny = st.ny, bJ = st.bJ;
        if (nx > 0) {
            if (nx > TRMAX || ny > b) {
                if (tid == 0) set_status(a.status, DEV_INTERNAL, a.info, K);
                return;
            }
            // stage producer t
            const int nxv = nx * bJ, tot = nxv + ny * bJ;
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int e = tid + k * NT;
                if (e < nxv) {
                    const int x = e / bJ;
                    Xs[x * PS + (e - x * bJ)] = st.v[k];
                } else if (e < tot) {
                    const int ee = e - nxv, y = ee / bJ;
                    Ys[y * PS + (ee - y * bJ)] = st.v[k];
                }
            }
            if (tid < nx) {
                int v = st.xl;
                if (v < 0 || v >= cnt) { set_status(a.status, DEV_INTERNAL, a.info, K); v = 0; }
                xl[tid] = v;
            }
            if (tid >= 64 && tid - 64 < ny) {
                int v = st.yc;
                if (v < 0 || v >= b) { set_status(a.status, DEV_INTERNAL, a.info, K); v = 0; }
                yc[tid - 64] = v;
            }
        }
        __syncthreads();
        // the next producer's panels load while this one is multiplied
        if (i + 1 < ntl) prefetch_producer<TS>(a, Lside, tl[i + 1], sa, cnt, s0, b, sxs, sxe, pbJ, pny, poff, pxv, pyv, pyp, st);
        if (nx > 0 && part >= 0) {
            // pivot-row tile: at most TRP x 64 outputs for the CTA's 512 threads, so 4 adjacent
            // lanes share an output and split its contraction (lane q takes k = q, q + 4, ...);
            // their partial sums are combined by a fixed butterfly (same order for every launch)
            constexpr int KS = 4;
            const int q = tid & (KS - 1);
            for (int base = 0; base < nx * ny; base += NT / KS) {
                const int e = base + tid / KS;
                bool on = e < nx * ny;
                int x = 0, y = 0;
                if (on) {
                    x = e / ny;
                    y = e - x * ny;
                    on = !(useact && !act[xl[x]]);
                }
                TA s0a = 0, s1a = 0;
                if (on) {
                    const TA *xr = Xs + x * PS, *yr = Ys + y * PS;
                    int k = q;
                    for (; k + KS < bJ; k += 2 * KS) {
                        s0a = fma(xr[k], yr[k], s0a);
                        s1a = fma(xr[k + KS], yr[k + KS], s1a);
                    }
                    if (k < bJ) s0a = fma(xr[k], yr[k], s0a);
                }
                TA sum = s0a + s1a;
                sum += __shfl_xor_sync(FULL_MASK, sum, 1);
                sum += __shfl_xor_sync(FULL_MASK, sum, 2);
                if (on && q == 0) {
                    flops += 2LL * bJ;
                    T[xl[x] * b + yc[y]] -= sum;
                }
            }
        } else if (nx > 0) {
            for (int e = tid; e < nx * ny; e += NT) {
                const int x = e / ny, y = e - x * ny;
                if (useact && !act[xl[x]]) continue;
                flops += 2LL * bJ;
                const TA *xr = Xs + x * PS, *yr = Ys + y * PS;
                // four independent partial sums: a dependent FP64 FMA takes ~64 cycles here
                TA s0a = 0, s1a = 0, s2a = 0, s3a = 0;
                int k = 0;
                for (; k + 3 < bJ; k += 4) {
                    s0a = fma(xr[k], yr[k], s0a);
                    s1a = fma(xr[k + 1], yr[k + 1], s1a);
                    s2a = fma(xr[k + 2], yr[k + 2], s2a);
                    s3a = fma(xr[k + 3], yr[k + 3], s3a);
                }
                for (; k < bJ; ++k) s0a = fma(xr[k], yr[k], s0a);
                T[xl[x] * b + yc[y]] -= (s0a + s1a) + (s2a + s3a);
            }
        }
        __syncthreads();
    }
    TA *out = part >= 0 ? (TA *)a.TLP + (int64_t)part * BILU_MAX_BLOCK * BILU_MAX_BLOCK + (int64_t)sa * b
                        : (TA *)(Lside ? a.TL : a.TU) + (int64_t)sa * b;
    for (int e = tid; e < cnt * b; e += NT) out[e] = T[e];
    // per-thread counts of the products computed, summed over the CTA
    {
        long long f = flops;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(FULL_MASK, f, o);
        __syncthreads();
        long long *wsum = (long long *)Xs;  // staging area is free now
        if (lane == 0) wsum[warp] = f;
        __syncthreads();
        if (tid == 0) {
            long long tot = 0;
            for (int w = 0; w < NW; ++w) tot += wsum[w];
            if (tot) atomicAdd((unsigned long long *)(a.info + (Lside ? INFO_FLOP_UPD_L : INFO_FLOP_UPD_U)),
                               (unsigned long long)tot);
            if (useact && sskip[0])
                atomicAdd((unsigned long long *)(a.info + (Lside ? INFO_SKIP_ROWS : INFO_SKIP_COLS)),
                          (unsigned long long)sskip[0]);
        }
    }
}

// ---------------------------------------------------------------- phase C
// LU with partial pivoting of the pivot block in shared memory (one CTA), with the
// perturbation of Sec. 3.6.  Writes P (possibly perturbed) to Pblk, LU and perm to scratch.
//
// On this GPU every FP64 instruction (compares included) issues on a pipe with 1/64 of the
// FP32 rate, so the step is organised to keep FP64 instructions off the critical path:
//  * rows stay in place; a logical permutation phys[] (physical row at each position,
//    double-buffered) replaces the row swaps;
//  * pivot search compares |values| as 64-bit integers (the ordering of non-negative
//    doubles is the ordering of their bit patterns), ties go to the smaller logical position
//    (LAPACK's first index of the largest |.| in the swapped order);
//  * lookahead: while warps 1.. update the trailing columns j+2.. with column j, warp 0
//    updates column j+1, picks its pivot, forms 1/pivot and the multipliers of column j+1,
//    so a column step costs one CTA barrier.
__device__ __forceinline__ unsigned long long absbits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// Warp 0, one column step: the column `col` of the rows at logical positions col..b-1 of
// phys_in gets the last rank-1 update (multipliers of column col-1 times the pivot row's value
// u) in registers; the pivot is chosen among those values (largest |.|, ties to the smaller
// position: LAPACK's first index in the swapped order); phys_out = phys_in with positions col
// and q swapped (copied while the reductions run); the column is written back as multipliers
// v * (1/pivot) for every row but the pivot row, which keeps its value.  *sbad = col when the
// pivot magnitude is <= thresh (then nothing is scaled).
__device__ __forceinline__ void lu_column_step(double *M, const int32_t *phys_in, int32_t *phys_out, int b, int col,
                                               bool update, double u, double thresh, double *srp, int *sp,
                                               int *sbad) {
    const int lane = threadIdx.x & 31;
    const int k0 = col + lane, k1 = k0 + 32;
    const int i0 = k0 < b ? phys_in[k0] : 0, i1 = k1 < b ? phys_in[k1] : 0;
    double v0 = 0.0, v1 = 0.0;
    if (k0 < b) {
        v0 = M[i0 * PS + col];
        if (update) v0 = fma(-M[i0 * PS + col - 1], u, v0);
    }
    if (k1 < b) {
        v1 = M[i1 * PS + col];
        if (update) v1 = fma(-M[i1 * PS + col - 1], u, v1);
    }
    // each lane: its candidate (|value| compared as the integer bit pattern); an empty lane
    // offers |0| at position b, which never beats a real candidate
    const unsigned long long a0 = k0 < b ? absbits(v0) : 0ULL, a1 = k1 < b ? absbits(v1) : 0ULL;
    unsigned long long bv = a0;
    int bk = k0 < b ? k0 : b;
    double bval = v0;
    if (k1 < b && a1 > bv) { bv = a1; bk = k1; bval = v1; }
    // the reciprocal of every lane's candidate starts now and overlaps the reduction
    const double rloc = (bk < b && bv != 0ULL) ? recip_nr(bval) : 0.0;
    for (int k = lane; k < b; k += 32) phys_out[k] = phys_in[k];
    const unsigned hi = (unsigned)(bv >> 32), lo = (unsigned)bv;
    const unsigned mhi = __reduce_max_sync(FULL_MASK, hi);
    const unsigned mlo = __reduce_max_sync(FULL_MASK, hi == mhi ? lo : 0u);
    const unsigned kk = (hi == mhi && lo == mlo) ? (unsigned)bk : 0xffffffffu;
    const int q = (int)__reduce_min_sync(FULL_MASK, kk);
    const int owner = (q - col) & 31;
    const double pv = __shfl_sync(FULL_MASK, bval, owner);
    const double rp = __shfl_sync(FULL_MASK, rloc, owner);
    const int p = __shfl_sync(FULL_MASK, q < col + 32 ? i0 : i1, owner);
    const bool bad = !(absbits(pv) > absbits(thresh));
    __syncwarp();
    if (lane == 0) {
        phys_out[col] = p;
        phys_out[q] = i0;  // the row that was at position col
        *srp = rp;
        *sp = p;
        if (bad) *sbad = col;
    }
    if (k0 < b) M[i0 * PS + col] = (!bad && i0 != p) ? v0 * rp : v0;
    if (k1 < b) M[i1 * PS + col] = (!bad && i1 != p) ? v1 * rp : v1;
}

template <class TS>
__device__ void phase_C(const FactorArgs &a, int K, char *smem) {
    using TA = typename Prec<TS>::TA;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    double *P = (double *)smem;                 // b x b (stride PS), current P (perturbed)
    double *M = P + BILU_MAX_BLOCK * PS;        // LU work, physical rows
    double *srp = M + BILU_MAX_BLOCK * PS;      // 2: 1/pivot per step parity
    int32_t *phys = (int32_t *)(srp + 2);       // 2 x 64: physical row at logical position
    int32_t *sp = phys + 2 * BILU_MAX_BLOCK;    // 2: pivot row per step parity
    int32_t *sh = sp + 2;                       // [0] bad column, [2] perturbation count
    unsigned long long *smax = (unsigned long long *)(sh + 4);
    {
        const int np = pivot_parts(a.G > 1 ? a.G - 1 : 1, (b + TRP - 1) / TRP);
        const TA *tp = (const TA *)a.TLP;
        for (int e = tid; e < b * b; e += NT) {
            const int r = e / b, c = e - r * b;
            TA v = ldv(tp + (int64_t)r * b + c);
            for (int q = 1; q < np; ++q) v += ldv(tp + (int64_t)q * BILU_MAX_BLOCK * BILU_MAX_BLOCK + (int64_t)r * b + c);
            P[r * PS + c] = (double)v;
        }
    }
    if (tid == 0) sh[2] = 0;
    __syncthreads();
    if (a.sym) {  // BILDL: the lower triangle defines the symmetric pivot block
        for (int e = tid; e < b * b; e += NT) {
            const int r = e / b, c = e - r * b;
            if (c > r) P[r * PS + c] = P[c * PS + r];
        }
        __syncthreads();
    }
    if (a.perturb) {
        // Sec. 3.6: all-zero columns, then all-zero rows, get their diagonal entry perturbed
        // (the diagonal wins the tie with the other, zero, entries).
        // One warp per column (then per row), its lanes over the entries.
        for (int c = warp; c < b; c += NW) {
            const bool nz = (lane < b && absbits(P[lane * PS + c]) != 0ULL) ||
                            (lane + 32 < b && absbits(P[(lane + 32) * PS + c]) != 0ULL);
            if (!__any_sync(FULL_MASK, nz) && lane == 0) {
                P[c * PS + c] = perturbed(P[c * PS + c], a.pert_tau, a.pert_rho, a.alpha);
                atomicAdd(sh + 2, 1);
            }
        }
        __syncthreads();
        for (int r = warp; r < b; r += NW) {
            const bool nz = (lane < b && absbits(P[r * PS + lane]) != 0ULL) ||
                            (lane + 32 < b && absbits(P[r * PS + lane + 32]) != 0ULL);
            if (!__any_sync(FULL_MASK, nz) && lane == 0) {
                P[r * PS + r] = perturbed(P[r * PS + r], a.pert_tau, a.pert_rho, a.alpha);
                atomicAdd(sh + 2, 1);
            }
        }
        __syncthreads();
    }
    bool done = false;
    for (int attempt = 0; attempt <= 2 * b && !done; ++attempt) {
        // copy P, max |P| (integer view), identity permutation
        unsigned long long mx = 0ULL;
        for (int e = tid; e < b * b; e += NT) {
            const int r = e / b, c = e - r * b;
            const double v = P[r * PS + c];
            M[r * PS + c] = v;
            mx = max(mx, absbits(v));
        }
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
        if (tid == 0) { *smax = 0ULL; sh[0] = -1; }
        if (tid < b) phys[tid] = tid;
        __syncthreads();
        if (lane == 0) atomicMax(smax, mx);
        __syncthreads();
        const double thresh = 1e-14 * __longlong_as_double((long long)*smax);
        // column 0: pivot and multipliers (warp 0)
        if (warp == 0) lu_column_step(M, phys, phys + BILU_MAX_BLOCK, b, 0, false, 0.0, thresh, srp, sp, sh);
        __syncthreads();
        for (int j = 0; j < b; ++j) {
            if (sh[0] >= 0) break;  // uniform: written before the last barrier
            const int cur = (j + 1) & 1;  // permutation after the swap of step j
            const int32_t *ph = phys + cur * BILU_MAX_BLOCK;
            const int p = sp[j & 1];
            const int m = b - j - 1;  // rows below the pivot (logical positions j+1..b-1)
            if (warp == 0) {
                // lookahead: column j+1 of the rows below, its pivot and multipliers
                if (m > 0)
                    lu_column_step(M, ph, phys + (cur ^ 1) * BILU_MAX_BLOCK, b, j + 1, true, M[p * PS + j + 1], thresh,
                                   srp + ((j + 1) & 1), sp + ((j + 1) & 1), sh);
            } else if (m > 1 && (m > 48 || (warp & 3) != 0)) {
                // trailing update of columns j+2.. with the multipliers of column j: while it
                // is large (more than 48 rows below the pivot) it bounds the step and takes all
                // 15 warps; then only the 12 warps off warp 0's scheduler partition (warps 4, 8,
                // 12 would delay warp 0's column chain, which then bounds the step)
                const bool all = m > 48;
                const int rank = all ? warp - 1 : warp - 1 - (warp >> 2);
                const int nw = all ? NW - 1 : 12;
                const int w = m - 1, tot = m * w;
                for (int e = rank * 32 + lane; e < tot; e += nw * 32) {
                    const int r = e / w, c = j + 2 + (e - r * w);
                    const int i = ph[j + 1 + r];
                    M[i * PS + c] = fma(-M[i * PS + j], M[p * PS + c], M[i * PS + c]);
                }
            }
            __syncthreads();
        }
        const int bad = sh[0];
        if (bad < 0) {
            done = true;
            const int fin = b & 1;  // buffer holding the final permutation
            const int64_t dofs = a.Dptr[K];
            for (int e = tid; e < b * b; e += NT) {
                const int r = e / b, c = e - r * b;
                a.Pblk[dofs + e] = P[r * PS + c];
                a.LU[e] = M[phys[fin * BILU_MAX_BLOCK + r] * PS + c];
            }
            for (int i = tid; i < b; i += NT) {
                const int pr = phys[fin * BILU_MAX_BLOCK + i];
                a.perm[i] = pr;
                a.LU[BILU_MAX_BLOCK * BILU_MAX_BLOCK + i] = recip_nr(M[pr * PS + i]);  // for the back substitutions
            }
            break;
        }
        if (!a.perturb) break;
        if (tid == 0) {
            int k = 0;
            for (int i = 1; i < b; ++i)
                if (absbits(P[i * PS + bad]) > absbits(P[k * PS + bad])) k = i;
            if (2.0 * fabs(P[bad * PS + bad]) >= fabs(P[k * PS + bad]) || a.sym) k = bad;  // BILDL: the diagonal
            P[k * PS + bad] = perturbed(P[k * PS + bad], a.pert_tau, a.pert_rho, a.alpha);
            sh[2] += 1;
        }
        __syncthreads();
    }
    if (!done) {
        if (tid == 0) set_status(a.status, DEV_SINGULAR, a.info, K);
        return;
    }
    if (tid == 0 && sh[2] > 0) atomicAdd((unsigned long long *)(a.info + INFO_NPERTURB), (unsigned long long)sh[2]);
}

// ---------------------------------------------------------------- phase C2
// Column c of D_K = P_K^{-1}: solve L U x = e_{perm^{-1}(c)} (P_K X = I), one warp per column.
__device__ void phase_C2(const FactorArgs &a, int K, char *smem) {
    // The solves are chains of dependent FP64 operations, so the columns are spread over the
    // group's CTAs: `per` columns per CTA and round (warps 0 .. per-1), at least two, and
    // more (up to one per warp, then further rounds) when the group has fewer than b/2 CTAs.
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    const int per = min(NW, max(2, (b + a.G - 1) / a.G));
    if (crank(a) * per >= b) return;
    double *M = (double *)smem;
    int32_t *prm = (int32_t *)(M + BILU_MAX_BLOCK * PS);
    double *rdiag = (double *)(prm + BILU_MAX_BLOCK);
    for (int e = tid; e < b * b; e += NT) {
        const int r = e / b, c = e - r * b;
        M[r * PS + c] = ldcg(a.LU + e);
    }
    for (int i = tid; i < b; i += NT) {
        prm[i] = ldcg(a.perm + i);
        rdiag[i] = ldcg(a.LU + BILU_MAX_BLOCK * BILU_MAX_BLOCK + i);
    }
    __syncthreads();
    if (warp >= per) return;
    double *D = a.Dinv + a.Dptr[K];
    for (int c = crank(a) * per + warp; c < b; c += a.G * per) {
        // lane owns rows lane and lane + 32; the right-hand side e has its one at position
        // kq (prm[kq] == c), so the forward solve starts there (the entries above stay 0)
        double y0 = (lane < b && prm[lane] == c) ? 1.0 : 0.0;
        double y1 = (lane + 32 < b && prm[lane + 32] == c) ? 1.0 : 0.0;
        const unsigned m0 = __ballot_sync(FULL_MASK, y0 != 0.0), m1 = __ballot_sync(FULL_MASK, y1 != 0.0);
        const int kq = m0 ? __ffs(m0) - 1 : (m1 ? __ffs(m1) + 31 : 0);
        for (int k = kq; k < b; ++k) {  // forward, unit lower
            const double yk = __shfl_sync(FULL_MASK, k < 32 ? y0 : y1, k & 31);
            if (lane > k && lane < b) y0 -= M[lane * PS + k] * yk;
            if (lane + 32 > k && lane + 32 < b) y1 -= M[(lane + 32) * PS + k] * yk;
        }
        for (int k = b - 1; k >= 0; --k) {  // backward, upper
            double own = k < 32 ? y0 : y1;
            if ((k & 31) == lane) own = own * rdiag[k];
            const double xk = __shfl_sync(FULL_MASK, own, k & 31);
            if (k < 32) { if (lane == k) y0 = xk; } else { if (lane + 32 == k) y1 = xk; }
            if (lane < k) y0 -= M[lane * PS + k] * xk;
            if (lane + 32 < k) y1 -= M[(lane + 32) * PS + k] * xk;
        }
        if (lane < b) D[lane * b + c] = y0;
        if (lane + 32 < b) D[(lane + 32) * b + c] = y1;
        const double csq = warp_sum((lane < b ? y0 * y0 : 0.0) + (lane + 32 < b ? y1 * y1 : 0.0));
        if (lane == 0) a.dcolsq[c] = csq;
    }
}

// ---------------------------------------------------------------- phase D
// Sample recording (whole warp): a candidate is taken when a counter-based hash of (seed, K,
// side, slot) falls below the rate threshold; its features (written by its tile in phase B)
// and its label (1 dropped, 0 kept) go to the next free sample.
__device__ __forceinline__ void record_sample(const FactorArgs &a, int K, int side, int slot, int gidx, bool kept) {
    const int lane = threadIdx.x & 31;
    const uint64_t h = mix64(a.rec_seed ^ mix64(((uint64_t)K << 34) ^ ((uint64_t)side << 33) ^ (uint64_t)(uint32_t)slot));
    if (!(a.rec_thresh == 0xffffffffu || (uint32_t)(h >> 32) < a.rec_thresh)) return;
    unsigned long long pos = 0;
    if (lane == 0) pos = atomicAdd(a.rec_count, 1ULL);
    pos = __shfl_sync(FULL_MASK, pos, 0);
    if (pos >= (unsigned long long)a.rec_cap) return;
    const float *f = (side ? a.featU : a.featL) + (int64_t)slot * MF;
    if (lane < MF) a.rec_x[pos * MF + lane] = ldcg(f + lane);
    if (lane == 0) {
        a.rec_y[pos] = kept ? 0.f : 1.f;
        a.rec_tag[pos] = ((long long)K << 33) | ((long long)side << 32) | (long long)(uint32_t)gidx;
    }
}

// Normalised rows l_i = T_L[i,:] D_K and columns u^_j = D_K T_U[:,j]; keep iff ||.||_2 > tau.
// A candidate is first tested against an upper bound of its norm, ||T_i D_K|| <= sum_k |T_ik|
// ||D_K(k,:)|| (||D_K T_j|| <= sum_k ||D_K(:,k)|| |T_kj| for a column; triangle inequality): b
// flops instead of the b^2 of the product.  When the bound, widened by the rounding of the
// product (gamma_b of the arithmetic, covered by the margin), is <= tau, the computed norm
// would be <= tau as well: the candidate is dropped unscaled (keep flag -2), with the decision
// the product would have given.
template <class TA> struct BoundMargin;
template <> struct BoundMargin<double> { static constexpr double v = 1e-10; };
template <> struct BoundMargin<float> { static constexpr double v = 1e-4; };

template <class TS>
__device__ void phase_D(const FactorArgs &a, int K, char *smem) {
    using TA = typename Prec<TS>::TA;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    const int mL = ldcg(a.kst + 0), mU = ldcg(a.kst + 1);
    const int nLc = mL - b, total = nLc + mU;
    // candidates round-robin over the CTAs first, then over their warps: the FP64 products
    // spread over every SM's FP64 pipe
    if (crank(a) >= total) return;
    TA *Ds = (TA *)smem;
    double *rn = (double *)(Ds + BILU_MAX_BLOCK * PS);  // row norms of D_K (as used, in TA)
    double *cn = rn + BILU_MAX_BLOCK;                   // column norms
    const double *D = a.Dinv + a.Dptr[K];
    for (int e = tid; e < b * b; e += NT) {
        const int r = e / b, c = e - r * b;
        // BILDL: D_K = (X + X^T) / 2 (phase E stores it)
        Ds[r * PS + c] = a.sym ? (TA)((ldcg(D + e) + ldcg(D + c * b + r)) * 0.5) : (TA)ldcg(D + e);
    }
    __syncthreads();
    for (int k = warp; k < b; k += NW) {
        double sr = 0.0, sc = 0.0;
        for (int c = lane; c < b; c += 32) {
            const double vr = (double)Ds[k * PS + c], vc = (double)Ds[c * PS + k];
            sr = fma(vr, vr, sr);
            sc = fma(vc, vc, sc);
        }
        sr = warp_sum(sr);
        sc = warp_sum(sc);
        if (lane == 0) {
            rn[k] = sqrt(sr);
            cn[k] = sqrt(sc);
        }
    }
    __syncthreads();
    const double tau_b = a.tau / (1.0 + BoundMargin<TA>::v);
    for (int item = crank(a) + a.G * warp; item < total; item += a.G * NW) {
        if (item < nLc) {
            const int slot = b + item;
            if ((a.skip_bound || a.learned) && ldcg(a.keepL + slot) < 0) continue;  // skipped: dropped
            TA *t = (TA *)a.TL + (int64_t)slot * b;
            const TA t0 = lane < b ? ldv(t + lane) : TA(0);
            const TA t1 = lane + 32 < b ? ldv(t + lane + 32) : TA(0);
            const double bnd = warp_sum((lane < b ? fabs((double)t0) * rn[lane] : 0.0) +
                                        (lane + 32 < b ? fabs((double)t1) * rn[lane + 32] : 0.0));
            if (bnd <= tau_b) {
                if (lane == 0) a.keepL[slot] = -2;
                if (a.record) record_sample(a, K, 0, slot, ldcg(a.rowsL + slot), false);
                continue;
            }
            TA l0 = 0, l1 = 0, l0b = 0, l1b = 0;
            int k = 0;
            for (; k + 1 < b; k += 2) {
                const TA tk = __shfl_sync(FULL_MASK, k < 32 ? t0 : t1, k & 31);
                const TA tk1 = __shfl_sync(FULL_MASK, k + 1 < 32 ? t0 : t1, (k + 1) & 31);
                if (lane < b) { l0 = fma(tk, Ds[k * PS + lane], l0); l0b = fma(tk1, Ds[(k + 1) * PS + lane], l0b); }
                if (lane + 32 < b) { l1 = fma(tk, Ds[k * PS + lane + 32], l1); l1b = fma(tk1, Ds[(k + 1) * PS + lane + 32], l1b); }
            }
            if (k < b) {
                const TA tk = __shfl_sync(FULL_MASK, k < 32 ? t0 : t1, k & 31);
                if (lane < b) l0 = fma(tk, Ds[k * PS + lane], l0);
                if (lane + 32 < b) l1 = fma(tk, Ds[k * PS + lane + 32], l1);
            }
            l0 += l0b;
            l1 += l1b;
            const double nrm2 = warp_sum((double)l0 * (double)l0 + (double)l1 * (double)l1);
            // BILDL keeps t_i (U-breve's column i) and writes l_i beside it
            TA *dst = a.sym ? (TA *)a.TUh + (int64_t)slot * b : t;
            if (a.sym) {
                const double tn2 = warp_sum((double)t0 * (double)t0 + (double)t1 * (double)t1);
                if (lane == 0) a.nrmU[slot] = sqrt(tn2);
            }
            if (lane < b) dst[lane] = l0;
            if (lane + 32 < b) dst[lane + 32] = l1;
            if (lane == 0) {
                const double nr = sqrt(nrm2);
                a.keepL[slot] = nr > a.tau ? 1 : 0;
                a.nrmL[slot] = nr;
            }
            if (a.record) record_sample(a, K, 0, slot, ldcg(a.rowsL + slot), sqrt(nrm2) > a.tau);
        } else {
            const int slot = item - nLc;
            if ((a.skip_bound || a.learned) && ldcg(a.keepU + slot) < 0) continue;  // skipped: dropped
            const TA *t = (const TA *)a.TU + (int64_t)slot * b;
            const TA t0 = lane < b ? ldv(t + lane) : TA(0);
            const TA t1 = lane + 32 < b ? ldv(t + lane + 32) : TA(0);
            const double bnd = warp_sum((lane < b ? fabs((double)t0) * cn[lane] : 0.0) +
                                        (lane + 32 < b ? fabs((double)t1) * cn[lane + 32] : 0.0));
            if (bnd <= tau_b) {
                if (lane == 0) a.keepU[slot] = -2;
                if (a.record) record_sample(a, K, 1, slot, ldcg(a.rowsU + slot), false);
                continue;
            }
            TA u0 = 0, u1 = 0, u0b = 0, u1b = 0;
            int k = 0;
            for (; k + 1 < b; k += 2) {
                const TA tk = __shfl_sync(FULL_MASK, k < 32 ? t0 : t1, k & 31);
                const TA tk1 = __shfl_sync(FULL_MASK, k + 1 < 32 ? t0 : t1, (k + 1) & 31);
                if (lane < b) { u0 = fma(Ds[lane * PS + k], tk, u0); u0b = fma(Ds[lane * PS + k + 1], tk1, u0b); }
                if (lane + 32 < b) { u1 = fma(Ds[(lane + 32) * PS + k], tk, u1); u1b = fma(Ds[(lane + 32) * PS + k + 1], tk1, u1b); }
            }
            if (k < b) {
                const TA tk = __shfl_sync(FULL_MASK, k < 32 ? t0 : t1, k & 31);
                if (lane < b) u0 = fma(Ds[lane * PS + k], tk, u0);
                if (lane + 32 < b) u1 = fma(Ds[(lane + 32) * PS + k], tk, u1);
            }
            u0 += u0b;
            u1 += u1b;
            TA *th = (TA *)a.TUh + (int64_t)slot * b;  // the normalised column, for the sweeps
            if (lane < b) th[lane] = u0;
            if (lane + 32 < b) th[lane + 32] = u1;
            const double nrm2 = warp_sum((double)u0 * (double)u0 + (double)u1 * (double)u1);
            const double tn2 = warp_sum((double)t0 * (double)t0 + (double)t1 * (double)t1);
            if (lane == 0) {
                a.keepU[slot] = sqrt(nrm2) > a.tau ? 1 : 0;
                a.nrmU[slot] = sqrt(tn2);  // norm of the stored (unnormalised) column
            }
            if (a.record) record_sample(a, K, 1, slot, ldcg(a.rowsU + slot), sqrt(nrm2) > a.tau);
        }
    }
}

// ---------------------------------------------------------------- phase E
// Compaction of the kept rows / columns (sorted) into the pools and producer appends.
// Candidate slots are cut into tiles of 32; tile T goes to CTA T % G, one warp per tile.
// A ballot ranks the tile's kept slots; the metadata of all kept slots is handled lane-
// parallel and their rows are copied by one flat loop, so the loads are issued together.
// Every CTA with a tile computes the tile prefix sums itself (no extra barrier).
template <class TS>
__device__ void phase_E(const FactorArgs &a, int K, char *smem) {
    using TA = typename Prec<TS>::TA;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    const int mL = ldcg(a.kst + 0), mU = ldcg(a.kst + 1);
    const int nLc = mL - b;
    const int tL = (nLc + 31) >> 5, tU = a.sym ? tL : (mU + 31) >> 5;  // BILDL: the U side mirrors L
    const int cr = crank(a);
    if (a.sym && cr == 0) {  // BILDL: store D_K = (X + X^T) / 2, as phase D used it
        double *D = a.Dinv + a.Dptr[K];
        for (int e = tid; e < b * b; e += NT) {
            const int r = e / b, c = e - r * b;
            if (c > r) {
                const double v = (ldcg(D + e) + ldcg(D + c * b + r)) * 0.5;
                D[e] = v;
                D[c * b + r] = v;
            }
        }
    }
    // tiles of 32 candidates, L side then U side in one sequence: CTA cr takes tiles cr,
    // cr + G, ... of it, so the two sides' tiles go to different CTAs
    const bool has_work = cr == 0 || cr < tL + tU;
    if (!has_work) return;
    int32_t *cnt = (int32_t *)smem;  // NT tile offsets of the current chunk
    int32_t *ws = cnt + NT;          // scan scratch (40)
    int32_t *sl = ws + 40;           // NW x 32: slot of the r-th kept entry of a warp's tile
    // pool positions of this block: after the previous block (chain schedule) or the bases
    // reserved for it in its group's chunks (tree schedule)
    const int64_t Lbase = ldcg(a.arena ? a.gcur + 8 : a.Lptr + K), LVbase = ldcg(a.arena ? a.gcur + 9 : a.Lvptr + K);
    const int64_t Ubase = ldcg(a.arena ? a.gcur + 10 : a.Uptr + K), UVbase = ldcg(a.arena ? a.gcur + 11 : a.Uvptr + K);
    int keptL, keptU, skipped = 0, bounded = 0;
    {
        // keep flags: 1 kept, 0 dropped by its norm, -1 skipped before its updates (norm bound,
        // classifier: neither scaled nor normed), -2 dropped by the bound of phase D (not scaled)
        int lk = 0, uk = 0, sk = 0, bk = 0;
        for (int s = tid; s < nLc; s += NT) {
            const int k = ldcg(a.keepL + b + s);
            lk += k == 1;
            sk += k == -1;
            bk += k == -2;
        }
        for (int s = tid; s < mU; s += NT) {
            const int k = ldcg(a.keepU + s);
            uk += k == 1;
            sk += k == -1;
            bk += k == -2;
        }
        block_excl_scan(lk, ws, &keptL);
        block_excl_scan(uk, ws, &keptU);
        block_excl_scan(sk, ws, &skipped);
        block_excl_scan(bk, ws, &bounded);
        if (a.sym) keptU = keptL;
    }
    const bool overflow = Lbase + keptL > a.capLrow || LVbase + (int64_t)keptL * b > a.capLval ||
                          Ubase + keptU > a.capUcol || UVbase + (int64_t)keptU * b > a.capUval;
    if (overflow) {
        if (cr == 0 && tid == 0) set_status(a.status, DEV_POOL_OVERFLOW, a.info, K);
        return;
    }
    if (cr == 0 && tid == 0) {
        if (a.arena) {
            a.Lptr[K] = Lbase;
            a.Lend[K] = Lbase + keptL;
            a.Lvptr[K] = LVbase;
            a.Uptr[K] = Ubase;
            a.Uend[K] = Ubase + keptU;
            a.Uvptr[K] = UVbase;
            // the group's cursors move past what the block kept (read again only by this thread)
            a.gcur[0] = Lbase + keptL;
            a.gcur[2] = LVbase + (int64_t)keptL * b;
            a.gcur[4] = Ubase + keptU;
            a.gcur[6] = UVbase + (int64_t)keptU * b;
        } else {
            a.Lptr[K + 1] = Lbase + keptL;
            a.Lvptr[K + 1] = LVbase + (int64_t)keptL * b;
            a.Uptr[K + 1] = Ubase + keptU;
            a.Uvptr[K + 1] = UVbase + (int64_t)keptU * b;
        }
        atomicAdd((unsigned long long *)(a.info + INFO_CAND_ROWS), (unsigned long long)nLc);
        atomicAdd((unsigned long long *)(a.info + INFO_CAND_COLS), (unsigned long long)mU);
        atomicAdd((unsigned long long *)(a.info + INFO_FLOP_SCALE), 2ULL * b * b * (unsigned long long)(nLc + mU - skipped - bounded));
        atomicAdd((unsigned long long *)(a.info + INFO_FLOP_NORM), 2ULL * b * (unsigned long long)(nLc + mU - skipped));
        if (bounded) atomicAdd((unsigned long long *)(a.info + INFO_BOUND_DROPS), (unsigned long long)bounded);
    }
    int32_t *wsl = sl + warp * 32;
    for (int side = 0; side < 2; ++side) {
        const bool isL = side == 0;
        const int ntile = isL ? tL : tU;
        const int gofs = isL ? 0 : tL;                           // sequence index of the side's first tile
        const int tfirst = ((cr - gofs) % a.G + a.G) % a.G;      // this CTA's first tile of the side
        if (tfirst >= ntile) continue;  // uniform in the CTA
        // BILDL: both passes read the L candidates; L takes l_i (in TUh), U-breve t_i (in TL)
        const bool Lc = isL || a.sym;
        const int sfirst = Lc ? b : 0, send = Lc ? mL : mU;
        const int32_t *kp = Lc ? a.keepL : a.keepU;
        const int32_t *rows = Lc ? a.rowsL : a.rowsU;
        const TA *Tb = (const TA *)(isL ? (a.sym ? a.TUh : a.TL) : (a.sym ? a.TL : a.TU));
        TS *pool = (TS *)(isL ? a.Lval : a.Uval) + (isL ? LVbase : UVbase);
        const TA *Th = (const TA *)a.TUh;                        // U side: the normalised columns
        TS *hpool = (TS *)a.Uhval + UVbase;
        int32_t *idxpool = isL ? a.Lrow + Lbase : a.Ucol + Ubase;
        double *nrmpool = isL ? a.Lnrm + Lbase : a.Unrm + Ubase;
        const double *nrmslot = isL ? a.nrmL : a.nrmU;
        int32_t *last = isL ? a.lastU : a.lastL;
        int32_t *pc = isL ? a.prodUcnt : a.prodLcnt;
        int32_t *pl = isL ? a.prodU : a.prodL;
        int carry = 0;
        for (int c0 = 0; c0 < ntile; c0 += NT) {
            const int cn = min(NT, ntile - c0);
            // tile counts: one warp per tile, a ballot over its 32 keep flags
            for (int T = warp; T < cn; T += NW) {
                const int sb = sfirst + (c0 + T) * 32, se = min(send, sb + 32);
                const bool kept = sb + lane < se && ldcg(kp + sb + lane) == 1;
                const unsigned m = __ballot_sync(FULL_MASK, kept);
                if (lane == 0) cnt[T] = __popc(m);
            }
            __syncthreads();
            const int my = tid < cn ? cnt[tid] : 0;
            int tot;
            const int ex = block_excl_scan(my, ws, &tot);
            if (tid < cn) cnt[tid] = carry + ex;
            __syncthreads();
            const int t0c = c0 + (((tfirst - c0) % a.G) + a.G) % a.G;  // first of this CTA's tiles >= c0
            if (t0c < c0 + cn && t0c + a.G >= c0 + cn) {
                // one tile of this CTA in the chunk: warp 0 compacts its indices, every warp
                // copies the kept rows, then warp 0 appends to the producer lists
                const int T = t0c;
                const int sb = sfirst + T * 32, se = min(send, sb + 32);
                const int64_t base = cnt[T - c0];
                bool kept = false;
                int idx = 0;
                if (warp == 0) {
                    kept = sb + lane < se && ldcg(kp + sb + lane) == 1;
                    const unsigned m = __ballot_sync(FULL_MASK, kept);
                    if (kept) {
                        const int rank = __popc(m & ((1u << lane) - 1u));
                        const int slot = sb + lane;
                        wsl[rank] = slot;
                        idx = ldcg(rows + slot);
                        idxpool[base + rank] = idx;
                        nrmpool[base + rank] = ldcg(nrmslot + slot);
                    }
                    if (lane == 0) ws[39] = __popc(m);
                }
                __syncthreads();
                const int tot_e = ws[39] * b;
                const int32_t *wsl0 = sl;  // warp 0's slot list
                for (int e = tid; e < tot_e; e += NT) {
                    const int r = e / b, cc = e - r * b;
                    pool[(base + r) * b + cc] = store_of<TS>((double)ldv(Tb + (int64_t)wsl0[r] * b + cc));
                    if (!isL) hpool[(base + r) * b + cc] = store_of<TS>((double)ldv(Th + (int64_t)wsl0[r] * b + cc));
                }
                if (kept) {
                    const int tb = a.blkof[idx];
                    if (atomicExch(last + tb, K + 1) != K + 1) {
                        const int pos = atomicAdd(pc + tb, 1);
                        if (pos < a.prodcap) pl[(int64_t)tb * a.prodcap + pos] = K;
                        else set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
                    }
                }
            } else
            for (int T = t0c + warp * a.G; T < c0 + cn; T += a.G * NW) {
                const int sb = sfirst + T * 32, se = min(send, sb + 32);
                const bool kept = sb + lane < se && ldcg(kp + sb + lane) == 1;
                const unsigned m = __ballot_sync(FULL_MASK, kept);
                const int nk = __popc(m);
                const int64_t base = cnt[T - c0];
                if (kept) {
                    const int rank = __popc(m & ((1u << lane) - 1u));
                    const int slot = sb + lane;
                    wsl[rank] = slot;
                    const int idx = ldcg(rows + slot);
                    idxpool[base + rank] = idx;
                    nrmpool[base + rank] = ldcg(nrmslot + slot);
                    const int tb = a.blkof[idx];
                    if (atomicExch(last + tb, K + 1) != K + 1) {
                        const int pos = atomicAdd(pc + tb, 1);
                        if (pos < a.prodcap) pl[(int64_t)tb * a.prodcap + pos] = K;
                        else set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
                    }
                }
                __syncwarp();
                // copy the nk kept rows (b values each), four elements in flight per lane
                const int tot_e = nk * b;
                for (int e0 = lane; e0 < tot_e; e0 += 128) {
                    TA v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + u * 32;
                        v[u] = 0;
                        if (e < tot_e) {
                            const int r = e / b, cc = e - r * b;
                            v[u] = ldv(Tb + (int64_t)wsl[r] * b + cc);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + u * 32;
                        if (e < tot_e) pool[(base + e / b) * b + (e % b)] = store_of<TS>((double)v[u]);
                    }
                    if (!isL) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int e = e0 + u * 32;
                            if (e < tot_e) {
                                const int r = e / b, cc = e - r * b;
                                hpool[(base + r) * b + cc] = store_of<TS>((double)ldv(Th + (int64_t)wsl[r] * b + cc));
                            }
                        }
                    }
                }
                __syncwarp();
            }
            carry += tot;
            __syncthreads();
        }
    }
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_add_release(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void trace_at(const FactorArgs &a, int slot, int v) {
    if (a.trace && threadIdx.x == 0) {
        a.trace[8 * blockIdx.x + slot] = v;
        __threadfence_system();
    }
}
__device__ __forceinline__ volatile int32_t *trace_hb(const FactorArgs &a) {
    return a.trace ? a.trace + 8 * blockIdx.x + 4 : nullptr;
}

// Pool space for block K in the tree schedule (CTA 0, thread 0 of the group, after the
// candidate sets are known): the block keeps at most its candidates, so each of the four
// pools must have that much left in the group's current chunk, or the group takes a new chunk
// from the pool's global cursor.  The bases are published to the group's CTAs by the next
// barriers (phase E reads them); a pool that is full reports DEV_POOL_OVERFLOW (the host grows
// the pools and runs the factorization again) and leaves bases at the capacity, so that phase E
// writes nothing.
__device__ void arena_reserve(const FactorArgs &a, int K, int64_t nLc, int64_t mU, int b) {
    const int64_t need[4] = {nLc, nLc * b, mU, mU * b};
    const int64_t chunk[4] = {a.chunkR, a.chunkV, a.chunkR, a.chunkV};
    const int64_t cap[4] = {a.capLrow, a.capLval, a.capUcol, a.capUval};
    for (int q = 0; q < 4; ++q) {
        int64_t cur = a.gcur[2 * q], end = a.gcur[2 * q + 1];
        if (cur + need[q] > end) {
            const int64_t sz = max(chunk[q], need[q]);
            cur = (int64_t)atomicAdd(a.acur + q, (unsigned long long)sz);
            end = cur + sz;
            if (end > cap[q]) {
                set_status(a.status, DEV_POOL_OVERFLOW, a.info, K);
                cur = end = cap[q];
            }
            a.gcur[2 * q] = cur;
            a.gcur[2 * q + 1] = end;
        }
        a.gcur[8 + q] = cur;
    }
}

// CTA 0's phase clock (ns, summed over the blocks it leads): A, B1+C, C2, Bs, D, E; time
// inside the pivot LU; waiting for the pivot-row tiles
struct StepTimers {
    uint64_t acc[6];
    uint64_t tprev, tlu, twait, tidle;
};

// One block step (per block K, five or six barrier phases among the a.G CTAs of the group):
//   A           candidate sets and update plans (CTA 0: L side, CTA 1: U side)
//   B1 + C      pivot-row tiles (two rows each, every producer hits them) on CTAs 1.., then
//               the pivot LU on CTA 0 as soon as those tiles are done, while the remaining
//               update tiles run on the other CTAs (skipped here under the norm-bound skip)
//   C2          D_K = P_K^{-1}
//   Bs          (norm-bound skip only) the remaining update tiles, bound-tested
//   D           scaling, norms, drop decisions
//   E           compaction and producer lists
// Returns false when a barrier reports an error (every CTA of the group returns at the same one).
template <class TS>
__device__ bool block_step(const FactorArgs &a, int K, char *smem, StepTimers &tm) {
    const uint32_t G = a.G + a.debug_extra_cta;
    const int cr = crank(a);
    auto lap = [&](int ph) {
        if (cr == 0 && threadIdx.x == 0) {
            const uint64_t t = gtimer();
            tm.acc[ph] += t - tm.tprev;
            tm.tprev = t;
            if (a.timeline) a.timeline[8 * (int64_t)K + 2 + ph] = (int64_t)t;
        }
    };
    if (a.timeline && cr == 0 && threadIdx.x == 0) {
        a.timeline[8 * (int64_t)K] = (int64_t)(blockIdx.x / a.G) + (a.G == (int)gridDim.x ? 1000 : 0);
        a.timeline[8 * (int64_t)K + 1] = (int64_t)gtimer();
    }
    const int b = a.bstart[K + 1] - a.bstart[K];
    if (cr == 0) phase_A(a, K, true, smem);
    if (cr == (1 % a.G)) {
        __syncthreads();
        if (!a.sym) {
            phase_A(a, K, false, smem);
        } else {  // BILDL: no row block (it is the column block's transpose)
            if (threadIdx.x == 0) {
                a.kst[1] = 0;
                a.kst[3] = 0;
            }
            if (a.sortprod) sort_row_producers(a, K, smem);
        }
    }
    trace_at(a, 2, 1);
    if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 1, trace_hb(a))) return false;
    lap(0);
    // candidate counts of this step (kept within the candidate buffers: phase A reports an
    // overflow and writes safe counts instead of overrunning them)
    const int capT = (int)min(a.capT, (int64_t)INT32_MAX);
    const int mL = max(b, min((int)ldcg(a.kst + 0), capT)), mU = max(0, min((int)ldcg(a.kst + 1), capT));
    const int nrestL = mL - b, nrest = nrestL + mU;
    const int npt = (b + TRP - 1) / TRP;
    if (a.arena && cr == 0 && threadIdx.x == 0) arena_reserve(a, K, nrestL, a.sym ? nrestL : mU, b);
    {
        const int W = a.G > 1 ? a.G - 1 : 1;  // CTAs taking tiles (CTA 0 factors the pivot block)
        const int np = pivot_parts(W, npt);    // producer slices per pivot-row tile
        const bool tc = tc_on<TS>(a);          // update tiles on the tensor cores (up to 128 rows)
        int TR = (nrest + W - 1) / W;
        TR = max(4, min(tc ? TC_ROWS : a.trcap, TR));
        const int nLt = (nrestL + TR - 1) / TR, nUt = (mU + TR - 1) / TR;
        // pivot-row tiles: TRP rows per producer slice, or on the tensor cores all b rows per slice
        const int npiv = tc ? np : npt * np;
        const int ntiles = npiv + (a.skip_bound ? 0 : nLt + nUt);
        if (a.G == 1 || cr > 0) {
            const int wid = a.G > 1 ? cr - 1 : 0;
            for (int it = wid; it < ntiles; it += W) {
                if (it < npiv) {
                    if (tc) {
                        phase_B_tile_tc(a, K, true, 0, b, smem, it, np);
                    } else {
                        const int sa = (it / np) * TRP;
                        phase_B_tile<TS>(a, K, true, sa, min(TRP, b - sa), smem, false, false, it % np, np);
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) red_add_release(a.pivdone, 1u);
                } else {
                    const int r = it - npiv;
                    const bool Ls = r < nLt;
                    const int sa = Ls ? b + r * TR : (r - nLt) * TR;
                    const int cnt = Ls ? min(TR, mL - sa) : min(TR, mU - sa);
                    if (tc) phase_B_tile_tc(a, K, Ls, sa, cnt, smem);
                    else phase_B_tile<TS>(a, K, Ls, sa, cnt, smem, false, a.learned || a.record);
                    __syncthreads();
                }
            }
        }
        if (cr == 0) {
            __shared__ int s_go;
            const uint64_t tw = gtimer();
            trace_at(a, 3, 7);
            if (threadIdx.x == 0) {
                int go = 1;
                if (a.G > 1) {
                    long long itn = 0;
                    while (ld_acquire_u32(a.pivdone) < (uint32_t)(tc_on<TS>(a) ? pivot_parts(a.G - 1, npt)
                                                                               : npt * pivot_parts(a.G - 1, npt))) {
                        if (a.trace && (itn & 1023) == 0) a.trace[8 * blockIdx.x + 6] = (int32_t)(itn >> 10);
                        if (++itn > a.spin_limit) {
                            if (atomicCAS(a.status, 0, DEV_TIMEOUT) == 0) a.info[INFO_TIMEOUT_SITE] = 7;
                            go = 0;
                            break;
                        }
                        if (itn > 64) __nanosleep(32);
                    }
                    atomicExch(a.pivdone, 0u);
                }
                s_go = go;
                tm.twait += gtimer() - tw;
            }
            trace_at(a, 3, 0);
            __syncthreads();
            if (s_go) {
                const uint64_t t0 = gtimer();
                phase_C<TS>(a, K, smem);
                if (threadIdx.x == 0) tm.tlu += gtimer() - t0;
            }
        }
    }
    trace_at(a, 2, 2);
    if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 2, trace_hb(a))) return false;
    lap(1);
    phase_C2(a, K, smem);
    trace_at(a, 2, 3);
    if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 3, trace_hb(a))) return false;
    lap(2);
    if (a.skip_bound) {
        int TR = (nrest + a.G - 1) / a.G;
        TR = max(4, min(a.trcap, TR));
        const int nLt = (nrestL + TR - 1) / TR, nUt = (mU + TR - 1) / TR;
        for (int it = cr; it < nLt + nUt; it += a.G) {
            const bool Ls = it < nLt;
            const int sa = Ls ? b + it * TR : (it - nLt) * TR;
            const int cnt = Ls ? min(TR, mL - sa) : min(TR, mU - sa);
            phase_B_tile<TS>(a, K, Ls, sa, cnt, smem, true);
            __syncthreads();
        }
        trace_at(a, 2, 4);
    if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 4, trace_hb(a))) return false;
    }
    lap(3);
    phase_D<TS>(a, K, smem);
    trace_at(a, 2, 5);
    if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 5, trace_hb(a))) return false;
    lap(4);
    phase_E<TS>(a, K, smem);
    trace_at(a, 2, 6);
    if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 6, trace_hb(a))) return false;
    lap(5);
    return true;
}

// CTA 0's clocks into the info array (added: the tree schedule sums over its groups)
__device__ void store_timers(const FactorArgs &a, const StepTimers &tm) {
    for (int p = 0; p < 6; ++p) atomicAdd((unsigned long long *)(a.info + INFO_PHASE_NS + p), (unsigned long long)tm.acc[p]);
    atomicAdd((unsigned long long *)(a.info + INFO_C2_WORK_NS), (unsigned long long)tm.tlu);
    atomicAdd((unsigned long long *)(a.info + INFO_B_WORK_NS), (unsigned long long)tm.twait);
    atomicAdd((unsigned long long *)(a.info + INFO_IDLE_NS), (unsigned long long)tm.tidle);
}

// The blocks K = 0..nb-1 one after another, each by the whole group.
template <class TS>
__device__ void factor_chain(const FactorArgs &a, char *smem) {
    StepTimers tm{};
    tm.tprev = gtimer();
    for (int K = 0; K < a.nb; ++K)
        if (!block_step<TS>(a, K, smem, tm)) return;
    if (crank(a) == 0 && threadIdx.x == 0) store_timers(a, tm);
}

template <class TS>
__global__ void __launch_bounds__(NT, 1) bilu_factor_kernel(FactorArgs a) {
    extern __shared__ __align__(16) char smem[];
    const bool tc = tc_on<TS>(a);
    tc_begin<TS>(tc);
    factor_chain<TS>(a, smem);
    tc_end<TS>(tc);
}

// Batch of independent matrices in one launch: the grid is cut into groups of G CTAs, each
// group takes the next matrix from a work queue (sorted largest first by the host), runs its
// block chain with the group's own barrier, and repeats until the queue is empty.
template <class TS>
__device__ void factor_batch_body(const FactorArgs *all, int nmat, int *queue,
                                                                  uint32_t *gbar, uint32_t *gpiv, int32_t *gslot,
                                                                  int32_t *gstat, int64_t *ginfo, int G,
                                                                  long long spin) {
    extern __shared__ __align__(16) char smem[];
    __shared__ FactorArgs s_a;
    __shared__ int s_m;
    const int grp = blockIdx.x / G, cr = blockIdx.x % G;
    uint32_t *bar = gbar + 4 * grp;
    int taken = nmat;  // CTA 0, thread 0: the matrix this group took last
    while (true) {
        if (cr == 0 && threadIdx.x == 0) {
            taken = atomicAdd(queue, 1);
            st_release_s32(gslot + grp, taken);
        }
        if (!grid_barrier(bar, (uint32_t)G, gstat + grp, spin, ginfo + grp * INFO_COUNT, 8)) {
            // the group is stuck: the matrix it took is reported as timed out, not as factored
            if (cr == 0 && threadIdx.x == 0 && taken < nmat) atomicCAS(all[taken].status, 0, DEV_TIMEOUT);
            return;
        }
        if (threadIdx.x == 0) s_m = ld_acquire_s32(gslot + grp);
        __syncthreads();
        const int m = s_m;
        if (m >= nmat) return;
        if (threadIdx.x == 0) {
            s_a = all[m];
            s_a.G = G;
            s_a.bar = bar;
            s_a.pivdone = gpiv + grp;
            s_a.spin_limit = spin;
        }
        __syncthreads();
        factor_chain<TS>(s_a, smem);
        __syncthreads();
        // other errors end the chain at the same barrier on every CTA of the group, and the
        // group goes on with the next matrix; after a timeout its barrier state is undefined
        if (threadIdx.x == 0) s_m = ld_acquire_s32(s_a.status);
        __syncthreads();
        if (s_m == DEV_TIMEOUT) {
            if (threadIdx.x == 0) atomicCAS(gstat + grp, 0, DEV_TIMEOUT);
            return;
        }
    }
}

template <class TS>
__global__ void __launch_bounds__(NT, 1) bilu_factor_batch_kernel(const FactorArgs *all, int nmat, int *queue,
                                                                  uint32_t *gbar, uint32_t *gpiv, int32_t *gslot,
                                                                  int32_t *gstat, int64_t *ginfo, int G,
                                                                  long long spin) {
    const bool tc = tc_on<TS>(all[0]);
    tc_begin<TS>(tc);
    factor_batch_body<TS>(all, nmat, queue, gbar, gpiv, gslot, gstat, ginfo, G, spin);
    tc_end<TS>(tc);
}

// ---------------------------------------------------------------- tree schedule
// Every block J that updates block K is a descendant of K in the block elimination tree
// (Sec. 3.3 reorders so that this tree has independent subtrees), so K can be factored as soon
// as its children are.  The grid is cut into groups of G CTAs; CTA 0 of a group takes the next
// entry of a queue of ready blocks (the leaves first, then every block whose last child has
// finished, in the order they become ready), the group runs block_step on it, and CTA 0
// counts the block off at its parent.  The chain of single-child blocks at the top of the tree
// (the trunk) runs afterwards on the whole grid.  Each block sees the same inputs and
// producer order (sorted) as in the chain schedule, so the factor is the same bit for bit.
struct TreeArgs {
    int32_t nb, split, ngroups, G, extra;
    const int32_t *parent;
    int32_t *pending;            // children of each block not finished yet
    int32_t *queue;              // ready blocks, -1 until filled
    int32_t *tctl;               // [0] queue head, [1] queue tail, [2 + g] block of group g
    uint32_t *fullbar;           // whole-grid barrier
};

__device__ __forceinline__ int32_t atom_add_acqrel_s32(int32_t *p, int32_t v) {
    int32_t old;
    asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <class TS>
__device__ void factor_tree_body(const FactorArgs *gargs, TreeArgs t) {
    extern __shared__ __align__(16) char smem[];
    __shared__ FactorArgs s_a;
    __shared__ int s_K;
    const int grp = blockIdx.x / t.G;
    StepTimers tm{};
    tm.tprev = gtimer();
    // mode 0: a CTA of group grp takes ready blocks; 1: the groups are done, the grid meets;
    // 2: the trunk on the whole grid (one block_step call site for all of them)
    int mode = grp < t.ngroups ? 0 : 1;
    // the CTAs past the last whole group (when G does not divide the grid) join only the trunk;
    // they hold group 0's arguments until then, so that every field they read is defined
    if (threadIdx.x == 0) s_a = gargs[mode == 0 ? grp : 0];
    __syncthreads();
    int Kt = t.split;
    while (true) {
        int K = -1;
        trace_at(s_a, 0, mode);
        if (mode == 0) {
            trace_at(s_a, 3, 8);
            if (crank(s_a) == 0 && threadIdx.x == 0) {
                // the next ready block; slots past the last block end the group's work.  The
                // block reaches the group's CTAs (this thread included) only through the slot
                // word after the barrier, so that a failed barrier leaves every thread at -1.
                const uint64_t t0 = gtimer();
                int Kp = -1;
                const int slot = atomicAdd(t.tctl, 1);
                if (slot < t.split) {
                    long long it = 0;
                    while ((Kp = ld_acquire_s32(t.queue + slot)) < 0) {
                        if (++it > s_a.spin_limit) {
                            if (atomicCAS(s_a.status, 0, DEV_TIMEOUT) == 0) s_a.info[INFO_TIMEOUT_SITE] = 9;
                            break;
                        }
                        if ((it & 63) == 0 && ld_acquire_s32(s_a.status) != DEV_OK) break;  // another group failed
                        if (s_a.trace && (it & 1023) == 0) s_a.trace[8 * blockIdx.x + 5] = (int32_t)(it >> 10);
                        if (it > 64) __nanosleep(64);
                    }
                }
                st_release_s32(t.tctl + 2 + grp, Kp);
                tm.tidle += gtimer() - t0;
            }
            trace_at(s_a, 3, 0);
            trace_at(s_a, 2, 8);
            if (grid_barrier(s_a.bar, s_a.G + s_a.debug_extra_cta, s_a.status, s_a.spin_limit, s_a.info, 8, trace_hb(s_a))) {
                if (threadIdx.x == 0) {
                    s_K = ld_acquire_s32(t.tctl + 2 + grp);
                    tm.tprev = gtimer();
                }
                __syncthreads();
                K = s_K;
                __syncthreads();
            }
            if (K < 0 || K >= t.split) mode = 1;
        }
        if (mode == 1) {
            if (grp < t.ngroups && crank(s_a) == 0 && threadIdx.x == 0) store_timers(s_a, tm);
            const FactorArgs &a0 = gargs[0];
            trace_at(s_a, 0, 1);
            trace_at(s_a, 2, 10);
            if (!grid_barrier(t.fullbar, gridDim.x + t.extra, a0.status, a0.spin_limit, a0.info, 10, trace_hb(s_a))) {
                trace_at(s_a, 0, 9);
                return;
            }
            if (t.split >= t.nb) {
                trace_at(s_a, 0, 9);
                return;
            }
            if (threadIdx.x == 0) {
                s_a = a0;
                s_a.G = gridDim.x;
                s_a.bar = t.fullbar;
            }
            __syncthreads();
            tm = StepTimers{};
            tm.tprev = gtimer();
            mode = 2;
        }
        if (mode == 2) {
            if (Kt >= t.nb) {
                if (blockIdx.x == 0 && threadIdx.x == 0) store_timers(s_a, tm);
                trace_at(s_a, 0, 9);
                return;
            }
            K = Kt++;
        }
        trace_at(s_a, 1, K);
        const bool ok = block_step<TS>(s_a, K, smem, tm);
        if (mode == 2) {
            if (!ok) {
                trace_at(s_a, 0, 9);
                return;
            }
            continue;
        }
        if (!ok) {  // every CTA of the group leaves at the same barrier; the grid meets
            mode = 1;
            continue;
        }
        if (crank(s_a) == 0 && threadIdx.x == 0) {
            // the block is complete (the barrier at the end of its step): count it off at its
            // parent, which is queued when this was its last unfinished child
            const int p = t.parent[K];
            if (p >= 0 && p < t.split && atom_add_acqrel_s32(t.pending + p, -1) == 1) {
                const int pos = atomicAdd(t.tctl + 1, 1);
                st_release_s32(t.queue + pos, p);
            }
        }
    }
}

template <class TS>
__global__ void __launch_bounds__(NT, 1) bilu_factor_tree_kernel(const FactorArgs *gargs, TreeArgs t) {
    const bool tc = tc_on<TS>(gargs[0]);
    tc_begin<TS>(tc);
    factor_tree_body<TS>(gargs, t);
    tc_end<TS>(tc);
}

// Closing copy of the tree schedule, part 1 (one CTA): block-ordered offsets of the kept rows
// and columns and of their values, the exclusive prefix sums of the blocks' counts.
__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long *ws, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const long long x = lane < nw ? ws[lane] : 0;
        long long xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(FULL_MASK, xi, o);
            if (lane >= o) xi += u;
        }
        if (lane < nw) ws[lane] = xi - x;
        if (lane == nw - 1) ws[32] = xi;
    }
    __syncthreads();
    const long long res = inc - v + ws[warp];
    *total = ws[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(1024) tree_offsets_kernel(int nb, const int32_t *bstart, const int64_t *aptr,
                                                            int64_t *Lptr, int64_t *Lvptr, int64_t *Uptr,
                                                            int64_t *Uvptr, int64_t cap0, int64_t cap1, int64_t cap2,
                                                            int64_t cap3, int32_t *status) {
    __shared__ long long ws[33];
    if (*status != DEV_OK) return;
    long long carry[4] = {0, 0, 0, 0};
    int64_t *out[4] = {Lptr, Lvptr, Uptr, Uvptr};
    for (int c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int K = c0 + threadIdx.x;
        long long v[4] = {0, 0, 0, 0};
        if (K < nb) {
            const long long bK = bstart[K + 1] - bstart[K];
            v[0] = aptr[(int64_t)nb + K] - aptr[K];
            v[1] = v[0] * bK;
            v[2] = aptr[4 * (int64_t)nb + K] - aptr[3 * (int64_t)nb + K];
            v[3] = v[2] * bK;
        }
        for (int q = 0; q < 4; ++q) {
            long long tot;
            const long long ex = block_excl_scan_ll(v[q], ws, &tot);
            if (K < nb) out[q][K] = carry[q] + ex;
            carry[q] += tot;
        }
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) out[q][nb] = carry[q];
        // the block-ordered pools must hold every kept entry (else grow them and run again)
        if (carry[0] > cap0 || carry[1] > cap1 || carry[2] > cap2 || carry[3] > cap3) *status = DEV_POOL_OVERFLOW;
    }
}

// Part 2: every block's kept row indices and values (and column indices and values) from its
// chunk positions to the block-ordered pools that the apply sweeps and bilu_export read.
template <class TS>
__global__ void __launch_bounds__(256) tree_copy_kernel(int nb, const int32_t *bstart, const int64_t *aptr,
                                                        const int64_t *Lptr, const int64_t *Lvptr, const int64_t *Uptr,
                                                        const int64_t *Uvptr, const int32_t *aLrow, const int32_t *aUcol,
                                                        const TS *aLval, const TS *aUval, const TS *aUhval, int32_t *Lrow,
                                                        int32_t *Ucol, TS *Lval, TS *Uval, TS *Uhval,
                                                        const int32_t *status) {
    if (*status != DEV_OK) return;
    for (int K = blockIdx.x; K < nb; K += gridDim.x) {
        const int64_t bK = bstart[K + 1] - bstart[K];
        const int64_t cL = aptr[(int64_t)nb + K] - aptr[K], cU = aptr[4 * (int64_t)nb + K] - aptr[3 * (int64_t)nb + K];
        const int32_t *sLr = aLrow + aptr[K], *sUc = aUcol + aptr[3 * (int64_t)nb + K];
        const TS *sLv = aLval + aptr[2 * (int64_t)nb + K], *sUv = aUval + aptr[5 * (int64_t)nb + K];
        int32_t *dLr = Lrow + Lptr[K], *dUc = Ucol + Uptr[K];
        TS *dLv = Lval + Lvptr[K], *dUv = Uval + Uvptr[K], *dUh = Uhval + Uvptr[K];
        const TS *sUh = aUhval + aptr[5 * (int64_t)nb + K];
        for (int64_t e = threadIdx.x; e < cL; e += blockDim.x) dLr[e] = sLr[e];
        for (int64_t e = threadIdx.x; e < cU; e += blockDim.x) dUc[e] = sUc[e];
        for (int64_t e = threadIdx.x; e < cL * bK; e += blockDim.x) dLv[e] = sLv[e];
        for (int64_t e = threadIdx.x; e < cU * bK; e += blockDim.x) {
            dUv[e] = sUv[e];
            dUh[e] = sUh[e];
        }
    }
}

// Self-test of recip_nr against the IEEE quotient 1.0 / p on n values spread over many
// binades (test hook).  out[0] = number of results more than one ulp away.
__global__ void recip_selftest_kernel(int n, unsigned long long seed, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long h = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ULL; h ^= h >> 29;
        const double mant = 1.0 + (double)(h & ((1ULL << 52) - 1)) / 4503599627370496.0;
        const int e = (int)((h >> 52) % 200) - 100;
        const double p = ((h >> 63) ? -1.0 : 1.0) * ldexp(mant, e);
        const double r = recip_nr(p), q = 1.0 / p;
        const long long d = __double_as_longlong(r) - __double_as_longlong(q);
        if (d > 1 || d < -1) atomicAdd(out, 1);
    }
}

}  // namespace

int recip_selftest(int n) {
    int *d = nullptr, h = -1;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return -1;
    cudaMemset(d, 0, sizeof(int));
    recip_selftest_kernel<<<128, 256>>>(n, 12345ULL, d);
    cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return cudaGetLastError() == cudaSuccess ? h : -1;
}

// ---------------------------------------------------------------- host side

void factor_free(bilu_ctx *c) {
    aggregate_free(c);
    dev_free(c->d_Lptr); dev_free(c->d_Lvptr); dev_free(c->d_Uptr); dev_free(c->d_Uvptr);
    dev_free(c->d_Lrow); dev_free(c->d_Ucol); dev_free(c->d_Lval); dev_free(c->d_Uval); dev_free(c->d_Uhval);
    dev_free(c->d_Dinv); dev_free(c->d_Pblk);
    dev_free(c->d_prodL); dev_free(c->d_prodLcnt); dev_free(c->d_prodU); dev_free(c->d_prodUcnt);
    dev_free(c->d_lastL); dev_free(c->d_lastU);
    dev_free(c->d_TL); dev_free(c->d_TU); dev_free(c->d_TUh); dev_free(c->d_TLP); dev_free(c->d_rowsL); dev_free(c->d_rowsU);
    dev_free(c->d_keepL); dev_free(c->d_keepU); dev_free(c->d_bmL); dev_free(c->d_bmU);
    dev_free(c->d_LU); dev_free(c->d_perm); dev_free(c->d_kstate); dev_free(c->d_status);
    dev_free(c->d_info); dev_free(c->d_bar);
    dev_free(c->d_wbL); dev_free(c->d_wbU); dev_free(c->d_xslotL); dev_free(c->d_xslotU);
    dev_free(c->d_pinfoL); dev_free(c->d_pinfoU);
    dev_free(c->d_Lnrm); dev_free(c->d_Unrm); dev_free(c->d_nrmL); dev_free(c->d_nrmU);
    dev_free(c->d_dcolsq); dev_free(c->d_pivdone);
    c->capLrow = c->capLval = c->capUcol = c->capUval = 0;
    dev_free(c->d_grp_big); dev_free(c->d_grp_reset);
    c->grp_n = 0;
    c->grp_big_bytes = c->grp_reset_bytes = 0;
    dev_free(c->d_aLrow); dev_free(c->d_aUcol); dev_free(c->d_aLval); dev_free(c->d_aUval); dev_free(c->d_aUhval);
    dev_free(c->d_aLnrm); dev_free(c->d_aUnrm); dev_free(c->d_aptr);
    for (auto &v : c->capA) v = 0;
}

namespace {

cudaError_t alloc_pools(bilu_ctx *c) {
    cudaError_t e;
    dev_free(c->d_Lrow); dev_free(c->d_Ucol); dev_free(c->d_Lval); dev_free(c->d_Uval); dev_free(c->d_Uhval);
    dev_free(c->d_Lnrm); dev_free(c->d_Unrm);
    if ((e = dev_alloc(&c->d_Lnrm, c->capLrow)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Unrm, c->capUcol)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Lrow, c->capLrow)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Ucol, c->capUcol)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Lval, c->capLval)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Uval, c->capUval)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Uhval, c->capUval)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t alloc_prod(bilu_ctx *c) {
    cudaError_t e;
    dev_free(c->d_prodL); dev_free(c->d_prodU); dev_free(c->d_xslotL); dev_free(c->d_xslotU);
    dev_free(c->d_pinfoL); dev_free(c->d_pinfoU);
    const int64_t nb = std::max<int64_t>(c->nb, 1);
    if ((e = dev_alloc(&c->d_prodL, nb * c->prodcap)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_prodU, nb * c->prodcap)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_pinfoL, (int64_t)PIS * c->prodcap)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_pinfoU, (int64_t)PIS * c->prodcap)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_xslotL, c->capXS)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_xslotU, c->capXS)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace

// test hooks (bilu_debug_set)
int g_debug_extra_cta = 0;          // the barrier waits for a CTA that never arrives
long long g_debug_spin_limit = 0;   // polls before a bounded wait gives up (0: default)
long long g_debug_batch_group = 0;  // batch group size (0: tuned)
long long g_debug_batch_trcap = 0;  // batch tile row cap (0: tuned)
int g_debug_tc_off = 0;             // BF16 update tiles on the FP32 units instead of the tensor cores
int g_debug_small_pools = 0;        // factorizations start from minimal pools and producer lists
int g_debug_poison = 0;             // factor storage is filled with NaN before every run
int g_debug_no_trunk = 0;           // the tree schedule leaves no trunk to the whole grid
int g_debug_trace = 0;              // the tree schedule prints one line per run to stderr

static void hint_key_of(const bilu_ctx *c, int64_t key[5]) {
    key[0] = c->n;
    key[1] = c->nnz;
    key[2] = c->nb;
    key[3] = c->p.precision;
    key[4] = c->p.symmetric;
}

static bool hint_matches(const bilu_ctx *c) {
    int64_t key[5];
    hint_key_of(c, key);
    for (int q = 0; q < 5; ++q)
        if (key[q] != c->hint_key[q]) return false;
    return true;
}

void factor_remember_pools(bilu_ctx *c) {
    hint_key_of(c, c->hint_key);
    const int64_t caps[8] = {c->capLrow, c->capLval, c->capUcol, c->capUval, c->capA[0], c->capA[1], c->capA[2], c->capA[3]};
    for (int q = 0; q < 8; ++q) c->hint_cap[q] = caps[q];
    c->hint_prodcap = c->prodcap;
}

bilu_status factor_alloc(bilu_ctx *c) {
    factor_free(c);
    const int64_t n = std::max<int64_t>(c->n, 1), nb = std::max<int64_t>(c->nb, 1);
    const int64_t nd = std::max<int64_t>(c->h_Dptr.back(), 1);
    const int bmax = std::max(c->bmax, 1), bmin = std::max(c->bmin, 1);
    // initial pools: up to 4 kept rows (and columns) per matrix row and block column width
    c->capLval = c->capUval = std::max<int64_t>(4 * n * bmax, 1024);
    c->capLrow = c->capUcol = std::max<int64_t>(c->capLval / bmin, 1024);
    c->capT = n + BILU_MAX_BLOCK;
    c->prodcap = 64;
    c->capXS = 4 * c->capT;
    if (hint_matches(c)) {  // the capacities the same kind of factorization ended with
        c->capLrow = std::max(c->capLrow, c->hint_cap[0]);
        c->capLval = std::max(c->capLval, c->hint_cap[1]);
        c->capUcol = std::max(c->capUcol, c->hint_cap[2]);
        c->capUval = std::max(c->capUval, c->hint_cap[3]);
        c->prodcap = std::max(c->prodcap, c->hint_prodcap);
        c->capXS = std::max<int64_t>(c->capXS, (int64_t)c->capT * (c->prodcap / 16));
    }
    if (g_debug_small_pools) {  // test hook: exercise the re-run paths
        c->capLval = c->capUval = c->capLrow = c->capUcol = 1024;
        c->prodcap = 4;
        c->capXS = c->capT;
    }
    cudaError_t e = cudaSuccess;
    if ((e = dev_alloc(&c->d_Lptr, nb + 1)) != cudaSuccess || (e = dev_alloc(&c->d_Lvptr, nb + 1)) != cudaSuccess ||
        (e = dev_alloc(&c->d_Uptr, nb + 1)) != cudaSuccess || (e = dev_alloc(&c->d_Uvptr, nb + 1)) != cudaSuccess ||
        (e = dev_alloc(&c->d_Dinv, nd)) != cudaSuccess || (e = dev_alloc(&c->d_Pblk, nd)) != cudaSuccess ||
        (e = dev_alloc(&c->d_prodLcnt, nb)) != cudaSuccess || (e = dev_alloc(&c->d_prodUcnt, nb)) != cudaSuccess ||
        (e = dev_alloc(&c->d_lastL, nb)) != cudaSuccess || (e = dev_alloc(&c->d_lastU, nb)) != cudaSuccess ||
        (e = dev_alloc(&c->d_TL, c->capT * bmax)) != cudaSuccess ||
        (e = dev_alloc(&c->d_TU, c->capT * bmax)) != cudaSuccess ||
        (e = dev_alloc(&c->d_TUh, c->capT * bmax)) != cudaSuccess ||
        (e = dev_alloc(&c->d_TLP, (int64_t)PPART * BILU_MAX_BLOCK * BILU_MAX_BLOCK)) != cudaSuccess ||
        (e = dev_alloc(&c->d_rowsL, c->capT)) != cudaSuccess || (e = dev_alloc(&c->d_rowsU, c->capT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_keepL, c->capT)) != cudaSuccess || (e = dev_alloc(&c->d_keepU, c->capT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_bmL, n / 32 + 2)) != cudaSuccess || (e = dev_alloc(&c->d_bmU, n / 32 + 2)) != cudaSuccess ||
        (e = dev_alloc(&c->d_wbL, n / 32 + 2)) != cudaSuccess || (e = dev_alloc(&c->d_wbU, n / 32 + 2)) != cudaSuccess ||
        (e = dev_alloc(&c->d_LU, BILU_MAX_BLOCK * BILU_MAX_BLOCK + BILU_MAX_BLOCK)) != cudaSuccess ||
        (e = dev_alloc(&c->d_perm, BILU_MAX_BLOCK)) != cudaSuccess || (e = dev_alloc(&c->d_kstate, 16)) != cudaSuccess ||
        (e = dev_alloc(&c->d_status, 4)) != cudaSuccess || (e = dev_alloc(&c->d_info, INFO_COUNT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_bar, 4)) != cudaSuccess || (e = dev_alloc(&c->d_nrmL, c->capT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_nrmU, c->capT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_dcolsq, BILU_MAX_BLOCK)) != cudaSuccess ||
        (e = dev_alloc(&c->d_pivdone, 4)) != cudaSuccess || (e = alloc_pools(c)) != cudaSuccess ||
        (e = alloc_prod(c)) != cudaSuccess) {
        factor_free(c);
        return e == cudaErrorMemoryAllocation ? set_err(c, BILU_ERR_OOM, "device allocation failed in factor")
                                              : cuda_err(c, e, "factor allocation");
    }
    return BILU_OK;
}


namespace {

const void *factor_kernel_for(int precision) {
    return precision == BILU_PREC_FP32   ? (const void *)bilu_factor_kernel<float>
           : precision == BILU_PREC_BF16 ? (const void *)bilu_factor_kernel<__nv_bfloat16>
                                         : (const void *)bilu_factor_kernel<double>;
}
const void *batch_kernel_for(int precision) {
    return precision == BILU_PREC_FP32   ? (const void *)bilu_factor_batch_kernel<float>
           : precision == BILU_PREC_BF16 ? (const void *)bilu_factor_batch_kernel<__nv_bfloat16>
                                         : (const void *)bilu_factor_batch_kernel<double>;
}

// Reset of the per-run device state of one context (stream-ordered on `st`).
cudaError_t prepare_run(bilu_ctx *c, cudaStream_t st) {
    const int64_t nb = std::max<int64_t>(c->nb, 1), n = std::max<int64_t>(c->n, 1);
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_Lptr, 0, (nb + 1) * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_Lvptr, 0, (nb + 1) * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_Uptr, 0, (nb + 1) * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_Uvptr, 0, (nb + 1) * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_prodLcnt, 0, nb * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_prodUcnt, 0, nb * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_lastL, 0, nb * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_lastU, 0, nb * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_bmL, 0, (n / 32 + 2) * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_bmU, 0, (n / 32 + 2) * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_info, 0, INFO_COUNT * sizeof(int64_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_bar, 0, 4 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if (g_debug_poison) {  // test hook: every value array (no index array) starts as NaN
        const int64_t nd = std::max<int64_t>(c->h_Dptr.back(), 1);
        const size_t vs = c->p.precision == BILU_PREC_FP64 ? 8 : c->p.precision == BILU_PREC_FP32 ? 4 : 2;
        const size_t as = c->p.precision == BILU_PREC_FP64 ? 8 : 4;
        const size_t tb = (size_t)c->capT * (size_t)std::max(c->bmax, 1) * as;
        struct { void *p; size_t bytes; } fill[] = {
            {c->d_Dinv, (size_t)nd * 8}, {c->d_Pblk, (size_t)nd * 8}, {c->d_Lval, (size_t)c->capLval * vs},
            {c->d_Uval, (size_t)c->capUval * vs}, {c->d_Uhval, (size_t)c->capUval * vs},
            {c->d_Lnrm, (size_t)c->capLrow * 8},
            {c->d_Unrm, (size_t)c->capUcol * 8}, {c->d_TL, tb}, {c->d_TU, tb},
            {c->d_LU, (size_t)(BILU_MAX_BLOCK * BILU_MAX_BLOCK + BILU_MAX_BLOCK) * 8},
            {c->d_dcolsq, (size_t)BILU_MAX_BLOCK * 8}, {c->d_nrmL, (size_t)c->capT * 8}, {c->d_nrmU, (size_t)c->capT * 8}};
        for (auto &f : fill)
            if ((e = cudaMemsetAsync(f.p, 0xff, f.bytes, st)) != cudaSuccess) return e;
    }
    if (c->rec_cap > 0) {  // recording: per-slot feature rows, the sample count of this run's start
        if (c->feat_cap < c->capT) {
            dev_free(c->d_featL);
            dev_free(c->d_featU);
            c->feat_cap = 0;
            if ((e = dev_alloc(&c->d_featL, c->capT * MF)) != cudaSuccess) return e;
            if ((e = dev_alloc(&c->d_featU, c->capT * MF)) != cudaSuccess) return e;
            c->feat_cap = c->capT;
        }
        if ((e = cudaMemcpyAsync(c->d_rec_count, &c->rec_base, sizeof(unsigned long long), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return e;
    }
    return cudaMemsetAsync(c->d_pivdone, 0, 4 * sizeof(uint32_t), st);
}

FactorArgs make_args(bilu_ctx *c, double droptol, int G) {
    FactorArgs a{};
    a.n = (int32_t)c->n; a.nb = c->nb; a.G = G; a.perturb = c->p.perturb;
    a.tau = droptol; a.alpha = c->alpha; a.pert_tau = c->p.pert_tau; a.pert_rho = c->p.pert_rho;
    a.spin_limit = g_debug_spin_limit > 0 ? g_debug_spin_limit : (1LL << 24);
    a.rowptr = c->d_rowptr; a.colind = c->d_colind; a.colptr = c->d_colptr; a.rowind = c->d_rowind;
    a.bstart = c->d_bstart; a.blkof = c->d_blkof; a.val = c->d_val; a.cval = c->d_cval; a.Dptr = c->d_Dptr;
    a.Lptr = c->d_Lptr; a.Lvptr = c->d_Lvptr; a.Uptr = c->d_Uptr; a.Uvptr = c->d_Uvptr;
    a.Lrow = c->d_Lrow; a.Ucol = c->d_Ucol; a.Lval = c->d_Lval; a.Uval = c->d_Uval; a.Uhval = c->d_Uhval;
    a.Dinv = c->d_Dinv; a.Pblk = c->d_Pblk;
    a.capLrow = c->capLrow; a.capLval = c->capLval; a.capUcol = c->capUcol; a.capUval = c->capUval;
    a.prodcap = c->prodcap;
    a.prodL = c->d_prodL; a.prodLcnt = c->d_prodLcnt; a.prodU = c->d_prodU; a.prodUcnt = c->d_prodUcnt;
    a.lastL = c->d_lastL; a.lastU = c->d_lastU;
    a.TL = c->d_TL; a.TU = c->d_TU; a.TUh = c->d_TUh; a.TLP = c->d_TLP; a.rowsL = c->d_rowsL; a.rowsU = c->d_rowsU;
    a.keepL = c->d_keepL; a.keepU = c->d_keepU; a.bmL = c->d_bmL; a.bmU = c->d_bmU;
    a.wbL = c->d_wbL; a.wbU = c->d_wbU; a.xslotL = c->d_xslotL; a.xslotU = c->d_xslotU;
    a.capXS = c->capXS; a.pinfoL = c->d_pinfoL; a.pinfoU = c->d_pinfoU; a.capT = c->capT;
    a.LU = c->d_LU; a.perm = c->d_perm; a.kst = c->d_kstate; a.status = c->d_status; a.info = c->d_info;
    a.bar = c->d_bar;
    a.debug_extra_cta = g_debug_extra_cta;
    a.trace = nullptr;
    a.timeline = nullptr;
    a.trcap = TRMAX;
    // recording takes exact samples: no skipping while it is on
    const bool rec = c->rec_cap > 0;
    a.skip_bound = c->p.skip == BILU_SKIP_BOUND && !rec ? 1 : 0;
    a.sym = c->p.symmetric ? 1 : 0;
    a.learned = c->p.skip == BILU_SKIP_LEARNED && !rec && c->d_mlp_w ? 1 : 0;
    a.zhi = (float)c->mlp_logit_hi;
    a.mlp_norm = c->d_mlp_norm;
    a.mlp_w = (const __half *)c->d_mlp_w;
    a.record = rec ? 1 : 0;
    a.rec_thresh = c->rec_thresh;
    // the plain BF16 updates run on the tensor cores (the skip modes and recording keep their
    // per-row tiles on the FP32 units)
    a.tc = c->p.precision == BILU_PREC_BF16 && !a.skip_bound && !a.learned && !rec && !g_debug_tc_off ? 1 : 0;
    a.rec_seed = c->rec_seed;
    a.rec_cap = c->rec_cap;
    a.featL = c->d_featL;
    a.featU = c->d_featU;
    a.rec_x = c->d_rec_x;
    a.rec_y = c->d_rec_y;
    a.rec_tag = (long long *)c->d_rec_tag;
    a.rec_count = c->d_rec_count;
    a.Lnrm = c->d_Lnrm; a.Unrm = c->d_Unrm; a.nrmL = c->d_nrmL; a.nrmU = c->d_nrmU;
    a.dcolsq = c->d_dcolsq; a.pivdone = c->d_pivdone;
    a.Lend = c->d_Lptr + 1;  // chain schedule: block K ends where block K + 1 starts
    a.Uend = c->d_Uptr + 1;
    a.arena = 0;
    a.sortprod = 0;
    return a;
}

// After a run: 0 = done, 1 = re-run (pools or producer lists were grown), < 0 = error status.
int finish_run(bilu_ctx *c, int32_t status, const int64_t *info, bilu_status *err) {
    if (status == DEV_POOL_OVERFLOW) {
        c->capLval *= 2; c->capUval *= 2; c->capLrow *= 2; c->capUcol *= 2;
        if (alloc_pools(c) != cudaSuccess) { *err = set_err(c, BILU_ERR_OOM, "growing L/U pools failed"); return -1; }
        c->pool_retries++;
        return 1;
    }
    if (status == DEV_PROD_OVERFLOW) {
        if (c->prodcap * 2 > PMAX) { *err = set_err(c, BILU_ERR_OOM, "more than 1024 producer blocks for one block"); return -1; }
        c->prodcap *= 2;
        c->capXS *= 2;
        if (alloc_prod(c) != cudaSuccess) { *err = set_err(c, BILU_ERR_OOM, "growing producer lists failed"); return -1; }
        c->pool_retries++;
        return 1;
    }
    if (status == DEV_TIMEOUT) { *err = set_err(c, BILU_ERR_TIMEOUT, "factor kernel: bounded wait gave up (site " + std::to_string(info[INFO_TIMEOUT_SITE]) + ")"); return -1; }
    if (status == DEV_SINGULAR) { *err = set_err(c, BILU_ERR_SINGULAR, "singular diagonal block " + std::to_string(info[INFO_FAIL_BLOCK])); return -1; }
    if (status == DEV_INTERNAL) { *err = set_err(c, BILU_ERR_CUDA, "factor kernel index check failed at block " + std::to_string(info[INFO_FAIL_BLOCK])); return -1; }
    if (status != DEV_OK) { *err = set_err(c, BILU_ERR_CUDA, "factor kernel status " + std::to_string(status)); return -1; }
    int64_t tails[4] = {0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    if (c->nb > 0) {
        if ((e = cudaMemcpy(&tails[0], c->d_Lptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&tails[1], c->d_Lvptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&tails[2], c->d_Uptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&tails[3], c->d_Uvptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            *err = cuda_err(c, e, "reading factor sizes");
            return -1;
        }
    }
    c->kept_rows = tails[0]; c->nnz_l = tails[1]; c->kept_cols = tails[2]; c->nnz_u = tails[3];
    c->cand_rows = info[INFO_CAND_ROWS]; c->cand_cols = info[INFO_CAND_COLS];
    c->nperturb = info[INFO_NPERTURB];
    c->flop_upd_l = info[INFO_FLOP_UPD_L];
    c->flop_upd_u = info[INFO_FLOP_UPD_U];
    c->flop_scale = info[INFO_FLOP_SCALE];
    c->flop_norm = info[INFO_FLOP_NORM];
    for (int p = 0; p < 6; ++p) c->phase_ms[p] = info[INFO_PHASE_NS + p] * 1e-6;
    c->phase_ms[6] = info[INFO_C2_WORK_NS] * 1e-6;
    c->phase_ms[7] = info[INFO_B_WORK_NS] * 1e-6;
    c->bound_drops = info[INFO_BOUND_DROPS];
    c->skipped_rows = info[INFO_SKIP_ROWS];
    c->skipped_cols = info[INFO_SKIP_COLS];
    double f_lu = 0.0;  // getrf (2/3 b^3) and inverse (4/3 b^3) per diagonal block
    for (int32_t K = 0; K < c->nb; ++K) {
        const double b = c->h_bstart[K + 1] - c->h_bstart[K];
        f_lu += 2.0 * b * b * b;
    }
    c->flops_factor = (double)c->flop_upd_l + (double)c->flop_upd_u + (double)c->flop_scale +
                      (double)c->flop_norm + f_lu;
    *err = c->nperturb > 0 ? BILU_PERTURBED : BILU_OK;
    return 0;
}

}  // namespace

// Recording: samples held before this factorization (a re-run restarts from there).
static cudaError_t record_begin(bilu_ctx *c) {
    if (c->rec_cap <= 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(&c->rec_base, c->d_rec_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (c->rec_base > (unsigned long long)c->rec_cap) c->rec_base = (unsigned long long)c->rec_cap;
    return e;
}

// ---------------------------------------------------------------- tree schedule, host side

namespace {

// One group's scratch, carved from the groups' two allocations (base == nullptr: sizes only).
// `big` holds the candidate buffers and plans, `reset` what must be zero before every run
// (bitmaps, barrier, pivot-tile count, producer de-duplication, chunk cursors).
struct GroupPtrs {
    double *TL, *TU, *TUh, *TLP, *LU, *nrmL, *nrmU, *dcolsq;
    int32_t *rowsL, *rowsU, *keepL, *keepU, *wbL, *wbU, *xslotL, *xslotU, *perm, *kst;
    int64_t *pinfoL, *pinfoU;
    uint32_t *bmL, *bmU, *bar, *pivdone;
    int32_t *lastL, *lastU;
    int64_t *gcur;
};

template <class T>
void take(char *base, size_t &off, T *&p, int64_t count) {
    off = (off + 255) & ~(size_t)255;
    p = base ? (T *)(base + off) : nullptr;
    off += (size_t)std::max<int64_t>(count, 1) * sizeof(T);
}

size_t carve_big(const bilu_ctx *c, char *base, GroupPtrs &g) {
    size_t off = 0;
    const int64_t bmax = std::max(c->bmax, 1), n = std::max<int64_t>(c->n, 1);
    take(base, off, g.TL, c->capT * bmax);
    take(base, off, g.TU, c->capT * bmax);
    take(base, off, g.TUh, c->capT * bmax);
    take(base, off, g.TLP, (int64_t)PPART * BILU_MAX_BLOCK * BILU_MAX_BLOCK);
    take(base, off, g.LU, BILU_MAX_BLOCK * BILU_MAX_BLOCK + BILU_MAX_BLOCK);
    take(base, off, g.nrmL, c->capT);
    take(base, off, g.nrmU, c->capT);
    take(base, off, g.dcolsq, BILU_MAX_BLOCK);
    take(base, off, g.rowsL, c->capT);
    take(base, off, g.rowsU, c->capT);
    take(base, off, g.keepL, c->capT);
    take(base, off, g.keepU, c->capT);
    take(base, off, g.wbL, n / 32 + 2);
    take(base, off, g.wbU, n / 32 + 2);
    take(base, off, g.xslotL, c->capXS);
    take(base, off, g.xslotU, c->capXS);
    take(base, off, g.perm, BILU_MAX_BLOCK);
    take(base, off, g.kst, 16);
    take(base, off, g.pinfoL, (int64_t)PIS * c->prodcap);
    take(base, off, g.pinfoU, (int64_t)PIS * c->prodcap);
    return (off + 255) & ~(size_t)255;
}

size_t carve_reset(const bilu_ctx *c, char *base, GroupPtrs &g) {
    size_t off = 0;
    const int64_t n = std::max<int64_t>(c->n, 1), nb = std::max<int64_t>(c->nb, 1);
    take(base, off, g.gcur, 16);
    take(base, off, g.bar, 4);
    take(base, off, g.pivdone, 4);
    take(base, off, g.bmL, n / 32 + 2);
    take(base, off, g.bmU, n / 32 + 2);
    take(base, off, g.lastL, nb);
    take(base, off, g.lastU, nb);
    return (off + 255) & ~(size_t)255;
}

cudaError_t alloc_groups(bilu_ctx *c, int ng) {
    if (c->grp_n == ng && c->grp_key[0] == c->capT && c->grp_key[1] == c->prodcap && c->grp_key[2] == c->capXS)
        return cudaSuccess;
    dev_free(c->d_grp_big);
    dev_free(c->d_grp_reset);
    c->grp_n = 0;
    GroupPtrs g{};
    c->grp_big_bytes = carve_big(c, nullptr, g);
    c->grp_reset_bytes = carve_reset(c, nullptr, g);
    cudaError_t e;
    if ((e = dev_alloc(&c->d_grp_big, (int64_t)(c->grp_big_bytes * ng))) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_grp_reset, (int64_t)(c->grp_reset_bytes * ng))) != cudaSuccess) return e;
    c->grp_n = ng;
    c->grp_key[0] = c->capT;
    c->grp_key[1] = c->prodcap;
    c->grp_key[2] = c->capXS;
    return cudaSuccess;
}

// The chunked pools of the tree schedule, as large as the block-ordered pools or larger.
cudaError_t alloc_arena(bilu_ctx *c, const int64_t cap[4]) {
    dev_free(c->d_aLrow); dev_free(c->d_aUcol); dev_free(c->d_aLval); dev_free(c->d_aUval); dev_free(c->d_aUhval);
    dev_free(c->d_aLnrm); dev_free(c->d_aUnrm);
    for (auto &v : c->capA) v = 0;
    cudaError_t e;
    if ((e = dev_alloc(&c->d_aLrow, cap[0])) != cudaSuccess || (e = dev_alloc(&c->d_aLnrm, cap[0])) != cudaSuccess ||
        (e = dev_alloc(&c->d_aLval, cap[1])) != cudaSuccess || (e = dev_alloc(&c->d_aUcol, cap[2])) != cudaSuccess ||
        (e = dev_alloc(&c->d_aUnrm, cap[2])) != cudaSuccess || (e = dev_alloc(&c->d_aUval, cap[3])) != cudaSuccess ||
        (e = dev_alloc(&c->d_aUhval, cap[3])) != cudaSuccess)
        return e;
    for (int q = 0; q < 4; ++q) c->capA[q] = cap[q];
    return cudaSuccess;
}

const void *tree_kernel_for(int precision) {
    return precision == BILU_PREC_FP32   ? (const void *)bilu_factor_tree_kernel<float>
           : precision == BILU_PREC_BF16 ? (const void *)bilu_factor_tree_kernel<__nv_bfloat16>
                                         : (const void *)bilu_factor_tree_kernel<double>;
}

template <class TS>
cudaError_t launch_tree_copy(bilu_ctx *c, int grid) {
    tree_copy_kernel<TS><<<grid, 256, 0, c->stream>>>(
        c->nb, c->d_bstart, c->d_aptr, c->d_Lptr, c->d_Lvptr, c->d_Uptr, c->d_Uvptr, c->d_aLrow, c->d_aUcol,
        (const TS *)c->d_aLval, (const TS *)c->d_aUval, (const TS *)c->d_aUhval, c->d_Lrow, c->d_Ucol,
        (TS *)c->d_Lval, (TS *)c->d_Uval, (TS *)c->d_Uhval,
        c->d_status);
    return cudaGetLastError();
}

}  // namespace

// CTAs per group of the tree schedule: the caller's, else an eighth of the SMs (8 groups; on
// the 64^3 benchmark groups of 19 CTAs beat 4, 8, 38 and 76).
int tree_group_ctas(const bilu_ctx *c) {
    if (c->p.group_ctas > 0) return std::max(1, std::min(c->nsm, c->p.group_ctas));
    // Default: a block's parallel work (its candidates' updates and scaling) grows with the
    // coupling of A's rows, its pivot LU does not.  Densely coupled rows (>= 32 entries, e.g.
    // the 27-point elasticity operator) keep 8 groups of an eighth of the SMs; sparse stencils
    // run more groups of fewer CTAs: 15, or 19 with BF16 storage, whose update tiles on the
    // tensor cores are cheap (measured group-size sweeps on 64^3 convection-diffusion and 48^3
    // elasticity).
    const double per_row = c->n > 0 ? (double)c->nnz / (double)c->n : 0.0;
    const int groups = per_row >= 32.0 ? 8 : (c->p.precision == BILU_PREC_BF16 ? 19 : 15);
    return std::max(1, c->nsm / groups);
}

// Tree schedule: groups of G CTAs factor independent subtrees of the block elimination tree,
// the whole grid the trunk; then the kept rows and columns are copied from the groups' chunks
// into the block-ordered pools.
static bilu_status factor_tree_run(bilu_ctx *c, double droptol) {
    if (c->p.skip == BILU_SKIP_LEARNED || c->rec_cap > 0)
        return set_err(c, BILU_ERR_ARG, "the tree schedule does not run the learned skip or sample recording");
    const void *kfn = tree_kernel_for(c->p.precision);
    BILU_CUDA(c, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    int per_sm = 0;
    BILU_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, NT, SMEM_BYTES));
    if (per_sm < 1) return set_err(c, BILU_ERR_CUDA, "tree factor kernel cannot be resident");
    const int grid = c->nsm;
    const int G = tree_group_ctas(c);
    const int ng = grid / G;
    const int32_t nb = c->nb;
    const int32_t split = g_debug_no_trunk ? nb : c->tree_split;
    {
        const bilu_status st = tree_init(c, split);
        if (st != BILU_OK) return st;
    }
    cudaEvent_t e0, e1;
    BILU_CUDA(c, cudaEventCreate(&e0));
    BILU_CUDA(c, cudaEventCreate(&e1));
    bilu_status result = BILU_OK;
    bool finished = false;
    const bool hinted = hint_matches(c);
    for (int attempt = 0; attempt < 16; ++attempt) {
        int64_t need[4] = {c->capLrow, c->capLval, c->capUcol, c->capUval};
        for (int q = 0; q < 4 && hinted && attempt == 0; ++q) need[q] = std::max(need[q], c->hint_cap[4 + q]);
        if (c->capA[0] < need[0] || c->capA[1] < need[1] || c->capA[2] < need[2] || c->capA[3] < need[3] ||
            c->d_aptr == nullptr) {
            const int64_t cap[4] = {std::max(need[0], c->capA[0]), std::max(need[1], c->capA[1]),
                                    std::max(need[2], c->capA[2]), std::max(need[3], c->capA[3])};
            if (alloc_arena(c, cap) != cudaSuccess) { result = set_err(c, BILU_ERR_OOM, "tree factor: arena allocation failed"); break; }
            if (!c->d_aptr && dev_alloc(&c->d_aptr, 6 * (int64_t)std::max(nb, 1)) != cudaSuccess) {
                result = set_err(c, BILU_ERR_OOM, "tree factor: allocation failed");
                break;
            }
        }
        if (alloc_groups(c, ng) != cudaSuccess) { result = set_err(c, BILU_ERR_OOM, "tree factor: group scratch allocation failed"); break; }
        BILU_CUDA(c, prepare_run(c, c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_grp_reset, 0, c->grp_reset_bytes * ng, c->stream));
        const int64_t words = 14 + (int64_t)c->nsm + 2 * (int64_t)std::max(nb, 1);
        BILU_CUDA(c, cudaMemcpyAsync(c->d_tree, c->d_tree0, words * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
        std::vector<FactorArgs> h(ng);
        for (int g = 0; g < ng; ++g) {
            GroupPtrs gp{};
            carve_big(c, c->d_grp_big + (size_t)g * c->grp_big_bytes, gp);
            carve_reset(c, c->d_grp_reset + (size_t)g * c->grp_reset_bytes, gp);
            FactorArgs a = make_args(c, droptol, G);
            a.TL = gp.TL; a.TU = gp.TU; a.TUh = gp.TUh; a.TLP = gp.TLP; a.LU = gp.LU; a.nrmL = gp.nrmL; a.nrmU = gp.nrmU;
            a.dcolsq = gp.dcolsq; a.rowsL = gp.rowsL; a.rowsU = gp.rowsU; a.keepL = gp.keepL; a.keepU = gp.keepU;
            a.wbL = gp.wbL; a.wbU = gp.wbU; a.xslotL = gp.xslotL; a.xslotU = gp.xslotU; a.perm = gp.perm;
            a.kst = gp.kst; a.pinfoL = gp.pinfoL; a.pinfoU = gp.pinfoU; a.bmL = gp.bmL; a.bmU = gp.bmU;
            a.bar = gp.bar; a.pivdone = gp.pivdone; a.lastL = gp.lastL; a.lastU = gp.lastU; a.gcur = gp.gcur;
            // the pools are the arena; block K's rows are [Lptr[K], Lend[K]) there
            a.Lrow = c->d_aLrow; a.Ucol = c->d_aUcol; a.Lval = c->d_aLval; a.Uval = c->d_aUval; a.Uhval = c->d_aUhval;
            a.Lnrm = c->d_aLnrm; a.Unrm = c->d_aUnrm;
            a.Lptr = c->d_aptr; a.Lend = c->d_aptr + nb; a.Lvptr = c->d_aptr + 2 * (int64_t)nb;
            a.Uptr = c->d_aptr + 3 * (int64_t)nb; a.Uend = c->d_aptr + 4 * (int64_t)nb;
            a.Uvptr = c->d_aptr + 5 * (int64_t)nb;
            a.capLrow = c->capA[0]; a.capLval = c->capA[1]; a.capUcol = c->capA[2]; a.capUval = c->capA[3];
            a.arena = 1;
            a.sortprod = 1;
            a.acur = (unsigned long long *)c->d_tree;
            a.chunkR = std::max<int64_t>(1024, c->capA[0] / (16 * (int64_t)ng));
            a.chunkV = std::max<int64_t>(1024 * (int64_t)std::max(c->bmax, 1), c->capA[1] / (16 * (int64_t)ng));
            h[g] = a;
        }
        int32_t *h_trace = nullptr, *d_trace = nullptr;  // test hook: per-CTA progress, readable while running
        if (g_debug_trace && cudaHostAlloc((void **)&h_trace, 8 * sizeof(int32_t) * grid, cudaHostAllocMapped) == cudaSuccess) {
            for (int i = 0; i < 8 * grid; ++i) h_trace[i] = -1;
            if (cudaHostGetDevicePointer((void **)&d_trace, h_trace, 0) != cudaSuccess) d_trace = nullptr;
            for (auto &a : h) a.trace = d_trace;
        }
        int64_t *d_tl = nullptr;
        if (g_debug_trace && dev_alloc(&d_tl, 8 * (int64_t)std::max(nb, 1)) == cudaSuccess) {
            cudaMemsetAsync(d_tl, 0, 8 * sizeof(int64_t) * std::max(nb, 1), c->stream);
            for (auto &a : h) a.timeline = d_tl;
        }
        FactorArgs *d_args = nullptr;
        if (dev_alloc(&d_args, ng) != cudaSuccess) { result = set_err(c, BILU_ERR_OOM, "tree factor: allocation failed"); break; }
        cudaError_t e = cudaMemcpyAsync(d_args, h.data(), ng * sizeof(FactorArgs), cudaMemcpyHostToDevice, c->stream);
        TreeArgs t{};
        t.nb = nb; t.split = split; t.ngroups = ng; t.G = G; t.extra = g_debug_extra_cta;
        t.parent = c->d_parent;
        t.fullbar = (uint32_t *)(c->d_tree + 8);
        t.tctl = c->d_tree + 12;
        t.pending = c->d_tree + 14 + c->nsm;
        t.queue = t.pending + std::max(nb, 1);
        void *args[] = {&d_args, &t};
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess && nb > 0) {
            e = cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(NT), args, SMEM_BYTES, c->stream);
            if (e == cudaSuccess) {
                tree_offsets_kernel<<<1, 1024, 0, c->stream>>>(nb, c->d_bstart, c->d_aptr, c->d_Lptr, c->d_Lvptr,
                                                              c->d_Uptr, c->d_Uvptr, c->capLrow, c->capLval,
                                                              c->capUcol, c->capUval, c->d_status);
                e = cudaGetLastError();
            }
            const int cg = std::max(1, std::min<int>(nb, 4 * c->nsm));
            if (e == cudaSuccess)
                e = c->p.precision == BILU_PREC_FP32   ? launch_tree_copy<float>(c, cg)
                    : c->p.precision == BILU_PREC_BF16 ? launch_tree_copy<__nv_bfloat16>(c, cg)
                                                       : launch_tree_copy<double>(c, cg);
            c->launches += 3;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess && h_trace) {  // test hook: report where the CTAs are if the run takes long
            const auto t0 = std::chrono::steady_clock::now();
            int shots = 0;
            while (cudaStreamQuery(c->stream) == cudaErrorNotReady && shots < 3) {
                if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(5 + 5 * shots)) {
                    for (int b0 = 0; b0 < grid; ++b0)
                        if (h_trace[8 * b0] != 9)
                            fprintf(stderr, "t+%ds cta %d: mode %d block %d barrier %d wait %d barrier-polls/1024 %d "
                                    "pop-polls/1024 %d tile-wait-polls/1024 %d\n", 5 + 5 * shots, b0, h_trace[8 * b0],
                                    h_trace[8 * b0 + 1], h_trace[8 * b0 + 2], h_trace[8 * b0 + 3], h_trace[8 * b0 + 4],
                                    h_trace[8 * b0 + 5], h_trace[8 * b0 + 6]);
                    fflush(stderr);
                    ++shots;
                }
            }
        }
        int32_t status = 0;
        int64_t info[INFO_COUNT];
        unsigned long long used[4] = {0, 0, 0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(info, c->d_info, sizeof(info), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(used, c->d_tree, sizeof(used), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (h_trace) cudaFreeHost(h_trace);
        if (d_tl) {  // test hook: the per-block timeline, one line per block
            std::vector<int64_t> tl(8 * (size_t)std::max(nb, 1));
            if (cudaMemcpy(tl.data(), d_tl, tl.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) == cudaSuccess && e == cudaSuccess)
                for (int32_t K = 0; K < nb; ++K)
                    fprintf(stderr, "tl %d %lld %lld %lld %lld %lld %lld %lld %lld\n", K, (long long)tl[8 * K],
                            (long long)tl[8 * K + 1], (long long)tl[8 * K + 2], (long long)tl[8 * K + 3],
                            (long long)tl[8 * K + 4], (long long)tl[8 * K + 5], (long long)tl[8 * K + 6],
                            (long long)tl[8 * K + 7]);
            dev_free(d_tl);
        }
        dev_free(d_args);
        if (e != cudaSuccess) { result = cuda_err(c, e, "tree factor launch"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->t_factor_ms = ms;
        if (g_debug_trace)
            fprintf(stderr, "bilu tree factor: attempt %d status %d (block %lld, site %lld) %.3f ms; pools %lld %lld "
                    "%lld %lld, arena used %llu %llu %llu %llu of %lld %lld %lld %lld; prodcap %d capXS %lld\n",
                    attempt, status, (long long)info[INFO_FAIL_BLOCK], (long long)info[INFO_TIMEOUT_SITE], ms,
                    (long long)c->capLrow, (long long)c->capLval, (long long)c->capUcol, (long long)c->capUval,
                    used[0], used[1], used[2], used[3], (long long)c->capA[0], (long long)c->capA[1],
                    (long long)c->capA[2], (long long)c->capA[3], c->prodcap, (long long)c->capXS);
        if (status == DEV_POOL_OVERFLOW) {
            // the arena grows at once to what the failed run's chunks asked for (a cursor counts
            // every chunk handed out), the block-ordered pools to the kept totals the closing copy
            // found (when it ran), both at least doubled
            int64_t tot[4] = {0, 0, 0, 0};
            if (nb > 0) {
                BILU_CUDA(c, cudaMemcpy(&tot[0], c->d_Lptr + nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
                BILU_CUDA(c, cudaMemcpy(&tot[1], c->d_Lvptr + nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
                BILU_CUDA(c, cudaMemcpy(&tot[2], c->d_Uptr + nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
                BILU_CUDA(c, cudaMemcpy(&tot[3], c->d_Uvptr + nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
            }
            // what the whole factor needs, extrapolated from the blocks the groups had started
            // (queue head) when the run stopped, at most 16 times the chunks handed out: a heavy
            // fill then takes one or two re-runs instead of one per doubling
            int32_t head = 0;
            BILU_CUDA(c, cudaMemcpy(&head, c->d_tree + 12, sizeof(int32_t), cudaMemcpyDeviceToHost));
            const double scale = std::min(16.0, (double)std::max(nb, 1) / (double)std::max(1, std::min(head, nb)));
            int64_t *pc[4] = {&c->capLrow, &c->capLval, &c->capUcol, &c->capUval};
            int64_t cap[4];
            for (int q = 0; q < 4; ++q) {
                const int64_t est = (int64_t)((double)used[q] * scale);
                cap[q] = std::max({2 * c->capA[q], (int64_t)used[q] + (int64_t)used[q] / 4, est + est / 4});
                const bool grow = (int64_t)used[q] > c->capA[q] || tot[q] > *pc[q];
                if (grow) *pc[q] = std::max({2 * *pc[q], tot[q] + tot[q] / 4, est});
            }
            if (alloc_pools(c) != cudaSuccess || alloc_arena(c, cap) != cudaSuccess) {
                result = set_err(c, BILU_ERR_OOM, "tree factor: growing the pools failed");
                break;
            }
            c->pool_retries++;
            continue;
        }
        bilu_status err = BILU_OK;
        const int r = finish_run(c, status, info, &err);
        if (r == 1) continue;
        result = err;
        finished = r == 0;
        if (finished) {
            c->idle_ms = info[INFO_IDLE_NS] * 1e-6;
            // chunks left partly unused: keep a quarter of the arena free for the next run
            bool grow = false;
            for (int q = 0; q < 4; ++q) grow = grow || (int64_t)used[q] * 4 > c->capA[q] * 3;
            if (grow) {
                const int64_t cap[4] = {2 * c->capA[0], 2 * c->capA[1], 2 * c->capA[2], 2 * c->capA[3]};
                if (alloc_arena(c, cap) != cudaSuccess) result = set_err(c, BILU_ERR_OOM, "tree factor: arena growth failed");
            }
        }
        break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!finished && result >= 0) return set_err(c, BILU_ERR_OOM, "tree factor: too many pool re-runs");
    return result;
}

bilu_status factor_run(bilu_ctx *c, double droptol) {
    if (c->d_Lptr == nullptr) {
        bilu_status st = factor_alloc(c);
        if (st != BILU_OK) return st;
    }
    if (c->p.schedule == BILU_SCHED_TREE) return factor_tree_run(c, droptol);
    BILU_CUDA(c, record_begin(c));
    // kernel instance by the precision of the updates and the stored factor values
    const void *kfn = factor_kernel_for(c->p.precision);
    BILU_CUDA(c, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    int per_sm = 0;
    BILU_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, NT, SMEM_BYTES));
    if (per_sm < 1) return set_err(c, BILU_ERR_CUDA, "factor kernel cannot be resident");
    const int G = c->nsm;  // one CTA per SM

    cudaEvent_t e0, e1;
    BILU_CUDA(c, cudaEventCreate(&e0));
    BILU_CUDA(c, cudaEventCreate(&e1));
    bilu_status result = BILU_ERR_OOM;
    bool finished = false;
    for (int attempt = 0; attempt < 12; ++attempt) {
        BILU_CUDA(c, prepare_run(c, c->stream));
        FactorArgs a = make_args(c, droptol, G);
        void *args[] = {&a};
        BILU_CUDA(c, cudaEventRecord(e0, c->stream));
        if (c->nb > 0) {
            BILU_CUDA(c, cudaLaunchCooperativeKernel(kfn, dim3(G), dim3(NT), args, SMEM_BYTES, c->stream));
            c->launches += 1;
        }
        BILU_CUDA(c, cudaEventRecord(e1, c->stream));
        int32_t status = 0;
        int64_t info[INFO_COUNT];
        BILU_CUDA(c, cudaMemcpyAsync(&status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        BILU_CUDA(c, cudaMemcpyAsync(info, c->d_info, sizeof(info), cudaMemcpyDeviceToHost, c->stream));
        BILU_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->t_factor_ms = ms;
        bilu_status err = BILU_OK;
        const int r = finish_run(c, status, info, &err);
        if (r == 1) continue;
        result = err;
        finished = true;
        break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!finished) return set_err(c, BILU_ERR_OOM, "factor: too many pool re-runs");
    return result;
}

// ---------------------------------------------------------------- batched factorization

namespace {

struct BatchTune {
    int nsm, nmat, bmax, precision, G, trcap, tuned;
};
std::vector<BatchTune> g_batch_tune;  // group sizes and tile row caps chosen by the autotuner
std::mutex g_batch_tune_mu;           // guards g_batch_tune (calls on different contexts may overlap)

}  // namespace

// Factors every context's matrix in one cooperative launch: groups of G CTAs take matrices
// from a queue, largest first.  G, and then the most candidate rows per update tile, are
// chosen by timing candidates on the second call for a given (matrix count, largest block,
// precision) and cached.
bilu_status factor_batch_run(bilu_ctx *const *ctxs, int count, double droptol, double *ms_out) {
    bilu_ctx *c0 = ctxs[0];
    const int prec = c0->p.precision;
    int bmax = 0;
    for (int i = 0; i < count; ++i) {
        bilu_ctx *c = ctxs[i];
        if (!c->d_Lptr) {
            bilu_status st = factor_alloc(c);
            if (st != BILU_OK) return st;
        }
        bmax = std::max(bmax, c->bmax);
        BILU_CUDA(c0, record_begin(c));
    }
    const void *kfn = batch_kernel_for(prec);
    BILU_CUDA(c0, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    int per_sm = 0;
    BILU_CUDA(c0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, NT, SMEM_BYTES));
    if (per_sm < 1) return set_err(c0, BILU_ERR_CUDA, "batch factor kernel cannot be resident");
    const int nsm = c0->nsm;
    // matrices in the queue: largest first
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ctxs[x]->nnz > ctxs[y]->nnz; });
    // device buffers of this call (the batch API allocates per call)
    FactorArgs *d_args = nullptr;
    int *d_queue = nullptr;
    uint32_t *d_gbar = nullptr, *d_gpiv = nullptr;
    int32_t *d_gslot = nullptr, *d_gstat = nullptr;
    int64_t *d_ginfo = nullptr;
    auto release = [&]() {
        dev_free(d_args); dev_free(d_queue); dev_free(d_gbar); dev_free(d_gpiv); dev_free(d_gslot);
        dev_free(d_gstat); dev_free(d_ginfo);
    };
    if (dev_alloc(&d_args, count) != cudaSuccess || dev_alloc(&d_queue, 4) != cudaSuccess ||
        dev_alloc(&d_gbar, 4 * nsm) != cudaSuccess || dev_alloc(&d_gpiv, 4 * nsm) != cudaSuccess ||
        dev_alloc(&d_gslot, nsm) != cudaSuccess || dev_alloc(&d_gstat, nsm) != cudaSuccess ||
        dev_alloc(&d_ginfo, (int64_t)INFO_COUNT * nsm) != cudaSuccess) {
        release();
        return set_err(c0, BILU_ERR_OOM, "batch allocation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one launch over the matrices in `todo`; returns the kernel time
    auto launch = [&](const std::vector<int> &todo, int G, int trcap, float *ms) -> cudaError_t {
        cudaError_t e;
        std::vector<FactorArgs> h(todo.size());
        for (size_t k = 0; k < todo.size(); ++k) {
            bilu_ctx *c = ctxs[todo[k]];
            if ((e = prepare_run(c, c0->stream)) != cudaSuccess) return e;
            h[k] = make_args(c, droptol, G);
            h[k].trcap = std::max(4, std::min(TRMAX, trcap));
        }
        if ((e = cudaMemcpyAsync(d_args, h.data(), h.size() * sizeof(FactorArgs), cudaMemcpyHostToDevice, c0->stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(d_queue, 0, 4 * sizeof(int), c0->stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(d_gbar, 0, 4 * nsm * sizeof(uint32_t), c0->stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(d_gpiv, 0, 4 * nsm * sizeof(uint32_t), c0->stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(d_gstat, 0, nsm * sizeof(int32_t), c0->stream)) != cudaSuccess) return e;
        int nmat = (int)todo.size(), Gv = G;
        long long spin = g_debug_spin_limit > 0 ? g_debug_spin_limit : (1LL << 24);
        const int ngroups = nsm / G;
        void *args[] = {&d_args, &nmat, &d_queue, &d_gbar, &d_gpiv, &d_gslot, &d_gstat, &d_ginfo, &Gv, &spin};
        cudaEventRecord(e0, c0->stream);
        if ((e = cudaLaunchCooperativeKernel(kfn, dim3(ngroups * G), dim3(NT), args, SMEM_BYTES, c0->stream)) != cudaSuccess)
            return e;
        cudaEventRecord(e1, c0->stream);
        c0->launches += 1;
        if ((e = cudaStreamSynchronize(c0->stream)) != cudaSuccess) return e;
        cudaEventElapsedTime(ms, e0, e1);
        return cudaSuccess;
    };
    // Group size.  Candidates split the SMs into a power-of-two number of groups g (G = nsm / g
    // CTAs each), from about count / 8 groups (several matrices per group, larger groups) to
    // about 2 count (every matrix at once, smallest groups), G >= 2 so that the pivot LU of a
    // block overlaps its update tiles.  The first call for a (SM count, matrix count, largest
    // block, precision) runs with g = the power of two >= count / 4 (and grows the pools); the
    // next call times the candidates, largest G first, until one is slower than the one
    // before, and caches the fastest.
    std::vector<int> cands;
    for (int g = 1; g <= nsm; g *= 2) {
        const int Gc = nsm / g;
        if (Gc < 2 && nsm >= 2) break;
        if (8 * g < count && Gc > 2) continue;
        if (g > 2 * count) break;
        cands.push_back(Gc);
    }
    if (cands.empty()) cands.push_back(std::max(1, nsm / 2));
    int G = 0;
    auto same = [&](const BatchTune &t) {
        return t.nsm == nsm && t.nmat == count && t.bmax == bmax && t.precision == prec;
    };
    bool have = false, tuned = false;
    int cachedG = 0, cachedCap = TRMAX, cap = TRMAX;
    {
        std::lock_guard<std::mutex> lk(g_batch_tune_mu);
        for (const auto &t : g_batch_tune)
            if (same(t)) { have = true; tuned = t.tuned != 0; cachedG = t.G; cachedCap = t.trcap; }
    }
    std::vector<int> todo(order);
    float best_ms = 0.f;
    if (g_debug_batch_group > 0) {
        G = (int)std::min<long long>(g_debug_batch_group, nsm);
    } else if (!have) {
        int g = 1;
        while (4 * g < count && 2 * g <= nsm / 2) g *= 2;
        G = std::max(1, nsm / g);
        std::lock_guard<std::mutex> lk(g_batch_tune_mu);
        bool dup = false;
        for (const auto &t : g_batch_tune) dup = dup || same(t);
        if (!dup) g_batch_tune.push_back({nsm, count, bmax, prec, G, TRMAX, 0});
    } else if (!tuned) {
        float best = 1e30f;
        int bestG = cachedG, bestCap = TRMAX;
        bool ok = true;
        // one timed launch; false when it must stop tuning (a pool grew, or a launch error in *err)
        auto trial = [&](int Gc, int capc, float *ms, cudaError_t *err) -> bool {
            *err = launch(todo, Gc, capc, ms);
            if (*err != cudaSuccess) return false;
            for (int i : todo) {
                int32_t st = 0;
                cudaMemcpy(&st, ctxs[i]->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
                ok = ok && st == DEV_OK;
            }
            return ok;  // pools still growing: tune on a later call
        };
        cudaError_t e = cudaSuccess;
        for (int Gc : cands) {
            float ms = 0.f;
            if (!trial(Gc, TRMAX, &ms, &e)) break;
            if (ms < best) { best = ms; bestG = Gc; }
            else break;  // past the minimum
        }
        // then smaller update tiles at that group size: more tiles per block for the group's
        // CTAs when the matrices are small
        for (int capc = TRMAX / 2; ok && e == cudaSuccess && capc >= 4; capc /= 2) {
            float ms = 0.f;
            if (!trial(bestG, capc, &ms, &e)) break;
            if (ms < best) { best = ms; bestCap = capc; }
            else break;
        }
        if (e != cudaSuccess) { release(); cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_err(c0, e, "batch factor launch"); }
        G = bestG;
        cap = bestCap;
        if (ok) {
            std::lock_guard<std::mutex> lk(g_batch_tune_mu);
            for (auto &t : g_batch_tune)
                if (same(t)) { t.G = bestG; t.trcap = bestCap; t.tuned = 1; }
        }
    } else {
        G = cachedG;
        cap = cachedCap;
    }
    if (g_debug_batch_trcap > 0) cap = (int)std::min<long long>(g_debug_batch_trcap, TRMAX);
    bilu_status result = BILU_OK;
    for (int attempt = 0; attempt < 12 && !todo.empty(); ++attempt) {
        float ms = 0.f;
        cudaError_t e = launch(todo, G, cap, &ms);
        if (e != cudaSuccess) { release(); cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_err(c0, e, "batch factor launch"); }
        best_ms += ms;
        std::vector<int> again;
        for (int i : todo) {
            bilu_ctx *c = ctxs[i];
            int32_t status = 0;
            int64_t info[INFO_COUNT];
            cudaMemcpy(&status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
            cudaMemcpy(info, c->d_info, sizeof(info), cudaMemcpyDeviceToHost);
            c->t_factor_ms = ms;
            bilu_status err = BILU_OK;
            const int r = finish_run(c, status, info, &err);
            if (r == 1) again.push_back(i);
            else if (r < 0) result = err;
            else if (err == BILU_PERTURBED && result == BILU_OK) result = BILU_PERTURBED;
        }
        if (result < 0) break;
        todo.swap(again);
    }
    if (!todo.empty() && result >= 0) result = set_err(c0, BILU_ERR_OOM, "batch factor: too many pool re-runs");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    if (ms_out) *ms_out = best_ms;
    return result;
}
