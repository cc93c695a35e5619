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
#include <cmath>
#include <cstring>

#include "dev_common.cuh"

namespace {

constexpr int NT = 512;          // threads per CTA
constexpr int NW = NT / 32;      // warps per CTA
constexpr int TRMAX = 32;        // max candidate slots per accumulation tile
constexpr int PS = BILU_MAX_BLOCK + 1;  // padded row stride (doubles) of staged panels
constexpr int PMAX = 1024;       // max producers per block handled by the kernel
constexpr int SMEM_BYTES = 80 * 1024;

struct FactorArgs {
    int32_t n, nb, G, perturb;
    double tau, alpha, pert_tau, pert_rho;
    long long spin_limit;
    const int32_t *rowptr, *colind, *colptr, *rowind, *bstart, *blkof;
    const double *val, *cval;
    const int64_t *Dptr;
    int64_t *Lptr, *Lvptr, *Uptr, *Uvptr;
    int32_t *Lrow, *Ucol;
    double *Lval, *Uval, *Dinv, *Pblk;
    int64_t capLrow, capLval, capUcol, capUval;
    int32_t prodcap;
    int32_t *prodL, *prodLcnt, *prodU, *prodUcnt, *lastL, *lastU;
    double *TL, *TU;
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
};

// pinfo layout (per producer t of the current block)
enum { PI_J = 0, PI_BJ, PI_XCNT, PI_YCNT, PI_OFF, PI_XPOS, PI_XVAL, PI_YVAL, PI_YPOS, PIS };

__device__ __forceinline__ double perturbed(double d, double ptau, double prho, double alpha) {
    // Sec. 3.6: d (1 + rho beta_j) + sign(d) tau alpha with beta_j := 1 and sign(0) := +1
    return d * (1.0 + prho) + (d >= 0.0 ? 1.0 : -1.0) * ptau * alpha;
}

// ---------------------------------------------------------------- phase A
// Candidate set and update plan of one side (L: rows of the block column, U: columns of
// the block row) of block K; executed by one whole CTA.
__device__ void phase_A(const FactorArgs &a, int K, bool Lside, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    int32_t *xcnt = (int32_t *)smem;            // PMAX
    int32_t *off = xcnt + PMAX;                  // PMAX + 1
    int32_t *ws = off + PMAX + 1;                // 33
    int32_t *lohi = ws + 40;                     // 2

    const int32_t *plist = (Lside ? a.prodL : a.prodU) + (int64_t)K * a.prodcap;
    int pcnt = ldcg((Lside ? a.prodLcnt : a.prodUcnt) + K);
    if (pcnt > a.prodcap || pcnt > PMAX) {
        if (tid == 0) set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
        pcnt = 0;
    }
    int64_t *pinfo = Lside ? a.pinfoL : a.pinfoU;
    uint32_t *bm = Lside ? a.bmL : a.bmU;
    int32_t *wb = Lside ? a.wbL : a.wbU;
    int32_t *xslot = Lside ? a.xslotL : a.xslotU;
    int32_t *rows = Lside ? a.rowsL : a.rowsU;
    if (tid == 0) { lohi[0] = INT32_MAX; lohi[1] = -1; }

    // producer ranges: warp per producer
    for (int t = warp; t < pcnt; t += NW) {
        const int J = ldcg(plist + t);
        const int bJ = a.bstart[J + 1] - a.bstart[J];
        const int l0 = (int)ldcg(a.Lptr + J), l1 = (int)ldcg(a.Lptr + J + 1);
        const int u0 = (int)ldcg(a.Uptr + J), u1 = (int)ldcg(a.Uptr + J + 1);
        int xbeg, xend, ybeg, yend;
        int64_t xval, yval;
        if (Lside) {  // X: L_J rows >= s0, Y: U-breve_J columns in [s0, s1)
            xbeg = warp_lower_bound(a.Lrow, l0, l1, s0);
            xend = l1;
            ybeg = warp_lower_bound(a.Ucol, u0, u1, s0);
            yend = warp_lower_bound(a.Ucol, ybeg, u1, s1);
            xval = ldcg(a.Lvptr + J) + (int64_t)(xbeg - l0) * bJ;
            yval = ldcg(a.Uvptr + J) + (int64_t)(ybeg - u0) * bJ;
        } else {      // X: U-breve_J columns >= s1, Y: L_J rows in [s0, s1)
            xbeg = warp_lower_bound(a.Ucol, u0, u1, s1);
            xend = u1;
            ybeg = warp_lower_bound(a.Lrow, l0, l1, s0);
            yend = warp_lower_bound(a.Lrow, ybeg, l1, s1);
            xval = ldcg(a.Uvptr + J) + (int64_t)(xbeg - u0) * bJ;
            yval = ldcg(a.Lvptr + J) + (int64_t)(ybeg - l0) * bJ;
        }
        if (lane == 0) {
            int64_t *pi = pinfo + PIS * t;
            pi[PI_J] = J;
            pi[PI_BJ] = bJ;
            pi[PI_XCNT] = xend - xbeg;
            pi[PI_YCNT] = yend - ybeg;
            pi[PI_XPOS] = xbeg;
            pi[PI_XVAL] = xval;
            pi[PI_YVAL] = yval;
            pi[PI_YPOS] = ybeg;
            xcnt[t] = xend - xbeg;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int t = 0; t < pcnt; ++t) { off[t] = acc; acc += xcnt[t]; }
        off[pcnt] = acc;
    }
    __syncthreads();
    if ((int64_t)off[pcnt] > a.capXS) {
        if (tid == 0) set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
        return;
    }
    for (int t = tid; t < pcnt; t += NT) pinfo[PIS * t + PI_OFF] = off[t];

    // mark candidates >= s1 in the bitmap
    int lo = INT32_MAX, hi = -1;
    if (Lside) {
        const int e0 = a.colptr[s0], e1 = a.colptr[s1];
        for (int e = e0 + tid; e < e1; e += NT) {
            const int i = a.rowind[e];
            if (i >= s1) { atomicOr(bm + (i >> 5), 1u << (i & 31)); lo = min(lo, i); hi = max(hi, i); }
        }
    } else {
        const int e0 = a.rowptr[s0], e1 = a.rowptr[s1];
        for (int e = e0 + tid; e < e1; e += NT) {
            const int j = a.colind[e];
            if (j >= s1) { atomicOr(bm + (j >> 5), 1u << (j & 31)); lo = min(lo, j); hi = max(hi, j); }
        }
    }
    const int32_t *Xidx = Lside ? a.Lrow : a.Ucol;
    for (int t = 0; t < pcnt; ++t) {
        const int xpos = (int)ldcg(pinfo + PIS * t + PI_XPOS);
        for (int f = tid; f < xcnt[t]; f += NT) {
            const int i = ldcg(Xidx + xpos + f);
            if (i >= s1) { atomicOr(bm + (i >> 5), 1u << (i & 31)); lo = min(lo, i); hi = max(hi, i); }
        }
    }
    lo = __reduce_min_sync(FULL_MASK, lo);
    hi = __reduce_max_sync(FULL_MASK, hi);
    if (lane == 0) { atomicMin(lohi, lo); atomicMax(lohi + 1, hi); }
    __syncthreads();
    __threadfence_block();
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
    for (int t = 0; t < pcnt; ++t) {
        const int xpos = (int)ldcg(pinfo + PIS * t + PI_XPOS);
        for (int f = tid; f < xcnt[t]; f += NT) {
            const int i = ldcg(Xidx + xpos + f);
            int slot;
            if (i < s1) {
                slot = i - s0;  // pivot rows (L side only)
            } else {
                const uint32_t word = ldcg(bm + (i >> 5));
                slot = pre + ldcg(wb + ((i >> 5) - wlo)) + __popc(word & ((1u << (i & 31)) - 1u));
            }
            xslot[off[t] + f] = slot;
        }
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
__device__ void phase_B_tile(const FactorArgs &a, int K, bool Lside, int sa, int cnt, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    double *T = (double *)smem;                  // TRMAX * 64
    double *Xs = T + TRMAX * BILU_MAX_BLOCK;     // TRMAX * PS
    double *Ys = Xs + TRMAX * PS;                // 64 * PS
    int32_t *g = (int32_t *)(Ys + BILU_MAX_BLOCK * PS);  // TRMAX
    int32_t *xl = g + TRMAX;                     // TRMAX: local slot of staged X rows
    int32_t *yc = xl + TRMAX;                    // 64: column of staged Y rows
    int32_t *sxs = yc + BILU_MAX_BLOCK;          // PMAX
    int32_t *sxe = sxs + PMAX;                   // PMAX

    const int32_t *rows = Lside ? a.rowsL : a.rowsU;
    for (int r = tid; r < cnt; r += NT) g[r] = ldcg(rows + sa + r);
    for (int e = tid; e < cnt * b; e += NT) T[e] = 0.0;
    __syncthreads();
    // load A: L side rows i of A restricted to columns B_K; U side columns j restricted to rows B_K
    for (int r = warp; r < cnt; r += NW) {
        const int idx = g[r];
        if (Lside) {
            for (int e = a.rowptr[idx] + lane; e < a.rowptr[idx + 1]; e += 32) {
                const int c = a.colind[e];
                if (c >= s0 && c < s1) T[r * b + (c - s0)] = a.val[e];
            }
        } else {
            for (int e = a.colptr[idx] + lane; e < a.colptr[idx + 1]; e += 32) {
                const int rr = a.rowind[e];
                if (rr >= s0 && rr < s1) T[r * b + (rr - s0)] = a.cval[e];
            }
        }
    }
    const int pcnt = ldcg(a.kst + (Lside ? 2 : 3));
    const int64_t *pinfo = Lside ? a.pinfoL : a.pinfoU;
    const int32_t *xslot = Lside ? a.xslotL : a.xslotU;
    // X entries of each producer that fall into this tile (slots are sorted)
    for (int t = warp; t < pcnt; t += NW) {
        const int xc = (int)ldcg(pinfo + PIS * t + PI_XCNT);
        const int o = (int)ldcg(pinfo + PIS * t + PI_OFF);
        const int xs = warp_lower_bound(xslot + o, 0, xc, sa);
        const int xe = warp_lower_bound(xslot + o, xs, xc, sa + cnt);
        if (lane == 0) { sxs[t] = xs; sxe[t] = xe; }
    }
    __syncthreads();
    const double *Xpool = Lside ? a.Lval : a.Uval;
    const double *Ypool = Lside ? a.Uval : a.Lval;
    const int32_t *Yidx = Lside ? a.Ucol : a.Lrow;
    for (int t = 0; t < pcnt; ++t) {
        const int nx = sxe[t] - sxs[t];
        const int ny = (int)ldcg(pinfo + PIS * t + PI_YCNT);
        if (nx <= 0 || ny <= 0) continue;  // uniform across the CTA
        if (nx > TRMAX || ny > b) {
            if (tid == 0) set_status(a.status, DEV_INTERNAL, a.info, K);
            return;
        }
        const int bJ = (int)ldcg(pinfo + PIS * t + PI_BJ);
        const int o = (int)ldcg(pinfo + PIS * t + PI_OFF);
        const int64_t xval = ldcg(pinfo + PIS * t + PI_XVAL) + (int64_t)sxs[t] * bJ;
        const int64_t yval = ldcg(pinfo + PIS * t + PI_YVAL);
        // Y position: for the L side the U-breve columns in B_K, for the U side the L rows in B_K
        for (int e = tid; e < nx * bJ; e += NT) {
            const int x = e / bJ, k = e - x * bJ;
            Xs[x * PS + k] = ldcg(Xpool + xval + e);
        }
        for (int e = tid; e < ny * bJ; e += NT) {
            const int y = e / bJ, k = e - y * bJ;
            Ys[y * PS + k] = ldcg(Ypool + yval + e);
        }
        if (tid < nx) {
            int v = ldcg(xslot + o + sxs[t] + tid) - sa;
            if (v < 0 || v >= cnt) { set_status(a.status, DEV_INTERNAL, a.info, K); v = 0; }
            xl[tid] = v;
        }
        if (tid >= 64 && tid - 64 < ny) {
            const int y = tid - 64;
            const int64_t ypos = ldcg(pinfo + PIS * t + PI_YPOS);
            int v = ldcg(Yidx + ypos + y) - s0;
            if (v < 0 || v >= b) { set_status(a.status, DEV_INTERNAL, a.info, K); v = 0; }
            yc[y] = v;
        }
        __syncthreads();
        for (int e = tid; e < nx * ny; e += NT) {
            const int x = e / ny, y = e - x * ny;
            const double *xr = Xs + x * PS, *yr = Ys + y * PS;
            double s = 0.0;
            for (int k = 0; k < bJ; ++k) s = fma(xr[k], yr[k], s);
            T[xl[x] * b + yc[y]] -= s;
        }
        __syncthreads();
    }
    double *out = (Lside ? a.TL : a.TU) + (int64_t)sa * b;
    for (int e = tid; e < cnt * b; e += NT) out[e] = T[e];
}

// ---------------------------------------------------------------- phase C
// LU with partial pivoting of the pivot block in shared memory (one CTA), with the
// perturbation of Sec. 3.6.  Writes P (possibly perturbed) to Pblk, LU and perm to scratch.
__device__ void phase_C(const FactorArgs &a, int K, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    double *P = (double *)smem;                 // b x b (stride PS), current P (perturbed)
    double *M = P + BILU_MAX_BLOCK * PS;        // LU work
    int32_t *prm = (int32_t *)(M + BILU_MAX_BLOCK * PS);  // 64
    int32_t *sh = prm + BILU_MAX_BLOCK;         // [0] pivot row, [1] bad column, [2] count
    double *shd = (double *)(sh + 8);           // [0] amax, [1] pmax
    for (int e = tid; e < b * b; e += NT) {
        const int r = e / b, c = e - r * b;
        P[r * PS + c] = ldcg(a.TL + (int64_t)r * b + c);
    }
    if (tid == 0) sh[2] = 0;
    __syncthreads();
    if (a.perturb) {
        // all-zero columns, then all-zero rows: perturb the diagonal entry
        if (tid == 0) {
            int cnt = 0;
            for (int j = 0; j < b; ++j) {
                bool zero = true;
                for (int i = 0; i < b; ++i) zero &= (P[i * PS + j] == 0.0);
                if (zero) { P[j * PS + j] = perturbed(P[j * PS + j], a.pert_tau, a.pert_rho, a.alpha); ++cnt; }
            }
            for (int i = 0; i < b; ++i) {
                bool zero = true;
                for (int j = 0; j < b; ++j) zero &= (P[i * PS + j] == 0.0);
                if (zero) { P[i * PS + i] = perturbed(P[i * PS + i], a.pert_tau, a.pert_rho, a.alpha); ++cnt; }
            }
            sh[2] = cnt;
        }
        __syncthreads();
    }
    bool done = false;
    for (int attempt = 0; attempt <= 2 * b && !done; ++attempt) {
        // max |P| and copy to the work array
        double mx = 0.0;
        for (int e = tid; e < b * b; e += NT) {
            const int r = e / b, c = e - r * b;
            const double v = P[r * PS + c];
            M[r * PS + c] = v;
            mx = fmax(mx, fabs(v));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL_MASK, mx, o));
        if (tid == 0) shd[1] = 0.0;
        __syncthreads();
        if (lane == 0) {
            // atomicMax on doubles via the ordered int64 view of non-negative values
            atomicMax((unsigned long long *)&shd[1], (unsigned long long)__double_as_longlong(mx));
        }
        for (int i = tid; i < b; i += NT) prm[i] = i;
        if (tid == 0) sh[1] = -1;
        __syncthreads();
        const double thresh = 1e-14 * shd[1];
        for (int j = 0; j < b; ++j) {
            if (warp == 0) {
                // first index of the largest |.| in column j, rows j..b-1
                double best = -1.0;
                int bi = b;
                for (int i = j + lane; i < b; i += 32) {
                    const double v = fabs(M[i * PS + j]);
                    if (v > best) { best = v; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_xor_sync(FULL_MASK, best, o);
                    const int oi = __shfl_xor_sync(FULL_MASK, bi, o);
                    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
                }
                if (lane == 0) { sh[0] = bi; shd[0] = best; }
            }
            __syncthreads();
            if (!(shd[0] > thresh)) {  // singular / ill-conditioned pivot
                if (tid == 0) sh[1] = j;
                __syncthreads();
                break;
            }
            const int p = sh[0];
            if (p != j) {
                for (int c = tid; c < b; c += NT) {
                    const double t = M[j * PS + c];
                    M[j * PS + c] = M[p * PS + c];
                    M[p * PS + c] = t;
                }
                if (tid == 0) { const int t = prm[j]; prm[j] = prm[p]; prm[p] = t; }
            }
            __syncthreads();
            const double piv = M[j * PS + j];
            for (int i = j + 1 + tid; i < b; i += NT) M[i * PS + j] /= piv;
            __syncthreads();
            const int m = b - j - 1;
            for (int e = tid; e < m * m; e += NT) {
                const int i = j + 1 + e / m, c = j + 1 + e % m;
                M[i * PS + c] -= M[i * PS + j] * M[j * PS + c];
            }
            __syncthreads();
        }
        const int bad = sh[1];
        if (bad < 0) { done = true; break; }
        if (!a.perturb) break;
        if (tid == 0) {
            int k = 0;
            for (int i = 1; i < b; ++i)
                if (fabs(P[i * PS + bad]) > fabs(P[k * PS + bad])) k = i;
            if (2.0 * fabs(P[bad * PS + bad]) >= fabs(P[k * PS + bad])) k = bad;
            P[k * PS + bad] = perturbed(P[k * PS + bad], a.pert_tau, a.pert_rho, a.alpha);
            sh[2] += 1;
        }
        __syncthreads();
    }
    if (!done) {
        if (tid == 0) set_status(a.status, DEV_SINGULAR, a.info, K);
        return;
    }
    const int64_t dofs = a.Dptr[K];
    for (int e = tid; e < b * b; e += NT) {
        const int r = e / b, c = e - r * b;
        a.Pblk[dofs + e] = P[r * PS + c];
        a.LU[e] = M[r * PS + c];
    }
    for (int i = tid; i < b; i += NT) a.perm[i] = prm[i];
    if (tid == 0 && sh[2] > 0) atomicAdd((unsigned long long *)(a.info + INFO_NPERTURB), (unsigned long long)sh[2]);
}

// ---------------------------------------------------------------- phase C2
// Column c of D_K = P_K^{-1}: solve L U x = e_{perm^{-1}(c)} (P_K X = I), one warp per column.
__device__ void phase_C2(const FactorArgs &a, int K, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    const int first = blockIdx.x * NW;
    if (first >= b) return;
    double *M = (double *)smem;
    int32_t *prm = (int32_t *)(M + BILU_MAX_BLOCK * PS);
    for (int e = tid; e < b * b; e += NT) {
        const int r = e / b, c = e - r * b;
        M[r * PS + c] = ldcg(a.LU + e);
    }
    for (int i = tid; i < b; i += NT) prm[i] = ldcg(a.perm + i);
    __syncthreads();
    const int c = first + warp;
    if (c >= b) return;
    // lane owns rows lane and lane + 32
    double y0 = (lane < b && prm[lane] == c) ? 1.0 : 0.0;
    double y1 = (lane + 32 < b && prm[lane + 32] == c) ? 1.0 : 0.0;
    for (int k = 0; k < b; ++k) {  // forward, unit lower
        const double yk = __shfl_sync(FULL_MASK, k < 32 ? y0 : y1, k & 31);
        if (lane > k && lane < b) y0 -= M[lane * PS + k] * yk;
        if (lane + 32 > k && lane + 32 < b) y1 -= M[(lane + 32) * PS + k] * yk;
    }
    for (int k = b - 1; k >= 0; --k) {  // backward, upper
        double own = k < 32 ? y0 : y1;
        if ((k & 31) == lane) own = own / M[k * PS + k];
        const double xk = __shfl_sync(FULL_MASK, own, k & 31);
        if (k < 32) { if (lane == k) y0 = xk; } else { if (lane + 32 == k) y1 = xk; }
        if (lane < k) y0 -= M[lane * PS + k] * xk;
        if (lane + 32 < k) y1 -= M[(lane + 32) * PS + k] * xk;
    }
    double *D = a.Dinv + a.Dptr[K];
    if (lane < b) D[lane * b + c] = y0;
    if (lane + 32 < b) D[(lane + 32) * b + c] = y1;
}

// ---------------------------------------------------------------- phase D
// Normalised rows l_i = T_L[i,:] D_K and columns u^_j = D_K T_U[:,j]; keep iff ||.||_2 > tau.
__device__ void phase_D(const FactorArgs &a, int K, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    const int mL = ldcg(a.kst + 0), mU = ldcg(a.kst + 1);
    const int nLc = mL - b, total = nLc + mU;
    if (blockIdx.x * NW >= total) return;
    double *Ds = (double *)smem;
    const double *D = a.Dinv + a.Dptr[K];
    for (int e = tid; e < b * b; e += NT) {
        const int r = e / b, c = e - r * b;
        Ds[r * PS + c] = ldcg(D + e);
    }
    __syncthreads();
    for (int item = blockIdx.x * NW + warp; item < total; item += a.G * NW) {
        if (item < nLc) {
            const int slot = b + item;
            double *t = a.TL + (int64_t)slot * b;
            const double t0 = lane < b ? ldcg(t + lane) : 0.0;
            const double t1 = lane + 32 < b ? ldcg(t + lane + 32) : 0.0;
            double l0 = 0.0, l1 = 0.0;
            for (int k = 0; k < b; ++k) {
                const double tk = __shfl_sync(FULL_MASK, k < 32 ? t0 : t1, k & 31);
                if (lane < b) l0 = fma(tk, Ds[k * PS + lane], l0);
                if (lane + 32 < b) l1 = fma(tk, Ds[k * PS + lane + 32], l1);
            }
            const double nrm2 = warp_sum(l0 * l0 + l1 * l1);
            if (lane < b) t[lane] = l0;
            if (lane + 32 < b) t[lane + 32] = l1;
            if (lane == 0) a.keepL[slot] = sqrt(nrm2) > a.tau ? 1 : 0;
        } else {
            const int slot = item - nLc;
            const double *t = a.TU + (int64_t)slot * b;
            const double t0 = lane < b ? ldcg(t + lane) : 0.0;
            const double t1 = lane + 32 < b ? ldcg(t + lane + 32) : 0.0;
            double u0 = 0.0, u1 = 0.0;
            for (int k = 0; k < b; ++k) {
                const double tk = __shfl_sync(FULL_MASK, k < 32 ? t0 : t1, k & 31);
                if (lane < b) u0 = fma(Ds[lane * PS + k], tk, u0);
                if (lane + 32 < b) u1 = fma(Ds[(lane + 32) * PS + k], tk, u1);
            }
            const double nrm2 = warp_sum(u0 * u0 + u1 * u1);
            if (lane == 0) a.keepU[slot] = sqrt(nrm2) > a.tau ? 1 : 0;
        }
    }
}

// ---------------------------------------------------------------- phase E
// Compaction of the kept rows / columns (sorted) into the pools and producer appends.
// Candidate slots are cut into tiles of 32; one warp per tile ranks its kept slots with a
// ballot.  Every CTA with work computes the tile prefix sums itself (no extra barrier).
__device__ void phase_E(const FactorArgs &a, int K, char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
    const int mL = ldcg(a.kst + 0), mU = ldcg(a.kst + 1);
    const int nLc = mL - b;
    const int tL = (nLc + 31) >> 5, tU = (mU + 31) >> 5;
    int32_t *cnt = (int32_t *)smem;  // NT tile offsets of the current chunk
    int32_t *ws = cnt + NT;          // scan scratch
    const int64_t Lbase = ldcg(a.Lptr + K), LVbase = ldcg(a.Lvptr + K);
    const int64_t Ubase = ldcg(a.Uptr + K), UVbase = ldcg(a.Uvptr + K);
    const bool has_work = blockIdx.x == 0 || blockIdx.x * NW < max(tL, tU);
    if (!has_work) return;
    int keptL, keptU;
    {
        int lk = 0, uk = 0;
        for (int s = tid; s < nLc; s += NT) lk += ldcg(a.keepL + b + s);
        for (int s = tid; s < mU; s += NT) uk += ldcg(a.keepU + s);
        block_excl_scan(lk, ws, &keptL);
        block_excl_scan(uk, ws, &keptU);
    }
    const bool overflow = Lbase + keptL > a.capLrow || LVbase + (int64_t)keptL * b > a.capLval ||
                          Ubase + keptU > a.capUcol || UVbase + (int64_t)keptU * b > a.capUval;
    if (overflow) {
        if (blockIdx.x == 0 && tid == 0) set_status(a.status, DEV_POOL_OVERFLOW, a.info, K);
        return;
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.Lptr[K + 1] = Lbase + keptL;
        a.Lvptr[K + 1] = LVbase + (int64_t)keptL * b;
        a.Uptr[K + 1] = Ubase + keptU;
        a.Uvptr[K + 1] = UVbase + (int64_t)keptU * b;
        atomicAdd((unsigned long long *)(a.info + INFO_CAND_ROWS), (unsigned long long)nLc);
        atomicAdd((unsigned long long *)(a.info + INFO_CAND_COLS), (unsigned long long)mU);
    }
    for (int side = 0; side < 2; ++side) {
        const bool isL = side == 0;
        const int ntile = isL ? tL : tU;
        const int sfirst = isL ? b : 0, send = isL ? mL : mU;
        const int32_t *kp = isL ? a.keepL : a.keepU;
        int carry = 0;
        for (int c0 = 0; c0 < ntile; c0 += NT) {
            const int cn = min(NT, ntile - c0);
            int my = 0;
            if (tid < cn) {
                const int sb = sfirst + (c0 + tid) * 32, se = min(send, sb + 32);
                for (int s = sb; s < se; ++s) my += ldcg(kp + s);
            }
            int tot;
            const int ex = block_excl_scan(my, ws, &tot);
            if (tid < cn) cnt[tid] = carry + ex;
            __syncthreads();
            for (int T = c0 + blockIdx.x * NW + warp; T < c0 + cn; T += a.G * NW) {
                const int sb = sfirst + T * 32, se = min(send, sb + 32);
                const int s = sb + lane;
                const bool kept = s < se && ldcg(kp + s) != 0;
                const unsigned m = __ballot_sync(FULL_MASK, kept);
                const int64_t base = cnt[T - c0];
                unsigned mm = m;
                while (mm) {
                    const int l = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const int slot = sb + l;
                    const int64_t o = base + __popc(m & ((1u << l) - 1u));
                    const int idx = ldcg((isL ? a.rowsL : a.rowsU) + slot);
                    const double *src = (isL ? a.TL : a.TU) + (int64_t)slot * b;
                    double *dst = isL ? a.Lval + LVbase + o * b : a.Uval + UVbase + o * b;
                    for (int c = lane; c < b; c += 32) dst[c] = ldcg(src + c);
                    if (lane == 0) {
                        const int tb = a.blkof[idx];
                        int32_t *last = isL ? a.lastU : a.lastL;
                        int32_t *pc = isL ? a.prodUcnt : a.prodLcnt;
                        int32_t *pl = isL ? a.prodU : a.prodL;
                        if (isL) a.Lrow[Lbase + o] = idx; else a.Ucol[Ubase + o] = idx;
                        if (atomicExch(last + tb, K) != K) {
                            const int pos = atomicAdd(pc + tb, 1);
                            if (pos < a.prodcap) pl[(int64_t)tb * a.prodcap + pos] = K;
                            else set_status(a.status, DEV_PROD_OVERFLOW, a.info, K);
                        }
                    }
                }
            }
            carry += tot;
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(NT, 1) bilu_factor_kernel(FactorArgs a) {
    extern __shared__ __align__(16) char smem[];
    const uint32_t G = a.G + a.debug_extra_cta;
    for (int K = 0; K < a.nb; ++K) {
        const int s0 = a.bstart[K], s1 = a.bstart[K + 1];
        const int b = s1 - s0;
        // A: candidate sets (CTA 0: L side, CTA 1 % G: U side)
        if (blockIdx.x == 0) phase_A(a, K, true, smem);
        if (blockIdx.x == (1 % a.G)) {
            __syncthreads();
            phase_A(a, K, false, smem);
        }
        if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 1)) return;
        // B: accumulation tiles
        {
            const int mL = ldcg(a.kst + 0), mU = ldcg(a.kst + 1);
            int TR = (mL + mU + a.G - 1) / a.G;
            TR = max(4, min(TRMAX, TR));
            const int nLt = (mL + TR - 1) / TR, nUt = (mU + TR - 1) / TR;
            for (int it = blockIdx.x; it < nLt + nUt; it += a.G) {
                const bool Ls = it < nLt;
                const int sa = (Ls ? it : it - nLt) * TR;
                const int cnt = min(TR, (Ls ? mL : mU) - sa);
                phase_B_tile(a, K, Ls, sa, cnt, smem);
                __syncthreads();
            }
        }
        if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 2)) return;
        if (blockIdx.x == 0) phase_C(a, K, smem);
        if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 3)) return;
        phase_C2(a, K, smem);
        if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 4)) return;
        phase_D(a, K, smem);
        if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 5)) return;
        phase_E(a, K, smem);
        if (!grid_barrier(a.bar, G, a.status, a.spin_limit, a.info, 6)) return;
        (void)b;
    }
}

}  // namespace

// ---------------------------------------------------------------- host side

void factor_free(bilu_ctx *c) {
    dev_free(c->d_Lptr); dev_free(c->d_Lvptr); dev_free(c->d_Uptr); dev_free(c->d_Uvptr);
    dev_free(c->d_Lrow); dev_free(c->d_Ucol); dev_free(c->d_Lval); dev_free(c->d_Uval);
    dev_free(c->d_Dinv); dev_free(c->d_Pblk);
    dev_free(c->d_prodL); dev_free(c->d_prodLcnt); dev_free(c->d_prodU); dev_free(c->d_prodUcnt);
    dev_free(c->d_lastL); dev_free(c->d_lastU);
    dev_free(c->d_TL); dev_free(c->d_TU); dev_free(c->d_rowsL); dev_free(c->d_rowsU);
    dev_free(c->d_keepL); dev_free(c->d_keepU); dev_free(c->d_bmL); dev_free(c->d_bmU);
    dev_free(c->d_LU); dev_free(c->d_perm); dev_free(c->d_kstate); dev_free(c->d_status);
    dev_free(c->d_info); dev_free(c->d_bar);
    dev_free(c->d_wbL); dev_free(c->d_wbU); dev_free(c->d_xslotL); dev_free(c->d_xslotU);
    dev_free(c->d_pinfoL); dev_free(c->d_pinfoU);
    c->capLrow = c->capLval = c->capUcol = c->capUval = 0;
}

namespace {

cudaError_t alloc_pools(bilu_ctx *c) {
    cudaError_t e;
    dev_free(c->d_Lrow); dev_free(c->d_Ucol); dev_free(c->d_Lval); dev_free(c->d_Uval);
    if ((e = dev_alloc(&c->d_Lrow, c->capLrow)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Ucol, c->capUcol)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Lval, c->capLval)) != cudaSuccess) return e;
    if ((e = dev_alloc(&c->d_Uval, c->capUval)) != cudaSuccess) return e;
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
    cudaError_t e = cudaSuccess;
    if ((e = dev_alloc(&c->d_Lptr, nb + 1)) != cudaSuccess || (e = dev_alloc(&c->d_Lvptr, nb + 1)) != cudaSuccess ||
        (e = dev_alloc(&c->d_Uptr, nb + 1)) != cudaSuccess || (e = dev_alloc(&c->d_Uvptr, nb + 1)) != cudaSuccess ||
        (e = dev_alloc(&c->d_Dinv, nd)) != cudaSuccess || (e = dev_alloc(&c->d_Pblk, nd)) != cudaSuccess ||
        (e = dev_alloc(&c->d_prodLcnt, nb)) != cudaSuccess || (e = dev_alloc(&c->d_prodUcnt, nb)) != cudaSuccess ||
        (e = dev_alloc(&c->d_lastL, nb)) != cudaSuccess || (e = dev_alloc(&c->d_lastU, nb)) != cudaSuccess ||
        (e = dev_alloc(&c->d_TL, c->capT * bmax)) != cudaSuccess ||
        (e = dev_alloc(&c->d_TU, c->capT * bmax)) != cudaSuccess ||
        (e = dev_alloc(&c->d_rowsL, c->capT)) != cudaSuccess || (e = dev_alloc(&c->d_rowsU, c->capT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_keepL, c->capT)) != cudaSuccess || (e = dev_alloc(&c->d_keepU, c->capT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_bmL, n / 32 + 2)) != cudaSuccess || (e = dev_alloc(&c->d_bmU, n / 32 + 2)) != cudaSuccess ||
        (e = dev_alloc(&c->d_wbL, n / 32 + 2)) != cudaSuccess || (e = dev_alloc(&c->d_wbU, n / 32 + 2)) != cudaSuccess ||
        (e = dev_alloc(&c->d_LU, BILU_MAX_BLOCK * BILU_MAX_BLOCK)) != cudaSuccess ||
        (e = dev_alloc(&c->d_perm, BILU_MAX_BLOCK)) != cudaSuccess || (e = dev_alloc(&c->d_kstate, 16)) != cudaSuccess ||
        (e = dev_alloc(&c->d_status, 4)) != cudaSuccess || (e = dev_alloc(&c->d_info, INFO_COUNT)) != cudaSuccess ||
        (e = dev_alloc(&c->d_bar, 4)) != cudaSuccess || (e = alloc_pools(c)) != cudaSuccess ||
        (e = alloc_prod(c)) != cudaSuccess) {
        factor_free(c);
        return e == cudaErrorMemoryAllocation ? set_err(c, BILU_ERR_OOM, "device allocation failed in factor")
                                              : cuda_err(c, e, "factor allocation");
    }
    return BILU_OK;
}

int g_debug_extra_cta = 0;  // test hook (bilu_debug_set): barrier waits for a CTA that never arrives
long long g_debug_spin_limit = 0;

bilu_status factor_run(bilu_ctx *c, double droptol) {
    if (c->d_Lptr == nullptr) {
        bilu_status st = factor_alloc(c);
        if (st != BILU_OK) return st;
    }
    BILU_CUDA(c, cudaFuncSetAttribute(bilu_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    int per_sm = 0;
    BILU_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bilu_factor_kernel, NT, SMEM_BYTES));
    if (per_sm < 1) return set_err(c, BILU_ERR_CUDA, "factor kernel cannot be resident");
    const int G = c->nsm;  // one CTA per SM

    cudaEvent_t e0, e1;
    BILU_CUDA(c, cudaEventCreate(&e0));
    BILU_CUDA(c, cudaEventCreate(&e1));
    for (int attempt = 0; attempt < 12; ++attempt) {
        const int64_t nb = std::max<int64_t>(c->nb, 1), n = std::max<int64_t>(c->n, 1);
        BILU_CUDA(c, cudaMemsetAsync(c->d_Lptr, 0, (nb + 1) * sizeof(int64_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_Lvptr, 0, (nb + 1) * sizeof(int64_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_Uptr, 0, (nb + 1) * sizeof(int64_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_Uvptr, 0, (nb + 1) * sizeof(int64_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_prodLcnt, 0, nb * sizeof(int32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_prodUcnt, 0, nb * sizeof(int32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_lastL, 0xff, nb * sizeof(int32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_lastU, 0xff, nb * sizeof(int32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_bmL, 0, (n / 32 + 2) * sizeof(uint32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_bmU, 0, (n / 32 + 2) * sizeof(uint32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int32_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_info, 0, INFO_COUNT * sizeof(int64_t), c->stream));
        BILU_CUDA(c, cudaMemsetAsync(c->d_bar, 0, 4 * sizeof(uint32_t), c->stream));

        FactorArgs a{};
        a.n = (int32_t)c->n; a.nb = c->nb; a.G = G; a.perturb = c->p.perturb;
        a.tau = droptol; a.alpha = c->alpha; a.pert_tau = c->p.pert_tau; a.pert_rho = c->p.pert_rho;
        a.spin_limit = g_debug_spin_limit > 0 ? g_debug_spin_limit : (1LL << 24);
        a.rowptr = c->d_rowptr; a.colind = c->d_colind; a.colptr = c->d_colptr; a.rowind = c->d_rowind;
        a.bstart = c->d_bstart; a.blkof = c->d_blkof; a.val = c->d_val; a.cval = c->d_cval; a.Dptr = c->d_Dptr;
        a.Lptr = c->d_Lptr; a.Lvptr = c->d_Lvptr; a.Uptr = c->d_Uptr; a.Uvptr = c->d_Uvptr;
        a.Lrow = c->d_Lrow; a.Ucol = c->d_Ucol; a.Lval = c->d_Lval; a.Uval = c->d_Uval;
        a.Dinv = c->d_Dinv; a.Pblk = c->d_Pblk;
        a.capLrow = c->capLrow; a.capLval = c->capLval; a.capUcol = c->capUcol; a.capUval = c->capUval;
        a.prodcap = c->prodcap;
        a.prodL = c->d_prodL; a.prodLcnt = c->d_prodLcnt; a.prodU = c->d_prodU; a.prodUcnt = c->d_prodUcnt;
        a.lastL = c->d_lastL; a.lastU = c->d_lastU;
        a.TL = c->d_TL; a.TU = c->d_TU; a.rowsL = c->d_rowsL; a.rowsU = c->d_rowsU;
        a.keepL = c->d_keepL; a.keepU = c->d_keepU; a.bmL = c->d_bmL; a.bmU = c->d_bmU;
        a.wbL = c->d_wbL; a.wbU = c->d_wbU; a.xslotL = c->d_xslotL; a.xslotU = c->d_xslotU;
        a.capXS = c->capXS; a.pinfoL = c->d_pinfoL; a.pinfoU = c->d_pinfoU; a.capT = c->capT;
        a.LU = c->d_LU; a.perm = c->d_perm; a.kst = c->d_kstate; a.status = c->d_status; a.info = c->d_info;
        a.bar = c->d_bar;
        a.debug_extra_cta = g_debug_extra_cta;

        void *args[] = {&a};
        BILU_CUDA(c, cudaEventRecord(e0, c->stream));
        if (c->nb > 0)
            BILU_CUDA(c, cudaLaunchCooperativeKernel((void *)bilu_factor_kernel, dim3(G), dim3(NT), args,
                                                     SMEM_BYTES, c->stream));
        BILU_CUDA(c, cudaEventRecord(e1, c->stream));
        int32_t status = 0;
        int64_t info[INFO_COUNT];
        BILU_CUDA(c, cudaMemcpyAsync(&status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        BILU_CUDA(c, cudaMemcpyAsync(info, c->d_info, sizeof(info), cudaMemcpyDeviceToHost, c->stream));
        BILU_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->t_factor_ms = ms;
        if (status == DEV_POOL_OVERFLOW) {
            c->capLval *= 2; c->capUval *= 2; c->capLrow *= 2; c->capUcol *= 2;
            cudaError_t ee = alloc_pools(c);
            if (ee != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return set_err(c, BILU_ERR_OOM, "growing L/U pools failed"); }
            c->pool_retries++;
            continue;
        }
        if (status == DEV_PROD_OVERFLOW) {
            if (c->prodcap * 2 > PMAX) { cudaEventDestroy(e0); cudaEventDestroy(e1); return set_err(c, BILU_ERR_OOM, "more than 1024 producer blocks for one block"); }
            c->prodcap *= 2;
            c->capXS *= 2;
            cudaError_t ee = alloc_prod(c);
            if (ee != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return set_err(c, BILU_ERR_OOM, "growing producer lists failed"); }
            c->pool_retries++;
            continue;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (status == DEV_TIMEOUT) return set_err(c, BILU_ERR_TIMEOUT, "factor kernel: bounded wait gave up (site " + std::to_string(info[INFO_TIMEOUT_SITE]) + ")");
        if (status == DEV_SINGULAR) return set_err(c, BILU_ERR_SINGULAR, "singular diagonal block " + std::to_string(info[INFO_FAIL_BLOCK]));
        if (status == DEV_INTERNAL) return set_err(c, BILU_ERR_CUDA, "factor kernel index check failed at block " + std::to_string(info[INFO_FAIL_BLOCK]));
        if (status != DEV_OK) return set_err(c, BILU_ERR_CUDA, "factor kernel status " + std::to_string(status));
        // results
        int64_t tails[4];
        BILU_CUDA(c, cudaMemcpy(&tails[0], c->d_Lptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
        BILU_CUDA(c, cudaMemcpy(&tails[1], c->d_Lvptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
        BILU_CUDA(c, cudaMemcpy(&tails[2], c->d_Uptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
        BILU_CUDA(c, cudaMemcpy(&tails[3], c->d_Uvptr + c->nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
        c->kept_rows = tails[0]; c->nnz_l = tails[1]; c->kept_cols = tails[2]; c->nnz_u = tails[3];
        c->cand_rows = info[INFO_CAND_ROWS]; c->cand_cols = info[INFO_CAND_COLS];
        c->nperturb = info[INFO_NPERTURB];
        return c->nperturb > 0 ? BILU_PERTURBED : BILU_OK;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return set_err(c, BILU_ERR_OOM, "factor: too many pool re-runs");
}
