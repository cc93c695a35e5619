// Preconditioner application z = M^{-1} r, M = L D^{-1} U (Sec. 2.2).
//
// Forward:  y_K = r_K - sum_J L_J(rows in B_K, :) y_J    (unit block lower L, gather form)
// Backward: z_K = D_K ( y_K - U-breve_K(:, C_K) z(C_K) ) (K from last to first)
// Both sweeps are persistent kernels: CTAs claim blocks in sweep order from a ticket
// counter and wait (bounded) on per-block completion flags of the blocks they read, so
// independent blocks of the block-dependency DAG run concurrently.  Summation orders are
// fixed (producers in increasing J, fixed per-thread partial sums), so results are
// bitwise reproducible.
#include <algorithm>

#include "dev_common.cuh"

namespace {

constexpr int AT = 512;        // threads per CTA
constexpr int AW = AT / 32;
constexpr long long APPLY_SPIN = 1LL << 22;

struct ApplyArgs {
    int32_t nb;
    const int32_t *bstart, *blkof;
    const int64_t *Lptr, *Lvptr, *Uptr, *Uvptr, *Dptr;
    const int32_t *Lrow, *Ucol;
    const void *Lval, *Uval;  // factor values, storage type TS of the kernel instance
    const void *Uhval;        // D_K U-breve_K, the layout of Uval (the backward sweep's columns)
    const double *Dinv;
    const int32_t *prodU, *prodUcnt;
    int32_t prodcap;
    const int2 *planF;     // per (K, t): L_J rows inside B_K
    const double *r;
    double *z;             // holds y after the forward sweep
    int32_t *flagF, *flagB;
    int32_t *st;           // [0] epoch, [1] forward ticket, [2] backward ticket, [3] status
    const int32_t *skip;   // optional: nonzero -> return immediately
};

// Arithmetic of the sweeps: FP64 for an FP64 factor; FP32 for the reduced-precision factors,
// whose stored values carry 8 (BF16) or 24 (FP32) significant bits, so FP32 products and sums
// (relative error ~2^-24 per operation) add nothing that the factor's own rounding does not
// already dominate.  The vectors r, y, z stay FP64 in memory; GMRES is FP64 throughout.
template <class TS> struct SweepT { using T = float; };
template <> struct SweepT<double> { using T = double; };
__device__ __forceinline__ float cval(float v) { return v; }
__device__ __forceinline__ float cval(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double cval(double v) { return v; }
__device__ __forceinline__ float warp_sum_t(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_t(double v) { return warp_sum(v); }

// The factor values a block will read, fetched into L2 while it waits for its dependencies
// (warp-cooperative, one 128-byte line per lane and step).
__device__ __forceinline__ void warp_prefetch_l2(const void *p, int64_t bytes) {
    const int lane = threadIdx.x & 31;
    const uintptr_t beg = (uintptr_t)p & ~(uintptr_t)127, end = (uintptr_t)p + (uintptr_t)bytes;
    for (uintptr_t q = beg + (uintptr_t)lane * 128; q < end; q += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}

__device__ __forceinline__ bool wait_flag(const int32_t *flag, int epoch, int32_t *status) {
    long long it = 0;
    while (ld_acquire_s32(flag) < epoch) {
        if (++it > APPLY_SPIN) {
            atomicCAS(status, 0, DEV_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

__global__ void __launch_bounds__(32) apply_begin_kernel(int32_t *st, const int32_t *skip) {
    if (skip && *skip) return;
    if (threadIdx.x == 0) {
        st[0] += 1;
        st[1] = 0;
        st[2] = 0;
    }
}

// Forward sweep, block K: the producers' metadata is loaded first; then, round by round, the
// rows of every producer that has completed are computed (dot products into dmat[t][r]) while
// the CTA waits (bounded) for the oldest producer still running, so that once the newest one
// (normally block K-1) is done little more than its rows lies on the sweep's critical path.  The rows are summed
// over the producers in increasing J (a fixed order, folded in as soon as a leading run of
// producers is done), so the result does not depend on the arrival order.
constexpr int FCH = 32;  // producers per chunk

template <class TS>
__global__ void __launch_bounds__(AT) apply_forward_kernel(ApplyArgs a) {
    using TC = typename SweepT<TS>::T;
    if (a.skip && ldcg(a.skip)) return;
    __shared__ TC acc[BILU_MAX_BLOCK];
    __shared__ TC dmat[FCH][BILU_MAX_BLOCK];
    __shared__ int sps[FCH], soff[FCH + 1], sbJ[FCH], ssJ[FCH], sJ[FCH], sst[FCH], scnt[FCH];
    __shared__ int srl[FCH], sro[FCH + 1];  // producers computed this round and their row offsets
    __shared__ int64_t sLv[FCH];
    __shared__ int s_K, s_ok, s_work, s_more, s_fold, s_nrd;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int epoch = ldcg(a.st);
    while (true) {
        if (tid == 0) s_K = atomicAdd(a.st + 1, 1);
        __syncthreads();
        const int K = s_K;
        __syncthreads();
        if (K >= a.nb) return;
        const int s0 = a.bstart[K], b = a.bstart[K + 1] - s0;
        if (tid < b) acc[tid] = (TC)a.r[s0 + tid];
        const int pc = ldcg(a.prodUcnt + K);
        for (int c0 = 0; c0 < pc; c0 += FCH) {
            const int cn = min(FCH, pc - c0);
            if (tid < cn) {
                const int J = ldcg(a.prodU + (int64_t)K * a.prodcap + c0 + tid);
                const int2 rg = a.planF[(int64_t)K * a.prodcap + c0 + tid];
                sps[tid] = rg.x;
                soff[tid + 1] = rg.y - rg.x;
                scnt[tid] = rg.y - rg.x;
                const int sj = a.bstart[J];
                ssJ[tid] = sj;
                sbJ[tid] = a.bstart[J + 1] - sj;
                sLv[tid] = a.Lvptr[J] + (int64_t)(rg.x - a.Lptr[J]) * (a.bstart[J + 1] - sj);
                sJ[tid] = J;
                sst[tid] = 0;  // 0 running, 1 to compute this round, 2 computed
            }
            if (tid == 0) s_fold = 0;
            for (int e = tid; e < cn * BILU_MAX_BLOCK; e += AT) (&dmat[0][0])[e] = TC(0);
            __syncthreads();
            if (tid == 0) {
                soff[0] = 0;
                for (int t = 0; t < cn; ++t) soff[t + 1] += soff[t];
            }
            // the chunk's L rows into L2 before the waits (warps 1.., one producer each)
            for (int t = warp - 1; warp > 0 && t < cn; t += AW - 1)
                warp_prefetch_l2((const TS *)a.Lval + sLv[t], (int64_t)scnt[t] * sbJ[t] * (int64_t)sizeof(TS));
            __syncthreads();
            while (true) {
                if (warp == 0) {
                    int st = lane < cn ? sst[lane] : 2;
                    if (st == 1) st = 2;  // computed in the previous round
                    bool rdy = st == 0 && ld_acquire_s32(a.flagF + sJ[lane]) >= epoch;
                    unsigned mr = __ballot_sync(FULL_MASK, rdy);
                    unsigned mw = __ballot_sync(FULL_MASK, st == 0 && !rdy);
                    int ok = 1;
                    if (mr == 0 && mw != 0) {
                        // nothing new: wait for the oldest running producer (producers finish
                        // in order, so each round takes the ones completed meanwhile and only
                        // the newest is left once it is done); when it is the only one left it
                        // is taken at once, otherwise all are re-checked
                        const int tw = __ffs(mw) - 1;
                        if (lane == 0) ok = wait_flag(a.flagF + sJ[tw], epoch, a.st + 3) ? 1 : 0;
                        ok = __shfl_sync(FULL_MASK, ok, 0);
                        if (ok && __popc(mw) == 1 && lane == tw) rdy = true;
                        mr = __ballot_sync(FULL_MASK, rdy);
                        mw = __ballot_sync(FULL_MASK, st == 0 && !rdy);
                    }
                    if (rdy) st = 1;
                    if (lane < cn) sst[lane] = st;
                    // the round's producers in order, with their row offsets
                    const int rows_l = rdy ? soff[lane + 1] - soff[lane] : 0;
                    const int inc = warp_incl_scan(rows_l);
                    const int k = __popc(mr & ((1u << lane) - 1u));
                    if (rdy) {
                        srl[k] = lane;
                        sro[k] = inc - rows_l;
                    }
                    if (lane == 31) {
                        s_nrd = __popc(mr);
                        sro[__popc(mr)] = inc;
                    }
                    if (lane == 0) {
                        s_ok = ok;
                        s_work = mr != 0;
                        s_more = (mr | mw) != 0;
                    }
                }
                __syncthreads();
                if (!s_ok) return;
                // fold the leading run of computed producers into acc, in producer order
                if (tid < b) {
                    TC v = acc[tid];
                    int t = s_fold;
                    while (t < cn && sst[t] == 2) v -= dmat[t++][tid];
                    acc[tid] = v;
                }
                if (!s_more) break;
                // the rows of this round's producers only: four per warp and iteration, their
                // loads in flight together; row -> producer by binary search over the offsets
                const int nrd = s_nrd, nrr = sro[nrd];
                for (int it0 = warp * 4; it0 < nrr; it0 += AW * 4) {
                    TC v[4];
                    int tt[4], pp[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int it = it0 + u;
                        v[u] = TC(0);
                        tt[u] = -1;
                        if (it < nrr) {
                            int lo = 0, hi = nrd - 1;  // largest k with sro[k] <= it
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (sro[mid] <= it) lo = mid; else hi = mid - 1;
                            }
                            const int t = srl[lo], ir = it - sro[lo];
                            const int bJ = sbJ[t];
                            const TS *row = (const TS *)a.Lval + sLv[t] + (int64_t)ir * bJ;
                            const double *yJ = a.z + ssJ[t];
                            if (lane < bJ) v[u] = cval(row[lane]) * (TC)ldcg(yJ + lane);
                            if (lane + 32 < bJ) v[u] = fma(cval(row[lane + 32]), (TC)ldcg(yJ + lane + 32), v[u]);
                            tt[u] = t;
                            pp[u] = sps[t] + ir;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const TC w = warp_sum_t(v[u]);
                        if (lane == 0 && tt[u] >= 0) dmat[tt[u]][a.Lrow[pp[u]] - s0] = w;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int t = s_fold;
                    while (t < cn && sst[t] == 2) ++t;
                    s_fold = t;
                }
                __syncthreads();
            }
            __syncthreads();
        }
        if (tid < b) a.z[s0 + tid] = (double)acc[tid];
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release_s32(a.flagF + K, epoch);
        }
    }
}

// Backward sweep, block K: z_K = D_K y_K - (D_K U-breve_K) z(C_K).  D_K y_K is formed first,
// before any wait (y_K is final after the forward sweep), so only the columns of the normalised
// U (stored by the factor) lie on the sweep's critical path.  The kept columns in blocks after
// K+1 (complete early) are multiplied while block K+1 -- the newest dependency -- may still be
// running; its own columns (the leading range, the columns are sorted) follow once it is done.
// The partial sums are formed in a fixed order, so the result does not depend on timing.
template <class TS>
__device__ __forceinline__ typename SweepT<TS>::T backward_columns(const ApplyArgs &a, int K, int b, int64_t q0,
                                                                    int64_t qa, int64_t qb, int g, int rr) {
    using TC = typename SweepT<TS>::T;
    constexpr int NG = AT / BILU_MAX_BLOCK;  // column groups
    TC s = TC(0);
    if (rr < b) {
        const TS *Uv = (const TS *)a.Uhval + a.Uvptr[K];
        int64_t q = qa + g;
        // four independent columns per iteration keep several loads in flight
        TC s1 = TC(0), s2 = TC(0), s3 = TC(0);
        for (; q + 3 * NG < qb; q += 4 * NG) {
            const TC u0 = cval(Uv[(q - q0) * b + rr]), u1 = cval(Uv[(q + NG - q0) * b + rr]);
            const TC u2 = cval(Uv[(q + 2 * NG - q0) * b + rr]), u3 = cval(Uv[(q + 3 * NG - q0) * b + rr]);
            const TC z0 = (TC)ldcg(a.z + a.Ucol[q]), z1 = (TC)ldcg(a.z + a.Ucol[q + NG]);
            const TC z2 = (TC)ldcg(a.z + a.Ucol[q + 2 * NG]), z3 = (TC)ldcg(a.z + a.Ucol[q + 3 * NG]);
            s = fma(u0, z0, s);
            s1 = fma(u1, z1, s1);
            s2 = fma(u2, z2, s2);
            s3 = fma(u3, z3, s3);
        }
        for (; q < qb; q += NG) s = fma(cval(Uv[(q - q0) * b + rr]), (TC)ldcg(a.z + a.Ucol[q]), s);
        s = (s + s1) + (s2 + s3);
    }
    return s;
}

// Waits (warp 0, bounded) for the blocks holding the kept columns [qa, qb) (sorted, so each
// block forms one run; the first lane of a run waits on its flag).  Returns 0 on timeout.
__device__ __forceinline__ int wait_column_blocks(const ApplyArgs &a, int64_t qa, int64_t qb, int epoch) {
    const int lane = threadIdx.x & 31;
    int ok = 1, last = -1;
    for (int64_t qbase = qa; qbase < qb; qbase += 32) {
        const int64_t q = qbase + lane;
        const int blk = q < qb ? a.blkof[a.Ucol[q]] : -1;
        int prev = __shfl_up_sync(FULL_MASK, blk, 1);
        if (lane == 0) prev = last;
        const bool first = q < qb && blk != prev;
        int okl = 1;
        if (first) okl = wait_flag(a.flagB + blk, epoch, a.st + 3) ? 1 : 0;
        ok = ok && __all_sync(FULL_MASK, okl);
        last = __shfl_sync(FULL_MASK, blk, 31);
        if (!ok) break;
    }
    return ok;
}

constexpr int RMAX = 512;  // column runs (distinct later blocks) per block held in shared memory

template <class TS>
__global__ void __launch_bounds__(AT) apply_backward_kernel(ApplyArgs a) {
    using TC = typename SweepT<TS>::T;
    if (a.skip && ldcg(a.skip)) return;
    constexpr int NG = AT / BILU_MAX_BLOCK;  // column groups
    __shared__ TC part[NG][BILU_MAX_BLOCK];
    __shared__ TC tv[BILU_MAX_BLOCK], yv[BILU_MAX_BLOCK];
    __shared__ int32_t rq[RMAX + 1], rblk[RMAX];
    __shared__ int s_K, s_ok, s_nr, s_take;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int epoch = ldcg(a.st);
    while (true) {
        if (tid == 0) s_K = atomicAdd(a.st + 2, 1);
        __syncthreads();
        const int K = a.nb - 1 - s_K;
        __syncthreads();
        if (K < 0) return;
        const int s0 = a.bstart[K], b = a.bstart[K + 1] - s0;
        const int64_t q0 = a.Uptr[K], q1 = a.Uptr[K + 1];
        const int g = tid / BILU_MAX_BLOCK, rr = tid % BILU_MAX_BLOCK;
        if (tid < b) yv[tid] = (TC)ldcg(a.z + s0 + tid);
        // the normalised U columns into L2 before the waits
        if (warp == 1) warp_prefetch_l2((const TS *)a.Uhval + a.Uvptr[K], (q1 - q0) * b * (int64_t)sizeof(TS));
        __syncthreads();
        {
            // tv = D_K y_K: warp per row, four rows in flight
            const double *D = a.Dinv + a.Dptr[K];
            const TC y0 = lane < b ? yv[lane] : TC(0), y1 = lane + 32 < b ? yv[lane + 32] : TC(0);
            for (int r0 = warp * 4; r0 < b; r0 += AW * 4) {
                TC v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = r0 + u;
                    v[u] = TC(0);
                    if (r < b) {
                        if (lane < b) v[u] = (TC)D[(int64_t)r * b + lane] * y0;
                        if (lane + 32 < b) v[u] = fma((TC)D[(int64_t)r * b + lane + 32], y1, v[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const TC w = warp_sum_t(v[u]);
                    if (lane == 0 && r0 + u < b) tv[r0 + u] = w;
                }
            }
        }
        // runs of kept columns by block (the columns are sorted): run i = [rq[i], rq[i+1])
        if (warp == 0) {
            int nr = 0, last = -1;
            for (int64_t qbase = q0; qbase < q1 && nr <= RMAX; qbase += 32) {
                const int64_t q = qbase + lane;
                const int blk = q < q1 ? a.blkof[a.Ucol[q]] : -1;
                int prev = __shfl_up_sync(FULL_MASK, blk, 1);
                if (lane == 0) prev = last;
                const bool first = q < q1 && blk != prev;
                const unsigned m = __ballot_sync(FULL_MASK, first);
                const int pos = nr + __popc(m & ((1u << lane) - 1u));
                if (first && pos < RMAX) {
                    rq[pos] = (int32_t)(q - q0);
                    rblk[pos] = blk;
                }
                nr += __popc(m);
                last = __shfl_sync(FULL_MASK, blk, 31);
            }
            if (lane == 0) {
                s_nr = nr;
                if (nr <= RMAX) rq[nr] = (int32_t)(q1 - q0);
            }
        }
        __syncthreads();
        const int nr = s_nr;
        if (nr > RMAX) {
            // too many runs for the shared list: wait for all of them, then one pass
            if (warp == 0) {
                const int ok = wait_column_blocks(a, q0, q1, epoch);
                if (lane == 0) s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            part[g][rr] = backward_columns<TS>(a, K, b, q0, q0, q1, g, rr);
            __syncthreads();
            if (tid < b) {
                TC t = tv[tid];
                for (int gg = 0; gg < NG; ++gg) t -= part[gg][tid];
                tv[tid] = t;
            }
            __syncthreads();
        } else {
            // runs from the highest block down (the order in which the sweep completes them);
            // each round takes the completed ones, waiting (bounded) for the next when none is;
            // every run is summed over its columns in a fixed order and folded into t in run order
            int ri = nr - 1;
            while (ri >= 0) {
                if (warp == 0) {
                    const int r = ri - lane;
                    const bool rdy = r >= 0 && ld_acquire_s32(a.flagB + rblk[r]) >= epoch;
                    const unsigned m = __ballot_sync(FULL_MASK, rdy);
                    int take = __ffs(~m) - 1;  // leading completed runs
                    if (m == 0xffffffffu) take = 32;
                    int ok = 1;
                    if (take == 0) {
                        if (lane == 0) ok = wait_flag(a.flagB + rblk[ri], epoch, a.st + 3) ? 1 : 0;
                        ok = __shfl_sync(FULL_MASK, ok, 0);
                        take = 1;
                    }
                    if (lane == 0) {
                        s_ok = ok;
                        s_take = min(take, ri + 1);
                    }
                }
                __syncthreads();
                if (!s_ok) return;
                const int take = s_take;
                for (int j = 0; j < take; ++j) {
                    const int r = ri - j;
                    part[g][rr] = backward_columns<TS>(a, K, b, q0, q0 + rq[r], q0 + rq[r + 1], g, rr);
                    __syncthreads();
                    if (tid < b) {
                        TC t = tv[tid];
                        for (int gg = 0; gg < NG; ++gg) t -= part[gg][tid];
                        tv[tid] = t;
                    }
                    __syncthreads();
                }
                ri -= take;
            }
        }
        if (tid < b) a.z[s0 + tid] = (double)tv[tid];
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release_s32(a.flagB + K, epoch);
        }
    }
}

// Apply plan: for block K and its t-th forward producer J, the kept rows of L_J inside B_K.
__global__ void apply_plan_kernel(int32_t nb, int32_t prodcap, const int32_t *bstart, const int64_t *Lptr,
                                  const int32_t *Lrow, const int32_t *prodU, const int32_t *prodUcnt,
                                  int2 *planF) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t total = (int64_t)nb * prodcap;
    for (int64_t w = gw; w < total; w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int K = (int)(w / prodcap), t = (int)(w % prodcap);
        if (t >= prodUcnt[K]) continue;
        const int J = prodU[(int64_t)K * prodcap + t];
        const int s0 = bstart[K], s1 = bstart[K + 1];
        const int ps = warp_lower_bound(Lrow, (int)Lptr[J], (int)Lptr[J + 1], s0);
        const int pe = warp_lower_bound(Lrow, ps, (int)Lptr[J + 1], s1);
        if (lane == 0) planF[w] = make_int2(ps, pe);
    }
}

}  // namespace

void apply_free(bilu_ctx *c) {
    dev_free(c->d_planF);
    dev_free(c->d_flagF);
    dev_free(c->d_flagB);
    dev_free(c->d_apst);
    dev_free(c->d_stage_in);
    dev_free(c->d_stage_out);
}

bilu_status apply_alloc(bilu_ctx *c) {
    apply_free(c);
    const int64_t nb = std::max<int64_t>(c->nb, 1);
    if (dev_alloc(&c->d_flagF, nb) != cudaSuccess || dev_alloc(&c->d_flagB, nb) != cudaSuccess ||
        dev_alloc(&c->d_planF, nb * (int64_t)factor_view(c).prodcap) != cudaSuccess || dev_alloc(&c->d_apst, 8) != cudaSuccess) {
        apply_free(c);
        return set_err(c, BILU_ERR_OOM, "apply allocation failed");
    }
    BILU_CUDA(c, cudaMemsetAsync(c->d_flagF, 0, nb * sizeof(int32_t), c->stream));
    BILU_CUDA(c, cudaMemsetAsync(c->d_flagB, 0, nb * sizeof(int32_t), c->stream));
    BILU_CUDA(c, cudaMemsetAsync(c->d_apst, 0, 8 * sizeof(int32_t), c->stream));
    const FactorView v = factor_view(c);
    const int64_t warps = nb * v.prodcap;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((warps * 32 + threads - 1) / threads, 65535);
    if (c->nb > 0) {
        apply_plan_kernel<<<(unsigned)blocks, threads, 0, c->stream>>>(c->nb, v.prodcap, v.bstart, v.Lptr, v.Lrow,
                                                                     v.prodU, v.prodUcnt, c->d_planF);
        c->launches += 1;
    }
    BILU_CUDA(c, cudaGetLastError());
    return BILU_OK;
}

bilu_status apply_launch(bilu_ctx *c, const double *d_r, double *d_z, const int32_t *skip) {
    const FactorView v = factor_view(c);  // the merged blocks after progressive aggregation
    ApplyArgs a{};
    a.nb = c->nb;
    a.bstart = v.bstart;
    a.blkof = v.blkof;
    a.Lptr = v.Lptr; a.Lvptr = v.Lvptr; a.Uptr = v.Uptr; a.Uvptr = v.Uvptr; a.Dptr = v.Dptr;
    a.Lrow = v.Lrow; a.Ucol = v.Ucol; a.Lval = v.Lval; a.Uval = v.Uval; a.Dinv = v.Dinv;
    a.Uhval = v.Uhval;
    a.prodU = v.prodU; a.prodUcnt = v.prodUcnt; a.prodcap = v.prodcap;
    a.planF = c->d_planF;
    a.r = d_r;
    a.z = d_z;
    a.flagF = c->d_flagF;
    a.flagB = c->d_flagB;
    a.st = c->d_apst;
    a.skip = skip;
    const int G = c->apply_grid > 0 ? c->apply_grid : c->nsm * 2;
    apply_begin_kernel<<<1, 32, 0, c->stream>>>(c->d_apst, skip);
    if (c->p.precision == BILU_PREC_FP32) {
        apply_forward_kernel<float><<<G, AT, 0, c->stream>>>(a);
        apply_backward_kernel<float><<<G, AT, 0, c->stream>>>(a);
    } else if (c->p.precision == BILU_PREC_BF16) {
        apply_forward_kernel<__nv_bfloat16><<<G, AT, 0, c->stream>>>(a);
        apply_backward_kernel<__nv_bfloat16><<<G, AT, 0, c->stream>>>(a);
    } else {
        apply_forward_kernel<double><<<G, AT, 0, c->stream>>>(a);
        apply_backward_kernel<double><<<G, AT, 0, c->stream>>>(a);
    }
    c->launches += 3;
    BILU_CUDA(c, cudaGetLastError());
    return BILU_OK;
}

bilu_status apply_run(bilu_ctx *c, const double *d_r, double *d_z) { return apply_launch(c, d_r, d_z, nullptr); }
