// Device helpers shared by the library's kernels: cache-bypassing loads, warp and block
// reductions / scans, a bounded grid barrier for cooperative persistent kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bilu_internal.h"

#define FULL_MASK 0xffffffffu

// Loads of data written by other CTAs during the same launch: bypass L1 (which is not
// coherent across SMs), read from L2.
template <class T>
__device__ __forceinline__ T ldcg(const T *p) {
    return __ldcg(p);
}

// factor values of any storage precision, widened to FP64
__device__ __forceinline__ double dval(double v) { return v; }
__device__ __forceinline__ double dval(float v) { return (double)v; }
__device__ __forceinline__ double dval(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_acquire_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s32(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan over the block; returns the thread's exclusive prefix and writes the
// block total to *total.  `ws` is shared scratch of >= 33 ints.  All threads must call.
__device__ __forceinline__ int block_excl_scan(int v, int *ws, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int x = lane < nw ? ws[lane] : 0;
        int xi = warp_incl_scan(x);
        if (lane < nw) ws[lane] = xi - x;
        if (lane == nw - 1) ws[32] = xi;
    }
    __syncthreads();
    int res = inc - v + ws[warp];
    *total = ws[32];
    __syncthreads();
    return res;
}

// First position in sorted a[lo, hi) with a[pos] >= key, computed by a full warp
// (32-ary search: two dependent L2 round trips for lists of up to ~1000 entries).
__device__ __forceinline__ int warp_lower_bound(const int32_t *a, int lo, int hi, int key) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) >> 5;
        const int pos = lo + lane * step;
        const bool ge = (pos < hi) ? (ldcg(a + pos) >= key) : true;
        const unsigned m = __ballot_sync(FULL_MASK, ge);
        if (m == 0) {  // every probe < key: the answer lies after the last probe
            lo = lo + 31 * step + 1;
            continue;
        }
        const int f = __ffs(m) - 1;
        if (f == 0) return lo;
        const int nlo = lo + (f - 1) * step + 1;
        const int nhi = min(hi, lo + f * step);
        lo = nlo;
        hi = nhi;
    }
    const int pos = lo + lane;
    const bool ge = (pos < hi) ? (ldcg(a + pos) >= key) : true;
    const unsigned m = __ballot_sync(FULL_MASK, ge);
    return m ? lo + __ffs(m) - 1 : hi;
}

// Bounded grid barrier for a cooperative launch of G CTAs.  bar[0] counts arrivals,
// bar[1] is the generation, bar[2] the status word as the last arriving CTA read it.  Every
// CTA takes its exit decision from that snapshot, so all of them leave at the same barrier
// even when one CTA raises an error in the next phase while another is still on its way out
// of this one.  A wait that exceeds spin_limit polls records DEV_TIMEOUT (after which the
// barrier's state is undefined: a timeout ends the launch).  Returns false (uniformly in the
// CTA, and across the CTAs) when the status snapshot holds an error.
__device__ __forceinline__ uint32_t atom_add_acqrel_u32(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_add_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_barrier(uint32_t *bar, uint32_t G, int32_t *status,
                                             long long spin_limit, int64_t *info, int site,
                                             volatile int32_t *heartbeat = nullptr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t gen = ld_acquire_u32(bar + 1);
        // acq_rel: this CTA's writes (ordered before by __syncthreads) are released, and the
        // last arriver acquires everything the others released, including their status writes
        const uint32_t arrived = atom_add_acqrel_u32(bar, 1u);
        if (arrived == G - 1) {
            const int32_t st = ld_acquire_s32(status);
            st_relaxed_u32(bar + 2, (uint32_t)st);
            atomicExch(bar, 0u);
            red_add_release_u32(bar + 1, 1u);  // publishes the snapshot with the new generation
            ok = st == DEV_OK;
        } else {
            long long it = 0;
            while (ld_acquire_u32(bar + 1) == gen) {
                if (++it > spin_limit) {
                    if (atomicCAS(status, 0, DEV_TIMEOUT) == 0) info[INFO_TIMEOUT_SITE] = site;
                    ok = 0;
                    break;
                }
                if (heartbeat && (it & 1023) == 0) *heartbeat = (int32_t)(it >> 10);  // test hook
                if (it > 64) __nanosleep(32);
            }
            // the snapshot cannot be overwritten before this CTA arrives at the next barrier
            if (ok) ok = (int32_t)ld_relaxed_u32(bar + 2) == DEV_OK;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// 1/p by Newton-Raphson iteration on f(x) = 1/x - p (x <- x + x (1 - p x), each step about
// doubles the number of correct bits).  The start value is the single-precision reciprocal of
// the top 23 bits of p's mantissa, formed and widened by integer bit operations (FP64 <-> FP32
// conversions issue on the slow FP64 pipe of this GPU); its relative error is below 2^-22, so
// two steps reach double precision.  The exponent is handled exactly by bit manipulation.
// Within about one ulp of the IEEE quotient; four dependent FP64 FMAs instead of a full
// division (a divide has a ~650-cycle latency on this GPU).  Values far from 1 in magnitude
// (including 0, inf, NaN) use the IEEE division.
__device__ __forceinline__ double recip_nr(double p) {
    const long long bits = __double_as_longlong(p);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex < 64 || ex > 1982) return 1.0 / p;
    const long long mb = bits & 0xfffffffffffffLL;
    const double m = __longlong_as_double(mb | (1023LL << 52) | (bits & (1LL << 63)));  // |m| in [1, 2), sign of p
    const float m32 = __int_as_float((int)(0x3f800000u | (unsigned)(mb >> 29) | ((unsigned)(bits >> 32) & 0x80000000u)));
    const unsigned xb = (unsigned)__float_as_int(__frcp_rn(m32));
    double x = __longlong_as_double(((long long)(xb & 0x80000000u) << 32) |
                                    ((long long)(((xb >> 23) & 0xff) - 127 + 1023) << 52) |
                                    ((long long)(xb & 0x7fffff) << 29));
    double e = fma(-m, x, 1.0);
    x = fma(x, e, x);
    e = fma(-m, x, 1.0);
    x = fma(x, e, x);
    return x * __longlong_as_double((long long)(2046 - ex) << 52);  // times 2^(1023 - ex)
}

__device__ __forceinline__ void set_status(int32_t *status, int code, int64_t *info, int64_t where) {
    if (atomicCAS(status, 0, code) == 0) info[INFO_FAIL_BLOCK] = where;
}
