// Preconditioner application for callers that cannot allocate device memory.
//
// bilu_apply relies on device buffers the context allocated when the factor was computed
// (completion flags, sweep tickets, the forward-sweep plan) and, for host vectors, on
// staging buffers allocated on first use.  Some callers cannot allocate at the moment they
// apply the preconditioner: programs whose device memory is owned by a fixed pool or by
// another framework's allocator, and real-time loops that must not enter the allocator.
// bilu_apply_noalloc serves them: it allocates nothing.  Its only scratch is the fixed array
// below; the forward plan is recomputed inside the kernel by searching the kept row lists.
// A bounded wait that gives up ends the sweeps early; a last small kernel then fills z with
// NaN, so that a timeout cannot pass for a result.
//
// The scratch is one file-scope __device__ array, so every GPU that loads the library holds
// it until the process exits, and all calls on a device share it: calls that overlap on
// the GPU (different streams, or different contexts at the same time) race.
#include <mutex>

#include "dev_common.cuh"

extern int g_debug_extra_cta;         // test hooks (bilu_debug_set)
extern long long g_debug_spin_limit;

namespace {

constexpr int NA_MAX_BLOCKS = 65536;  // diagonal blocks the fixed scratch can serve
constexpr int NT = 512;
constexpr int NW = NT / 32;
constexpr int FCH = 32;               // producers per chunk of the forward sweep
constexpr long long NA_SPIN = 1LL << 22;

struct NoAllocScratch {
    int32_t flagF[NA_MAX_BLOCKS];  // forward sweep: block done
    int32_t flagB[NA_MAX_BLOCKS];  // backward sweep: block done
    int32_t st[8];                 // [1] forward ticket, [2] backward ticket, [3] status
};

// 512 KB + 32 bytes on every device that loads the library.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int NA_MAX_DEVICES = 64;
NoAllocScratch *g_scratch_addr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

struct NaArgs {
    int32_t nb, prodcap;
    const int32_t *bstart, *blkof;
    const int64_t *Lptr, *Lvptr, *Uptr, *Uvptr, *Dptr;
    const int32_t *Lrow, *Ucol;
    const double *Lval, *Uval, *Dinv;
    const int32_t *prodU, *prodUcnt;
    const double *r;
    double *z;
    NoAllocScratch *sc;
    long long spin;       // polls before a wait gives up
    int32_t debug_wait;   // test hook: block 0 of the forward sweep waits for a flag nothing sets
};

__device__ __forceinline__ bool na_wait(const int32_t *flag, int32_t *status, long long spin) {
    long long it = 0;
    while (ld_acquire_s32(flag) < 1) {
        if (++it > spin) {
            atomicCAS(status, 0, DEV_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// Forward sweep y_K = r_K - sum_J L_J(rows in B_K, :) y_J (Sec. 2.2), blocks claimed in
// increasing order; the rows of L_J inside B_K are found by warp searches.
__global__ void __launch_bounds__(NT) na_forward_kernel(NaArgs a) {
    __shared__ double acc[BILU_MAX_BLOCK];
    __shared__ double dmat[FCH][BILU_MAX_BLOCK];
    __shared__ int sJ[FCH], sps[FCH], soff[FCH + 1], sbJ[FCH], ssJ[FCH];
    __shared__ int64_t sLv[FCH];
    __shared__ int s_K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t *st = a.sc->st;
    while (true) {
        if (tid == 0) s_K = atomicAdd(st + 1, 1);
        __syncthreads();
        const int K = s_K;
        __syncthreads();
        if (K >= a.nb) return;
        if (a.debug_wait && K == 0) {  // flagF[nb] is cleared by the call and never set
            const int ok = tid == 0 ? (na_wait(a.sc->flagF + a.nb, st + 3, a.spin) ? 1 : 0) : 1;
            if (!__syncthreads_and(ok)) return;
        }
        const int s0 = a.bstart[K], s1 = a.bstart[K + 1], b = s1 - s0;
        if (tid < b) acc[tid] = a.r[s0 + tid];
        const int pc = a.prodUcnt[K];
        for (int c0 = 0; c0 < pc; c0 += FCH) {
            const int cn = min(FCH, pc - c0);
            int ok = 1;
            if (tid < cn) {
                const int J = a.prodU[(int64_t)K * a.prodcap + c0 + tid];
                sJ[tid] = J;
                ok = na_wait(a.sc->flagF + J, st + 3, a.spin) ? 1 : 0;
            }
            if (!__syncthreads_and(ok)) return;
            for (int t = warp; t < cn; t += NW) {
                const int J = sJ[t];
                const int l0 = (int)a.Lptr[J], l1 = (int)a.Lptr[J + 1];
                const int ps = warp_lower_bound(a.Lrow, l0, l1, s0);
                const int pe = warp_lower_bound(a.Lrow, ps, l1, s1);
                if (lane == 0) {
                    const int sj = a.bstart[J], bJ = a.bstart[J + 1] - sj;
                    sps[t] = ps;
                    soff[t + 1] = pe - ps;
                    ssJ[t] = sj;
                    sbJ[t] = bJ;
                    sLv[t] = a.Lvptr[J] + (int64_t)(ps - l0) * bJ;
                }
            }
            __syncthreads();
            if (tid == 0) {
                soff[0] = 0;
                for (int t = 0; t < cn; ++t) soff[t + 1] += soff[t];
            }
            for (int e = tid; e < cn * BILU_MAX_BLOCK; e += NT) (&dmat[0][0])[e] = 0.0;
            __syncthreads();
            const int nrows = soff[cn];
            for (int it = warp; it < nrows; it += NW) {
                int t = 0;
                while (soff[t + 1] <= it) ++t;
                const int bJ = sbJ[t];
                const double *row = a.Lval + sLv[t] + (int64_t)(it - soff[t]) * bJ;
                const double *yJ = a.z + ssJ[t];
                double v = 0.0;
                if (lane < bJ) v = row[lane] * ldcg(yJ + lane);
                if (lane + 32 < bJ) v = fma(row[lane + 32], ldcg(yJ + lane + 32), v);
                v = warp_sum(v);
                if (lane == 0) dmat[t][a.Lrow[sps[t] + (it - soff[t])] - s0] = v;
            }
            __syncthreads();
            if (tid < b) {
                double s = acc[tid];
                for (int t = 0; t < cn; ++t) s -= dmat[t][tid];
                acc[tid] = s;
            }
            __syncthreads();
        }
        if (tid < b) a.z[s0 + tid] = acc[tid];
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release_s32(a.sc->flagF + K, 1);
        }
    }
}

// Backward sweep z_K = D_K (y_K - U-breve_K(:, C_K) z(C_K)), blocks claimed last to first.
__global__ void __launch_bounds__(NT) na_backward_kernel(NaArgs a) {
    constexpr int NG = NT / BILU_MAX_BLOCK;
    __shared__ double part[NG][BILU_MAX_BLOCK];
    __shared__ double tv[BILU_MAX_BLOCK];
    __shared__ int s_K, s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t *st = a.sc->st;
    while (true) {
        if (tid == 0) s_K = atomicAdd(st + 2, 1);
        __syncthreads();
        const int K = a.nb - 1 - s_K;
        __syncthreads();
        if (K < 0) return;
        const int s0 = a.bstart[K], b = a.bstart[K + 1] - s0;
        const int64_t q0 = a.Uptr[K], q1 = a.Uptr[K + 1];
        if (warp == 0) {
            int ok = 1, last = -1;
            for (int64_t qb = q0; qb < q1; qb += 32) {
                const int64_t q = qb + lane;
                const int blk = q < q1 ? a.blkof[a.Ucol[q]] : -1;
                int prev = __shfl_up_sync(FULL_MASK, blk, 1);
                if (lane == 0) prev = last;
                const bool first = q < q1 && blk != prev;
                int okl = 1;
                if (first) okl = na_wait(a.sc->flagB + blk, st + 3, a.spin) ? 1 : 0;
                ok = ok && __all_sync(FULL_MASK, okl);
                last = __shfl_sync(FULL_MASK, blk, 31);
                if (!ok) break;
            }
            if (lane == 0) s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        const int g = tid / BILU_MAX_BLOCK, rr = tid % BILU_MAX_BLOCK;
        double s = 0.0;
        if (rr < b) {
            const double *Uv = a.Uval + a.Uvptr[K];
            for (int64_t q = q0 + g; q < q1; q += NG) s = fma(Uv[(q - q0) * b + rr], ldcg(a.z + a.Ucol[q]), s);
        }
        part[g][rr] = s;
        __syncthreads();
        if (tid < b) {
            double t = ldcg(a.z + s0 + tid);
            for (int gg = 0; gg < NG; ++gg) t -= part[gg][tid];
            tv[tid] = t;
        }
        __syncthreads();
        const double *D = a.Dinv + a.Dptr[K];
        const double t0 = lane < b ? tv[lane] : 0.0, t1 = lane + 32 < b ? tv[lane + 32] : 0.0;
        for (int r = warp; r < b; r += NW) {
            double v = 0.0;
            if (lane < b) v = D[(int64_t)r * b + lane] * t0;
            if (lane + 32 < b) v = fma(D[(int64_t)r * b + lane + 32], t1, v);
            v = warp_sum(v);
            if (lane == 0) a.z[s0 + r] = v;
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release_s32(a.sc->flagB + K, 1);
        }
    }
}

// After the sweeps: when a wait gave up, z is incomplete; every entry becomes NaN.
__global__ void __launch_bounds__(256) na_finish_kernel(NaArgs a, int64_t n) {
    if (ldcg(a.sc->st + 3) == DEV_OK) return;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a.z[i] = nan;
}

bool na_is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" bilu_status bilu_apply_noalloc(bilu_ctx *c, const double *r, double *z) {
    if (!c) return BILU_ERR_ARG;
    if (c->state < 2) return set_err(c, BILU_ERR_STATE, "bilu_apply_noalloc before bilu_factor");
    if (c->n == 0) return BILU_OK;
    if (!r || !z) return set_err(c, BILU_ERR_ARG, "null vector");
    if (r == z) return set_err(c, BILU_ERR_ARG, "r and z must not overlap");
    if (c->p.precision != BILU_PREC_FP64)
        return set_err(c, BILU_ERR_ARG, "bilu_apply_noalloc serves FP64 factors (use bilu_apply)");
    if (c->nb > NA_MAX_BLOCKS)
        return set_err(c, BILU_ERR_ARG, "bilu_apply_noalloc serves at most 65536 diagonal blocks; this factor has " +
                                            std::to_string(c->nb) + " (use bilu_apply)");
    if (c->device < 0 || c->device >= NA_MAX_DEVICES) return set_err(c, BILU_ERR_ARG, "device index too large");
    BILU_CUDA(c, cudaSetDevice(c->device));
    if (!na_is_device_ptr(r) || !na_is_device_ptr(z))
        return set_err(c, BILU_ERR_ARG, "bilu_apply_noalloc needs device pointers (host vectors need staging buffers)");
    NoAllocScratch *sc = nullptr;
    {
        // first call on a device: look up the device address of the scratch array (host
        // code sees only a host-side stand-in under that name)
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[c->device]) {
            NoAllocScratch *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_err(c, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_scratch_addr[c->device] = p;
        }
        sc = g_scratch_addr[c->device];
    }
    // the array keeps the previous call's contents: clear the flags this factor uses and the
    // sweep state
    const bool debug_wait = g_debug_extra_cta && c->nb < NA_MAX_BLOCKS;
    BILU_CUDA(c, cudaMemsetAsync(sc->flagF, 0, (size_t)(c->nb + (debug_wait ? 1 : 0)) * sizeof(int32_t), c->stream));
    BILU_CUDA(c, cudaMemsetAsync(sc->flagB, 0, (size_t)c->nb * sizeof(int32_t), c->stream));
    BILU_CUDA(c, cudaMemsetAsync(sc->st, 0, sizeof(sc->st), c->stream));
    NaArgs a{};
    const FactorView v = factor_view(c);  // the merged blocks after progressive aggregation
    a.nb = c->nb;
    a.prodcap = v.prodcap;
    a.bstart = v.bstart;
    a.blkof = v.blkof;
    a.Lptr = v.Lptr; a.Lvptr = v.Lvptr; a.Uptr = v.Uptr; a.Uvptr = v.Uvptr; a.Dptr = v.Dptr;
    a.Lrow = v.Lrow; a.Ucol = v.Ucol; a.Lval = (const double *)v.Lval; a.Uval = (const double *)v.Uval;
    a.Dinv = v.Dinv;
    a.prodU = v.prodU; a.prodUcnt = v.prodUcnt;
    a.r = r;
    a.z = z;
    a.sc = sc;
    a.spin = g_debug_spin_limit > 0 ? g_debug_spin_limit : NA_SPIN;
    a.debug_wait = debug_wait ? 1 : 0;
    const int G = c->nsm * 2;
    na_forward_kernel<<<G, NT, 0, c->stream>>>(a);
    na_backward_kernel<<<G, NT, 0, c->stream>>>(a);
    na_finish_kernel<<<c->nsm, 256, 0, c->stream>>>(a, c->n);
    c->launches += 3;
    BILU_CUDA(c, cudaGetLastError());
    return BILU_OK;
}
