// Right-preconditioned restarted GMRES(m) on the GPU (Saad and Schultz; the paper's
// experiments use GMRES(30), Sec. 4).
//
// A x = b is solved as A M^{-1} u = b, x = x0 + M^{-1} V y.  Arnoldi orthogonalises by
// classical Gram-Schmidt applied twice; the small least-squares problem is reduced with
// Givens rotations on the device.  One restart cycle (m Arnoldi steps, the update of x and
// the true residual) is captured once into a CUDA graph; every kernel of a step returns
// immediately once the cycle has converged, so the host synchronizes once per cycle.  All
// reductions use per-CTA partial sums combined in a fixed order, so results are bitwise
// reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dev_common.cuh"

namespace {

constexpr int VT = 256;   // threads per CTA of the vector kernels
constexpr int GMRES_MAX_RESTART = 1000;  // largest restart length m
enum { GI_ITS = 0, GI_JDONE, GI_DONE, GI_MAXIT, GI_M, GI_STOP, GI_COUNT = 8 };
enum { GS_BNORM = 0, GS_BETA, GS_TOL, GS_REL, GS_RELEST, GS_COUNT = 8 };

struct GmLayout {
    int m;
    int64_t H, g, cs, sn, y, scal, total;
    explicit GmLayout(int m_) : m(m_) {
        H = 0;
        g = H + (int64_t)(m + 1) * m;
        cs = g + m + 1;
        sn = cs + m;
        y = sn + m;
        scal = y + m;
        total = scal + GS_COUNT;
    }
};

// sum of G partials in a fixed order, by warp 0; result broadcast through shared memory
__device__ double sum_partials(const double *part, int G) {
    __shared__ double s_res;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < G; i += 32) v += ldcg(part + i);
        v = warp_sum(v);
        if (threadIdx.x == 0) s_res = v;
    }
    __syncthreads();
    const double r = s_res;
    __syncthreads();
    return r;
}

// block reduction of one value per thread, fixed order; thread 0 gets the result
__device__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

struct Chunk {
    int64_t lo, hi;
};
__device__ __forceinline__ Chunk chunk_of(int64_t n) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    Chunk c;
    c.lo = min(n, per * (int64_t)blockIdx.x);
    c.hi = min(n, c.lo + per);
    return c;
}

__device__ __forceinline__ bool skipped(const int32_t *gi) { return ldcg(gi + GI_DONE) != 0; }
// a batched solve stops the cycles of matrices that have converged
__device__ __forceinline__ bool stopped(const int32_t *gi) { return gi && ldcg(gi + GI_STOP) != 0; }

// y = A x (rows split in contiguous chunks; VL lanes per row)
template <int VL>
__device__ __forceinline__ double row_dot(const int32_t *rowptr, const int32_t *colind, const double *val,
                                          const double *x, int64_t i, int sub) {
    double s = 0.0;
    for (int e = rowptr[i] + sub; e < rowptr[i + 1]; e += VL) s = fma(val[e], ldcg(x + colind[e]), s);
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o, VL);
    return s;
}

template <int VL>
__global__ void __launch_bounds__(VT) spmv_kernel(int64_t n, const int32_t *rowptr, const int32_t *colind,
                                                  const double *val, const double *x, double *y,
                                                  const double *b, double *part, const int32_t *gi,
                                                  const int32_t *stop) {
    if ((gi && skipped(gi)) || stopped(stop)) return;
    const Chunk c = chunk_of(n);
    const int sub = threadIdx.x % VL, grp = threadIdx.x / VL, ngrp = VT / VL;
    double acc = 0.0;
    for (int64_t i0 = c.lo; i0 < c.hi; i0 += ngrp) {
        const int64_t i = i0 + grp;
        const bool valid = i < c.hi;
        const double s = row_dot<VL>(rowptr, colind, val, x, valid ? i : c.lo, sub);
        if (valid && sub == 0) {
            if (b) {  // residual r = b - A x and its squared norm
                const double r = b[i] - s;
                y[i] = r;
                acc = fma(r, r, acc);
            } else {
                y[i] = s;
            }
        }
    }
    if (part) {
        const double t = block_sum(acc);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(VT) dot_kernel(int64_t n, const double *x, const double *y, double *part) {
    const Chunk c = chunk_of(n);
    double acc = 0.0;
    for (int64_t i = c.lo + threadIdx.x; i < c.hi; i += VT) acc = fma(ldcg(x + i), ldcg(y + i), acc);
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Classical Gram-Schmidt, applied twice (CGS2), for Arnoldi column j: in each pass one kernel
// forms the partials of the j+1 products V_i^T w in one sweep of the CTA's chunk, the next sums
// them (every CTA, fixed order), adds them to column j of H and subtracts sum_i h_i v_i from w
// in one sweep; the second pass also starts ||w||^2.  Four launches per Arnoldi step instead
// of j+2 for modified Gram-Schmidt; both orthogonalise to working precision and give the same
// iterates in exact arithmetic.
constexpr int CGS_SLOT = 4;  // first partial slot of the products (slot i + CGS_SLOT: V_i^T w)

// one warp per product (warp k takes v_k, v_{k+8}, ...), four partial sums per lane, no block
// barrier: the j+1 products of the CTA's chunk proceed side by side
__global__ void __launch_bounds__(VT) cgs_dot_kernel(int64_t n, int j, const double *__restrict__ V,
                                                     const double *__restrict__ w, double *__restrict__ part,
                                                     const int32_t *gi, int G) {
    if (skipped(gi)) return;
    const Chunk c = chunk_of(n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i <= j; i += VT / 32) {
        const double *vi = V + (int64_t)i * n;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t e = c.lo + lane;
        for (; e + 96 < c.hi; e += 128) {
            a0 = fma(vi[e], w[e], a0);
            a1 = fma(vi[e + 32], w[e + 32], a1);
            a2 = fma(vi[e + 64], w[e + 64], a2);
            a3 = fma(vi[e + 96], w[e + 96], a3);
        }
        for (; e < c.hi; e += 32) a0 = fma(vi[e], w[e], a0);
        const double t = warp_sum((a0 + a1) + (a2 + a3));
        if (lane == 0) part[(int64_t)(CGS_SLOT + i) * G + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(VT) cgs_update_kernel(int64_t n, int j, int m, const double *__restrict__ V,
                                                        double *__restrict__ w, double *part, double *gm,
                                                        const int32_t *gi, int G, int pass) {
    if (skipped(gi)) return;
    __shared__ double h[GMRES_MAX_RESTART];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i <= j; i += VT / 32) {
        double v = 0.0;
        for (int k = lane; k < G; k += 32) v += ldcg(part + (int64_t)(CGS_SLOT + i) * G + k);
        v = warp_sum(v);
        if (lane == 0) h[i] = v;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= j; i += VT) {
            double *hij = gm + (int64_t)i * m + j;
            *hij = pass == 0 ? h[i] : *hij + h[i];
        }
    const Chunk c = chunk_of(n);
    double acc = 0.0;
    for (int64_t e = c.lo + threadIdx.x; e < c.hi; e += VT) {
        double we = w[e];
        for (int i = 0; i <= j; ++i) we = fma(-h[i], V[(int64_t)i * n + e], we);
        w[e] = we;
        acc = fma(we, we, acc);
    }
    if (pass == 1) {
        const double t = block_sum(acc);
        if (threadIdx.x == 0) part[2 * G + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(VT) normalize_kernel(int64_t n, int j, double *V, const double *w,
                                                       const double *part, const int32_t *gi, int G) {
    if (skipped(gi)) return;
    const Chunk c = chunk_of(n);
    const double hn = sqrt(sum_partials(part + 2 * G, G));
    if (hn == 0.0) return;
    const double rh = 1.0 / hn;  // one divide, then multiplies (FP64 divides are slow here)
    double *vn = V + (int64_t)(j + 1) * n;
    for (int64_t e = c.lo + threadIdx.x; e < c.hi; e += VT) vn[e] = w[e] * rh;
}

// Givens rotations on column j of H, update of g, convergence test (one warp).
__global__ void givens_kernel(int j, int m, double *gm, int32_t *gi, const double *part, int G, int64_t soff,
                              int64_t goff, int64_t csoff, int64_t snoff) {
    if (skipped(gi)) return;
    const double hn = sqrt(sum_partials(part + 2 * G, G));
    if (threadIdx.x != 0) return;
    double *H = gm, *g = gm + goff, *cs = gm + csoff, *sn = gm + snoff, *sc = gm + soff;
    H[(int64_t)(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = H[(int64_t)i * m + j], b2 = H[(int64_t)(i + 1) * m + j];
        H[(int64_t)i * m + j] = cs[i] * a + sn[i] * b2;
        H[(int64_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b2;
    }
    const double a = H[(int64_t)j * m + j], b2 = H[(int64_t)(j + 1) * m + j];
    const double den = hypot(a, b2);
    cs[j] = den == 0.0 ? 1.0 : a / den;
    sn[j] = den == 0.0 ? 0.0 : b2 / den;
    H[(int64_t)j * m + j] = den;
    H[(int64_t)(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    gi[GI_ITS] += 1;
    gi[GI_JDONE] = j + 1;
    sc[GS_RELEST] = fabs(g[j + 1]) / sc[GS_BNORM];
    if (fabs(g[j + 1]) <= sc[GS_TOL] * sc[GS_BNORM] || hn == 0.0 || gi[GI_ITS] >= gi[GI_MAXIT]) gi[GI_DONE] = 1;
}

// y = H(0:jd, 0:jd)^{-1} g (back substitution, one thread)
__global__ void solve_y_kernel(int m, double *gm, const int32_t *gi, int64_t goff, int64_t yoff) {
    if (threadIdx.x != 0 || stopped(gi)) return;
    const int jd = gi[GI_JDONE];
    const double *H = gm, *g = gm + goff;
    double *y = gm + yoff;
    for (int i = jd - 1; i >= 0; --i) {
        double s = g[i];
        for (int k = i + 1; k < jd; ++k) s -= H[(int64_t)i * m + k] * y[k];
        y[i] = s / H[(int64_t)i * m + i];
    }
}

// u = V(:, 0:jd) y
__global__ void __launch_bounds__(VT) combine_kernel(int64_t n, const double *V, const double *gm, const int32_t *gi,
                                                     int64_t yoff, double *u) {
    if (stopped(gi)) return;
    const Chunk c = chunk_of(n);
    const int jd = ldcg(gi + GI_JDONE);
    const double *y = gm + yoff;
    for (int64_t e = c.lo + threadIdx.x; e < c.hi; e += VT) {
        double s = 0.0;
        for (int k = 0; k < jd; ++k) s = fma(ldcg(y + k), V[(int64_t)k * n + e], s);
        u[e] = s;
    }
}

__global__ void __launch_bounds__(VT) axpy_kernel(int64_t n, const double *z, double *x, const int32_t *gi) {
    if (stopped(gi)) return;
    const Chunk c = chunk_of(n);
    for (int64_t e = c.lo + threadIdx.x; e < c.hi; e += VT) x[e] += z[e];
}

// beta = ||r||, relative true residual; mirror for the host
__global__ void cycle_end_kernel(double *gm, int32_t *gi, const double *part, int G, int64_t soff,
                                 double *h_scal, int32_t *h_gi) {
    const double beta = sqrt(sum_partials(part + 3 * G, G));
    if (threadIdx.x != 0) return;
    double *sc = gm + soff;
    sc[GS_BETA] = beta;
    sc[GS_REL] = sc[GS_BNORM] > 0.0 ? beta / sc[GS_BNORM] : 0.0;
    for (int k = 0; k < GS_COUNT; ++k) h_scal[k] = sc[k];
    for (int k = 0; k < GI_COUNT; ++k) h_gi[k] = gi[k];
}

// start of a cycle: v_0 = r / beta, g = beta e_1
__global__ void __launch_bounds__(VT) cycle_begin_kernel(int64_t n, int m, const double *r, double *V, double *gm,
                                                         int32_t *gi, int64_t soff, int64_t goff) {
    const double beta = ldcg(gm + soff + GS_BETA);
    const Chunk c = chunk_of(n);
    const double rb = 1.0 / beta;
    for (int64_t e = c.lo + threadIdx.x; e < c.hi; e += VT) V[e] = r[e] * rb;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double *g = gm + goff;
        for (int k = 0; k <= m; ++k) g[k] = 0.0;
        g[0] = beta;
        gi[GI_JDONE] = 0;
        gi[GI_DONE] = (gi[GI_ITS] >= gi[GI_MAXIT] || gi[GI_STOP]) ? 1 : 0;
    }
}

__global__ void setup_kernel(double *gm, int32_t *gi, const double *part, int G, int64_t soff, double tol, int maxit,
                             int m) {
    const double bn = sqrt(sum_partials(part + 3 * G, G));
    if (threadIdx.x != 0) return;
    double *sc = gm + soff;
    sc[GS_BNORM] = bn;
    sc[GS_TOL] = tol;
    gi[GI_ITS] = 0;
    gi[GI_JDONE] = 0;
    gi[GI_DONE] = 0;
    gi[GI_MAXIT] = maxit;
    gi[GI_M] = m;
    gi[GI_STOP] = 0;
}

}  // namespace

// A new factor invalidates the captured cycle (its sweeps read the factor's buffers); the
// workspace stays for the next solve.
void gmres_drop_graph(bilu_ctx *c) {
    if (c->gm_graph) cudaGraphExecDestroy(c->gm_graph);
    c->gm_graph = nullptr;
}

void gmres_free(bilu_ctx *c) {
    if (c->gm_graph) cudaGraphExecDestroy(c->gm_graph);
    c->gm_graph = nullptr;
    dev_free(c->d_V);
    dev_free(c->d_w);
    dev_free(c->d_z);
    dev_free(c->d_r);
    dev_free(c->d_u);
    dev_free(c->d_part);
    dev_free(c->d_gm);
    dev_free(c->d_gmi);
    dev_free(c->d_gb);
    dev_free(c->d_gx);
    if (c->h_gm_pinned) cudaFreeHost(c->h_gm_pinned);
    if (c->h_gmi_pinned) cudaFreeHost(c->h_gmi_pinned);
    c->h_gm_pinned = nullptr;
    c->h_gmi_pinned = nullptr;
    c->gm_restart = 0;
}

namespace {

int vector_grid(const bilu_ctx *c) { return 2 * c->nsm; }

void launch_spmv(bilu_ctx *c, const double *x, double *y, const double *b, double *part, const int32_t *gi,
                 const int32_t *stop = nullptr) {
    const int G = vector_grid(c);
    const double avg = c->n > 0 ? (double)c->nnz / (double)c->n : 0.0;
    if (avg <= 12) spmv_kernel<8><<<G, VT, 0, c->stream>>>(c->n, c->d_rowptr, c->d_colind, c->d_val, x, y, b, part, gi, stop);
    else if (avg <= 40) spmv_kernel<16><<<G, VT, 0, c->stream>>>(c->n, c->d_rowptr, c->d_colind, c->d_val, x, y, b, part, gi, stop);
    else spmv_kernel<32><<<G, VT, 0, c->stream>>>(c->n, c->d_rowptr, c->d_colind, c->d_val, x, y, b, part, gi, stop);
}

bilu_status gmres_alloc(bilu_ctx *c, int m) {
    gmres_free(c);
    const int64_t n = std::max<int64_t>(c->n, 1);
    GmLayout L(m);
    if (dev_alloc(&c->d_V, (int64_t)(m + 1) * n) != cudaSuccess || dev_alloc(&c->d_w, n) != cudaSuccess ||
        dev_alloc(&c->d_z, n) != cudaSuccess || dev_alloc(&c->d_r, n) != cudaSuccess ||
        dev_alloc(&c->d_u, n) != cudaSuccess || dev_alloc(&c->d_part, (int64_t)(CGS_SLOT + m + 1) * vector_grid(c)) != cudaSuccess ||
        dev_alloc(&c->d_gm, L.total) != cudaSuccess || dev_alloc(&c->d_gmi, GI_COUNT) != cudaSuccess ||
        dev_alloc(&c->d_gb, n) != cudaSuccess || dev_alloc(&c->d_gx, n) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_gm_pinned, GS_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_gmi_pinned, GI_COUNT * sizeof(int32_t)) != cudaSuccess) {
        gmres_free(c);
        return set_err(c, BILU_ERR_OOM, "gmres allocation failed");
    }
    BILU_CUDA(c, cudaMemsetAsync(c->d_gm, 0, L.total * sizeof(double), c->stream));
    c->gm_restart = m;
    return BILU_OK;
}

// Records one restart cycle on the context stream (used under stream capture).
bilu_status record_cycle(bilu_ctx *c, int m) {
    const int G = vector_grid(c);
    GmLayout L(m);
    const int64_t n = c->n;
    int32_t *gi = c->d_gmi;
    cycle_begin_kernel<<<G, VT, 0, c->stream>>>(n, m, c->d_r, c->d_V, c->d_gm, gi, L.scal, L.g);
    for (int j = 0; j < m; ++j) {
        bilu_status st = apply_launch(c, c->d_V + (int64_t)j * n, c->d_z, gi + GI_DONE);
        if (st != BILU_OK) return st;
        launch_spmv(c, c->d_z, c->d_w, nullptr, nullptr, gi);
        for (int pass = 0; pass < 2; ++pass) {
            cgs_dot_kernel<<<G, VT, 0, c->stream>>>(n, j, c->d_V, c->d_w, c->d_part, gi, G);
            cgs_update_kernel<<<G, VT, 0, c->stream>>>(n, j, m, c->d_V, c->d_w, c->d_part, c->d_gm, gi, G, pass);
        }
        normalize_kernel<<<G, VT, 0, c->stream>>>(n, j, c->d_V, c->d_w, c->d_part, gi, G);
        givens_kernel<<<1, 32, 0, c->stream>>>(j, m, c->d_gm, gi, c->d_part, G, L.scal, L.g, L.cs, L.sn);
    }
    solve_y_kernel<<<1, 32, 0, c->stream>>>(m, c->d_gm, gi, L.g, L.y);
    combine_kernel<<<G, VT, 0, c->stream>>>(n, c->d_V, c->d_gm, gi, L.y, c->d_u);
    bilu_status st = apply_launch(c, c->d_u, c->d_z, gi + GI_STOP);
    if (st != BILU_OK) return st;
    axpy_kernel<<<G, VT, 0, c->stream>>>(n, c->d_z, c->d_gx, gi);
    launch_spmv(c, c->d_gx, c->d_r, c->d_gb, c->d_part + 3 * G, nullptr, gi);
    cycle_end_kernel<<<1, 32, 0, c->stream>>>(c->d_gm, gi, c->d_part, G, L.scal, c->h_gm_pinned, c->h_gmi_pinned);
    BILU_CUDA(c, cudaGetLastError());
    return BILU_OK;
}

// initial residual and state of one solve (stream-ordered on c->stream)
void gmres_start(bilu_ctx *c, double tol, int m, int maxit) {
    const int G = vector_grid(c);
    GmLayout L(m);
    dot_kernel<<<G, VT, 0, c->stream>>>(c->n, c->d_gb, c->d_gb, c->d_part + 3 * G);
    setup_kernel<<<1, 32, 0, c->stream>>>(c->d_gm, c->d_gmi, c->d_part, G, L.scal, tol, maxit, m);
    launch_spmv(c, c->d_gx, c->d_r, c->d_gb, c->d_part + 3 * G, nullptr);
    cycle_end_kernel<<<1, 32, 0, c->stream>>>(c->d_gm, c->d_gmi, c->d_part, G, L.scal, c->h_gm_pinned, c->h_gmi_pinned);
    c->launches += 4;
}

int64_t count_kernel_nodes(cudaGraph_t graph) {
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    int64_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

}  // namespace

// Restarted GMRES on many independent systems at once: one CUDA graph holds a restart cycle
// of every system as a parallel branch; systems that have converged are stopped by a device
// flag, so every kernel of their branch returns at once.
bilu_status gmres_batch_run(bilu_ctx *const *ctxs, int count, const double *const *b, double *const *x, double tol,
                            int m, int maxit, gmres_info *info) {
    bilu_ctx *c0 = ctxs[0];
    const cudaStream_t master = c0->stream;  // every context is redirected to it below
    if (m < 1 || m > GMRES_MAX_RESTART || maxit < 0 || !(tol >= 0.0)) return set_err(c0, BILU_ERR_ARG, "bad gmres arguments");
    cudaEvent_t e0, e1;
    BILU_CUDA(c0, cudaEventCreate(&e0));
    BILU_CUDA(c0, cudaEventCreate(&e1));
    BILU_CUDA(c0, cudaEventRecord(e0, master));
    std::vector<cudaStream_t> own(count);
    for (int i = 0; i < count; ++i) own[i] = ctxs[i]->stream;
    // the contexts get their own streams back on every exit path
    struct Restore {
        bilu_ctx *const *ctxs;
        std::vector<cudaStream_t> &own;
        ~Restore() {
            for (size_t i = 0; i < own.size(); ++i) {
                ctxs[i]->stream = own[i];
                ctxs[i]->apply_grid = 0;
            }
        }
    } restore{ctxs, own};
    // The sweeps are chains of dependent blocks (latency-bound): each system's sweeps get an
    // equal share of the resident CTA slots, so that the branches of the graph run side by
    // side instead of one whole-GPU sweep after another.
    for (int i = 0; i < count; ++i) ctxs[i]->apply_grid = std::max(2, 2 * c0->nsm / count);
    for (int i = 0; i < count; ++i) {
        bilu_ctx *c = ctxs[i];
        if (c->gm_restart != m) {
            bilu_status st = gmres_alloc(c, m);
            if (st != BILU_OK) return st;
        }
        c->stream = master;
        BILU_CUDA(c0, cudaMemcpyAsync(c->d_gb, b[i], c->n * sizeof(double), cudaMemcpyDefault, master));
        BILU_CUDA(c0, cudaMemcpyAsync(c->d_gx, x[i], c->n * sizeof(double), cudaMemcpyDefault, master));
        gmres_start(c, tol, m, maxit);
    }
    BILU_CUDA(c0, cudaStreamSynchronize(master));
    // one graph: a branch per system, forked from and joined to c0's stream
    std::vector<cudaStream_t> br(count);
    std::vector<cudaEvent_t> ev(count + 1);
    for (int i = 0; i < count; ++i) BILU_CUDA(c0, cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking));
    for (int i = 0; i <= count; ++i) BILU_CUDA(c0, cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    cudaGraph_t graph;
    BILU_CUDA(c0, cudaStreamBeginCapture(master, cudaStreamCaptureModeThreadLocal));
    BILU_CUDA(c0, cudaEventRecord(ev[count], master));
    bilu_status rst = BILU_OK;
    for (int i = 0; i < count && rst == BILU_OK; ++i) {
        bilu_ctx *c = ctxs[i];
        cudaStreamWaitEvent(br[i], ev[count], 0);
        c->stream = br[i];
        const int64_t before = c->launches;
        rst = record_cycle(c, m);
        c->launches = before;
        cudaEventRecord(ev[i], br[i]);
        cudaStreamWaitEvent(master, ev[i], 0);
        c->stream = master;
    }
    cudaError_t ce = cudaStreamEndCapture(master, &graph);
    if (rst != BILU_OK) return rst;
    if (ce != cudaSuccess) return cuda_err(c0, ce, "cudaStreamEndCapture (batch)");
    cudaGraphExec_t exec = nullptr;
    const int64_t nodes = count_kernel_nodes(graph);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_err(c0, ce, "cudaGraphInstantiate (batch)");
    std::vector<int> restarts(count, 0);
    for (int cycle = 0; cycle < maxit + 1; ++cycle) {
        bool any = false;
        for (int i = 0; i < count; ++i) {
            bilu_ctx *c = ctxs[i];
            const bool active = c->h_gm_pinned[GS_BNORM] > 0.0 && c->h_gm_pinned[GS_REL] > tol &&
                                c->h_gmi_pinned[GI_ITS] < maxit;
            if (active) { any = true; ++restarts[i]; }
            const int32_t stop = active ? 0 : 1;
            BILU_CUDA(c0, cudaMemcpyAsync(c->d_gmi + GI_STOP, &stop, sizeof(int32_t), cudaMemcpyHostToDevice, master));
        }
        if (!any) break;
        BILU_CUDA(c0, cudaGraphLaunch(exec, master));
        c0->launches += nodes;
        BILU_CUDA(c0, cudaStreamSynchronize(master));
    }
    cudaGraphExecDestroy(exec);
    for (int i = 0; i < count; ++i) {
        cudaStreamDestroy(br[i]);
        cudaEventDestroy(ev[i]);
    }
    cudaEventDestroy(ev[count]);
    bilu_status result = BILU_OK;
    for (int i = 0; i < count; ++i) {
        bilu_ctx *c = ctxs[i];
        if (c->h_gm_pinned[GS_BNORM] == 0.0) BILU_CUDA(c0, cudaMemsetAsync(c->d_gx, 0, c->n * sizeof(double), master));
        BILU_CUDA(c0, cudaMemcpyAsync(x[i], c->d_gx, c->n * sizeof(double), cudaMemcpyDefault, master));
    }
    BILU_CUDA(c0, cudaEventRecord(e1, master));
    BILU_CUDA(c0, cudaStreamSynchronize(master));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < count; ++i) {
        bilu_ctx *c = ctxs[i];
        const bool zero = c->h_gm_pinned[GS_BNORM] == 0.0;
        const double rel = zero ? 0.0 : c->h_gm_pinned[GS_REL];
        if (info) {
            info[i].iters = zero ? 0 : c->h_gmi_pinned[GI_ITS];
            info[i].restarts = restarts[i];
            info[i].relres_true = rel;
            info[i].relres_est = c->h_gm_pinned[GS_RELEST];
            info[i].t_solve_ms = ms;
        }
        int32_t apst[4];
        BILU_CUDA(c0, cudaMemcpy(apst, c->d_apst, sizeof(apst), cudaMemcpyDeviceToHost));
        if (apst[3] != 0) return set_err(c0, BILU_ERR_TIMEOUT, "apply kernel: bounded wait gave up");
        if (rel > tol) result = BILU_NOT_CONVERGED;
    }
    return result;
}

bilu_status gmres_run(bilu_ctx *c, const double *b, double *x, double tol, int m, int maxit, gmres_info *info) {
    if (m < 1 || m > GMRES_MAX_RESTART || maxit < 0 || !(tol >= 0.0)) return set_err(c, BILU_ERR_ARG, "bad gmres arguments");
    if (c->gm_restart != m) {
        bilu_status st = gmres_alloc(c, m);
        if (st != BILU_OK) return st;
    }
    const int G = vector_grid(c);
    const int64_t n = c->n;
    GmLayout L(m);
    cudaEvent_t e0, e1;
    BILU_CUDA(c, cudaEventCreate(&e0));
    BILU_CUDA(c, cudaEventCreate(&e1));
    BILU_CUDA(c, cudaEventRecord(e0, c->stream));
    BILU_CUDA(c, cudaMemcpyAsync(c->d_gb, b, n * sizeof(double), cudaMemcpyDefault, c->stream));
    BILU_CUDA(c, cudaMemcpyAsync(c->d_gx, x, n * sizeof(double), cudaMemcpyDefault, c->stream));
    gmres_start(c, tol, m, maxit);
    BILU_CUDA(c, cudaGetLastError());
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    double bnorm = c->h_gm_pinned[GS_BNORM];
    double rel = c->h_gm_pinned[GS_REL];
    int restarts = 0;
    if (bnorm == 0.0) {
        BILU_CUDA(c, cudaMemsetAsync(c->d_gx, 0, n * sizeof(double), c->stream));
        rel = 0.0;
    } else {
        if (!c->gm_graph) {
            cudaGraph_t graph;
            BILU_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            const int64_t before = c->launches;
            bilu_status st = record_cycle(c, m);
            c->launches = before;  // captured, not launched: counted per graph launch
            cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
            if (st != BILU_OK) return st;
            if (ce != cudaSuccess) return cuda_err(c, ce, "cudaStreamEndCapture");
            c->gm_graph_kernels = count_kernel_nodes(graph);
            ce = cudaGraphInstantiate(&c->gm_graph, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_err(c, ce, "cudaGraphInstantiate");
        }
        while (rel > tol && c->h_gmi_pinned[GI_ITS] < maxit) {
            BILU_CUDA(c, cudaGraphLaunch(c->gm_graph, c->stream));
            c->launches += c->gm_graph_kernels;
            BILU_CUDA(c, cudaStreamSynchronize(c->stream));
            rel = c->h_gm_pinned[GS_REL];
            ++restarts;
        }
    }
    BILU_CUDA(c, cudaMemcpyAsync(x, c->d_gx, n * sizeof(double), cudaMemcpyDefault, c->stream));
    BILU_CUDA(c, cudaEventRecord(e1, c->stream));
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    int32_t apst[4];
    BILU_CUDA(c, cudaMemcpy(apst, c->d_apst, sizeof(apst), cudaMemcpyDeviceToHost));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iters = bnorm == 0.0 ? 0 : c->h_gmi_pinned[GI_ITS];
        info->restarts = restarts;
        info->relres_true = rel;
        info->relres_est = c->h_gm_pinned[GS_RELEST];
        info->t_solve_ms = ms;
    }
    if (apst[3] != 0) return set_err(c, BILU_ERR_TIMEOUT, "apply kernel: bounded wait gave up");
    return rel <= tol ? BILU_OK : BILU_NOT_CONVERGED;
}
