// Simplified QMR (Freund and Nachtigal; the solver the paper pairs with the symmetric variant
// BILDL, Sec. 4.2) on the GPU, preconditioned with the context's factor.
//
// One step: sigma = q^T A q, alpha = rho / sigma, r -= alpha A q, theta' = ||r|| / tau,
// c = (1 + theta'^2)^{-1/2}, tau = tau theta' c, d = c^2 theta^2 d + c^2 alpha q, x += d, the
// normwise backward error of x decides the stop, u = M^{-1} r, rho' = r^T u,
// q = u + (rho' / rho) q.  The vector kernels take contiguous row chunks; every reduction is a
// set of per-CTA partials combined in a fixed order by the next (one-warp) scalar kernel, so a
// solve is bitwise reproducible.  A batch of SQMR_STEPS steps is captured once into a CUDA
// graph; after convergence every kernel of a step returns at once, and the host synchronizes
// once per batch.
#include <cmath>
#include <vector>

#include "dev_common.cuh"

namespace {

constexpr int VT = 256;         // threads per CTA of the vector kernels
constexpr int SQMR_STEPS = 8;   // steps per graph launch

// integer state
enum { SI_ITS = 0, SI_DONE, SI_BREAK, SI_MAXIT, SI_COUNT = 8 };
// scalar state
enum {
    SS_RHO = 0, SS_ALPHA, SS_BETA, SS_THETA, SS_TAU, SS_E1, SS_E2, SS_ANORM, SS_BMAX, SS_BNORM, SS_ETA, SS_REL,
    SS_TOL, SS_COUNT = 16
};
// partial-sum slots (each G doubles)
enum { P_QT = 0, P_RR, P_RES, P_XMAX, P_RES2, P_RU, P_COUNT };

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

// a null state pointer: the kernel always runs (setup)
__device__ __forceinline__ bool finished(const int32_t *si) { return si && ldcg(si + SI_DONE) != 0; }

// block reductions in a fixed order; thread 0 gets the result
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
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}
__device__ double block_max(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max(v);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        r = warp_max(r);
    }
    __syncthreads();
    return r;
}
// one warp: the G partials of a slot, summed (or maxed) in a fixed order
__device__ __forceinline__ double partial_sum(const double *p, int G) {
    double v = 0.0;
    for (int i = threadIdx.x; i < G; i += 32) v += ldcg(p + i);
    return warp_sum(v);
}
__device__ __forceinline__ double partial_max(const double *p, int G) {
    double v = 0.0;
    for (int i = threadIdx.x; i < G; i += 32) v = fmax(v, ldcg(p + i));
    return warp_max(v);
}

template <int VL>
__device__ __forceinline__ double row_dot(const int32_t *rowptr, const int32_t *colind, const double *val,
                                          const double *x, int64_t i, int sub) {
    double s = 0.0;
    for (int e = rowptr[i] + sub; e < rowptr[i + 1]; e += VL) s = fma(val[e], ldcg(x + colind[e]), s);
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o, VL);
    return s;
}

struct Mat {
    int64_t n;
    const int32_t *rowptr, *colind;
    const double *val;
};

// t = A q and the partials of q^T t
template <int VL>
__global__ void __launch_bounds__(VT) spmv_dot_kernel(Mat A, const double *q, double *t, double *part,
                                                      const int32_t *si) {
    if (finished(si)) return;
    const Chunk c = chunk_of(A.n);
    const int sub = threadIdx.x % VL, grp = threadIdx.x / VL, ngrp = VT / VL;
    double acc = 0.0;
    for (int64_t i0 = c.lo; i0 < c.hi; i0 += ngrp) {
        const int64_t i = i0 + grp;
        const bool valid = i < c.hi;
        const double s = row_dot<VL>(A.rowptr, A.colind, A.val, q, valid ? i : c.lo, sub);
        if (valid && sub == 0) {
            t[i] = s;
            acc = fma(q[i], s, acc);
        }
    }
    const double tot = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// rt = b - A x with the partials of max |rt|, max |x| and ||rt||^2 (the stop test); with
// setup, also ||A||_inf (row sums) into the P_RU slot and max |b| into the P_QT slot
template <int VL>
__global__ void __launch_bounds__(VT) residual_kernel(Mat A, const double *b, const double *x, double *rt,
                                                      double *part, int G, const int32_t *si, int setup) {
    if (finished(si)) return;
    const Chunk c = chunk_of(A.n);
    const int sub = threadIdx.x % VL, grp = threadIdx.x / VL, ngrp = VT / VL;
    double rmax = 0.0, xmax = 0.0, r2 = 0.0, amax = 0.0, bmax = 0.0;
    for (int64_t i0 = c.lo; i0 < c.hi; i0 += ngrp) {
        const int64_t i = i0 + grp;
        const bool valid = i < c.hi;
        const int64_t ii = valid ? i : c.lo;
        const double s = row_dot<VL>(A.rowptr, A.colind, A.val, x, ii, sub);
        double asum = 0.0;
        if (setup) {
            for (int e = A.rowptr[ii] + sub; e < A.rowptr[ii + 1]; e += VL) asum += fabs(A.val[e]);
#pragma unroll
            for (int o = VL / 2; o > 0; o >>= 1) asum += __shfl_xor_sync(FULL_MASK, asum, o, VL);
        }
        if (valid && sub == 0) {
            const double r = b[i] - s;
            rt[i] = r;
            rmax = fmax(rmax, fabs(r));
            xmax = fmax(xmax, fabs(x[i]));
            r2 = fma(r, r, r2);
            amax = fmax(amax, asum);
            bmax = fmax(bmax, fabs(b[i]));
        }
    }
    rmax = block_max(rmax);
    xmax = block_max(xmax);
    r2 = block_sum(r2);
    if (setup) {
        amax = block_max(amax);
        bmax = block_max(bmax);
    }
    if (threadIdx.x == 0) {
        part[P_RES * G + blockIdx.x] = rmax;
        part[P_XMAX * G + blockIdx.x] = xmax;
        part[P_RES2 * G + blockIdx.x] = r2;
        if (setup) {
            part[P_RU * G + blockIdx.x] = amax;
            part[P_QT * G + blockIdx.x] = bmax;
        }
    }
}

// partials of x^T y
__global__ void __launch_bounds__(VT) dot_kernel(int64_t n, const double *x, const double *y, double *part,
                                                 const int32_t *si) {
    if (finished(si)) return;
    const Chunk c = chunk_of(n);
    double acc = 0.0;
    for (int64_t i = c.lo + threadIdx.x; i < c.hi; i += VT) acc = fma(x[i], y[i], acc);
    const double tot = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// r -= alpha t, partials of ||r||^2
__global__ void __launch_bounds__(VT) update_r_kernel(int64_t n, const double *t, double *r, const double *ss,
                                                      double *part, const int32_t *si) {
    if (finished(si)) return;
    const double alpha = ldcg(ss + SS_ALPHA);
    const Chunk c = chunk_of(n);
    double acc = 0.0;
    for (int64_t i = c.lo + threadIdx.x; i < c.hi; i += VT) {
        const double v = fma(-alpha, t[i], r[i]);
        r[i] = v;
        acc = fma(v, v, acc);
    }
    const double tot = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// d = e1 d + e2 q, x += d
__global__ void __launch_bounds__(VT) update_x_kernel(int64_t n, const double *q, double *d, double *x,
                                                      const double *ss, const int32_t *si) {
    if (finished(si)) return;
    const double e1 = ldcg(ss + SS_E1), e2 = ldcg(ss + SS_E2);
    const Chunk c = chunk_of(n);
    for (int64_t i = c.lo + threadIdx.x; i < c.hi; i += VT) {
        const double v = __dadd_rn(__dmul_rn(e1, d[i]), __dmul_rn(e2, q[i]));
        d[i] = v;
        x[i] += v;
    }
}

// q = u + beta q
__global__ void __launch_bounds__(VT) update_q_kernel(int64_t n, const double *u, double *q, const double *ss,
                                                      const int32_t *si) {
    if (finished(si)) return;
    const double beta = ldcg(ss + SS_BETA);
    const Chunk c = chunk_of(n);
    for (int64_t i = c.lo + threadIdx.x; i < c.hi; i += VT) q[i] = fma(beta, q[i], u[i]);
}

// ---- one-warp scalar kernels

// sigma = q^T A q; alpha = rho / sigma (a zero sigma is a breakdown)
__global__ void scalar_alpha_kernel(const double *part, int G, double *ss, int32_t *si) {
    if (finished(si)) return;
    const double sigma = partial_sum(part + P_QT * G, G);
    if (threadIdx.x != 0) return;
    if (sigma == 0.0) {
        si[SI_BREAK] = 1;
        si[SI_DONE] = 1;
        return;
    }
    ss[SS_ALPHA] = ss[SS_RHO] / sigma;
}

// theta' = ||r|| / tau, c, the coefficients of d, tau and theta moved on
__global__ void scalar_theta_kernel(const double *part, int G, double *ss, const int32_t *si) {
    if (finished(si)) return;
    const double rr = partial_sum(part + P_RR * G, G);
    if (threadIdx.x != 0) return;
    const double theta1 = sqrt(rr) / ss[SS_TAU];
    const double c = 1.0 / sqrt(1.0 + theta1 * theta1);
    const double c2 = c * c, th = ss[SS_THETA];
    ss[SS_E1] = c2 * th * th;
    ss[SS_E2] = c2 * ss[SS_ALPHA];
    ss[SS_TAU] = ss[SS_TAU] * theta1 * c;
    ss[SS_THETA] = theta1;
}

// backward error of x and the stop test; with setup, ||A||_inf and max |b| first
__global__ void scalar_stop_kernel(const double *part, int G, double *ss, int32_t *si, int setup, int count) {
    if (!setup && finished(si)) return;
    const double rmax = partial_max(part + P_RES * G, G), xmax = partial_max(part + P_XMAX * G, G);
    const double r2 = partial_sum(part + P_RES2 * G, G);
    double amax = 0.0, bmax = 0.0;
    if (setup) {
        amax = partial_max(part + P_RU * G, G);
        bmax = partial_max(part + P_QT * G, G);
    }
    if (threadIdx.x != 0) return;
    if (setup) {
        ss[SS_ANORM] = amax;
        ss[SS_BMAX] = bmax;
        ss[SS_BNORM] = sqrt(ss[SS_BNORM]);
    }
    const double den = ss[SS_ANORM] * xmax + ss[SS_BMAX];
    const double eta = den > 0.0 ? rmax / den : 0.0;
    ss[SS_ETA] = eta;
    ss[SS_REL] = ss[SS_BNORM] > 0.0 ? sqrt(r2) / ss[SS_BNORM] : 0.0;
    if (count) si[SI_ITS] += 1;
    if (eta <= ss[SS_TOL] || si[SI_ITS] >= si[SI_MAXIT]) si[SI_DONE] = 1;
    else if (count && ss[SS_RHO] == 0.0) { si[SI_BREAK] = 1; si[SI_DONE] = 1; }
    if (setup) {
        ss[SS_TAU] = sqrt(r2);
        ss[SS_THETA] = 0.0;
    }
}

// rho' = r^T u, beta = rho' / rho, rho moved on
__global__ void scalar_rho_kernel(const double *part, int G, double *ss, const int32_t *si, int setup) {
    if (finished(si)) return;
    const double ru = partial_sum(part + P_RU * G, G);
    if (threadIdx.x != 0) return;
    if (!setup) ss[SS_BETA] = ru / ss[SS_RHO];
    ss[SS_RHO] = ru;
}

__global__ void setup_kernel(double *ss, int32_t *si, double tol, int maxit, const double *part, int G) {
    const double bb = partial_sum(part + P_RU * G, G);
    if (threadIdx.x != 0) return;
    for (int k = 0; k < SS_COUNT; ++k) ss[k] = 0.0;
    ss[SS_TOL] = tol;
    ss[SS_BNORM] = bb;  // squared; scalar_stop_kernel takes the root
    for (int k = 0; k < SI_COUNT; ++k) si[k] = 0;
    si[SI_MAXIT] = maxit;
}

__global__ void mirror_kernel(const double *ss, const int32_t *si, double *h_ss, int32_t *h_si) {
    if (threadIdx.x != 0) return;
    for (int k = 0; k < SS_COUNT; ++k) h_ss[k] = ss[k];
    for (int k = 0; k < SI_COUNT; ++k) h_si[k] = si[k];
}

int vector_grid(const bilu_ctx *c) { return 2 * c->nsm; }

Mat mat_of(const bilu_ctx *c) { return Mat{c->n, c->d_rowptr, c->d_colind, c->d_val}; }

int lanes_per_row(const bilu_ctx *c) {
    const double avg = c->n > 0 ? (double)c->nnz / (double)c->n : 0.0;
    return avg <= 12 ? 8 : avg <= 40 ? 16 : 32;
}

void launch_spmv_dot(bilu_ctx *c, const double *q, double *t, double *part, const int32_t *si) {
    const int G = vector_grid(c);
    const Mat A = mat_of(c);
    switch (lanes_per_row(c)) {
        case 8: spmv_dot_kernel<8><<<G, VT, 0, c->stream>>>(A, q, t, part, si); break;
        case 16: spmv_dot_kernel<16><<<G, VT, 0, c->stream>>>(A, q, t, part, si); break;
        default: spmv_dot_kernel<32><<<G, VT, 0, c->stream>>>(A, q, t, part, si); break;
    }
}

void launch_residual(bilu_ctx *c, const double *b, const double *x, double *rt, double *part, const int32_t *si,
                     int setup) {
    const int G = vector_grid(c);
    const Mat A = mat_of(c);
    switch (lanes_per_row(c)) {
        case 8: residual_kernel<8><<<G, VT, 0, c->stream>>>(A, b, x, rt, part, G, si, setup); break;
        case 16: residual_kernel<16><<<G, VT, 0, c->stream>>>(A, b, x, rt, part, G, si, setup); break;
        default: residual_kernel<32><<<G, VT, 0, c->stream>>>(A, b, x, rt, part, G, si, setup); break;
    }
}

// workspace: r, t, q, d, u, rt, b, x (n each)
enum { V_R = 0, V_T, V_Q, V_D, V_U, V_RT, V_B, V_X, V_COUNT };

bilu_status sqmr_alloc(bilu_ctx *c) {
    sqmr_free(c);
    const int64_t n = std::max<int64_t>(c->n, 1);
    if (dev_alloc(&c->d_sq, V_COUNT * n) != cudaSuccess || dev_alloc(&c->d_sqpart, (int64_t)P_COUNT * vector_grid(c)) != cudaSuccess ||
        dev_alloc(&c->d_sqs, SS_COUNT) != cudaSuccess || dev_alloc(&c->d_sqi, SI_COUNT) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_sqs, SS_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_sqi, SI_COUNT * sizeof(int32_t)) != cudaSuccess) {
        sqmr_free(c);
        return set_err(c, BILU_ERR_OOM, "sqmr allocation failed");
    }
    c->sq_n = c->n;
    return BILU_OK;
}

// one step, recorded on the context stream (under stream capture)
bilu_status record_step(bilu_ctx *c) {
    const int G = vector_grid(c);
    const int64_t n = c->n;
    double *V = c->d_sq, *part = c->d_sqpart, *ss = c->d_sqs;
    int32_t *si = c->d_sqi;
    double *r = V + V_R * n, *t = V + V_T * n, *q = V + V_Q * n, *d = V + V_D * n, *u = V + V_U * n;
    double *rt = V + V_RT * n, *b = V + V_B * n, *x = V + V_X * n;
    launch_spmv_dot(c, q, t, part + P_QT * G, si);
    scalar_alpha_kernel<<<1, 32, 0, c->stream>>>(part, G, ss, si);
    update_r_kernel<<<G, VT, 0, c->stream>>>(n, t, r, ss, part + P_RR * G, si);
    scalar_theta_kernel<<<1, 32, 0, c->stream>>>(part, G, ss, si);
    update_x_kernel<<<G, VT, 0, c->stream>>>(n, q, d, x, ss, si);
    launch_residual(c, b, x, rt, part, si, 0);
    scalar_stop_kernel<<<1, 32, 0, c->stream>>>(part, G, ss, si, 0, 1);
    bilu_status st = apply_launch(c, r, u, si + SI_DONE);
    if (st != BILU_OK) return st;
    dot_kernel<<<G, VT, 0, c->stream>>>(n, r, u, part + P_RU * G, si);
    scalar_rho_kernel<<<1, 32, 0, c->stream>>>(part, G, ss, si, 0);
    update_q_kernel<<<G, VT, 0, c->stream>>>(n, u, q, ss, si);
    BILU_CUDA(c, cudaGetLastError());
    return BILU_OK;
}

int64_t kernel_nodes(cudaGraph_t graph) {
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

void sqmr_drop_graph(bilu_ctx *c) {
    if (c->sq_graph) cudaGraphExecDestroy(c->sq_graph);
    c->sq_graph = nullptr;
}

void sqmr_free(bilu_ctx *c) {
    if (c->sq_graph) cudaGraphExecDestroy(c->sq_graph);
    c->sq_graph = nullptr;
    dev_free(c->d_sq);
    dev_free(c->d_sqpart);
    dev_free(c->d_sqs);
    dev_free(c->d_sqi);
    if (c->h_sqs) cudaFreeHost(c->h_sqs);
    if (c->h_sqi) cudaFreeHost(c->h_sqi);
    c->h_sqs = nullptr;
    c->h_sqi = nullptr;
    c->sq_n = -1;
}

bilu_status sqmr_run(bilu_ctx *c, const double *b, double *x, double tol, int maxit, sqmr_info *info) {
    if (maxit < 0 || !(tol >= 0.0)) return set_err(c, BILU_ERR_ARG, "bad sqmr arguments");
    if (c->sq_n != c->n || !c->d_sq) {
        bilu_status st = sqmr_alloc(c);
        if (st != BILU_OK) return st;
    }
    const int G = vector_grid(c);
    const int64_t n = c->n;
    double *V = c->d_sq, *part = c->d_sqpart, *ss = c->d_sqs;
    int32_t *si = c->d_sqi;
    double *r = V + V_R * n, *q = V + V_Q * n, *d = V + V_D * n;
    double *db = V + V_B * n, *dx = V + V_X * n;
    cudaEvent_t e0, e1;
    BILU_CUDA(c, cudaEventCreate(&e0));
    BILU_CUDA(c, cudaEventCreate(&e1));
    BILU_CUDA(c, cudaEventRecord(e0, c->stream));
    BILU_CUDA(c, cudaMemcpyAsync(db, b, n * sizeof(double), cudaMemcpyDefault, c->stream));
    BILU_CUDA(c, cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyDefault, c->stream));
    BILU_CUDA(c, cudaMemsetAsync(d, 0, n * sizeof(double), c->stream));
    // ||b||^2 into the P_RU slot for the setup, then r = b - A x0 with ||A||_inf and max |b|
    dot_kernel<<<G, VT, 0, c->stream>>>(n, db, db, part + P_RU * G, nullptr);
    setup_kernel<<<1, 32, 0, c->stream>>>(ss, si, tol, maxit, part, G);
    launch_residual(c, db, dx, r, part, si, 1);
    scalar_stop_kernel<<<1, 32, 0, c->stream>>>(part, G, ss, si, 1, 0);
    bilu_status st = apply_launch(c, r, q, si + SI_DONE);
    if (st != BILU_OK) return st;
    dot_kernel<<<G, VT, 0, c->stream>>>(n, r, q, part + P_RU * G, si);
    scalar_rho_kernel<<<1, 32, 0, c->stream>>>(part, G, ss, si, 1);
    mirror_kernel<<<1, 32, 0, c->stream>>>(ss, si, c->h_sqs, c->h_sqi);
    c->launches += 8;
    BILU_CUDA(c, cudaGetLastError());
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!c->sq_graph) {
        cudaGraph_t graph;
        BILU_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = c->launches;
        for (int k = 0; k < SQMR_STEPS && st == BILU_OK; ++k) st = record_step(c);
        if (st == BILU_OK) mirror_kernel<<<1, 32, 0, c->stream>>>(ss, si, c->h_sqs, c->h_sqi);
        c->launches = before;  // captured, not launched: counted per graph launch
        cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
        if (st != BILU_OK) return st;
        if (ce != cudaSuccess) return cuda_err(c, ce, "cudaStreamEndCapture");
        c->sq_graph_kernels = kernel_nodes(graph);
        ce = cudaGraphInstantiate(&c->sq_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_err(c, ce, "cudaGraphInstantiate");
    }
    while (!c->h_sqi[SI_DONE]) {
        BILU_CUDA(c, cudaGraphLaunch(c->sq_graph, c->stream));
        c->launches += c->sq_graph_kernels;
        BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    BILU_CUDA(c, cudaMemcpyAsync(x, dx, n * sizeof(double), cudaMemcpyDefault, c->stream));
    BILU_CUDA(c, cudaEventRecord(e1, c->stream));
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int32_t apst[4];
    BILU_CUDA(c, cudaMemcpy(apst, c->d_apst, sizeof(apst), cudaMemcpyDeviceToHost));
    const double eta = c->h_sqs[SS_ETA];
    if (info) {
        info->iters = c->h_sqi[SI_ITS];
        info->breakdown = c->h_sqi[SI_BREAK];
        info->backward_error = eta;
        info->relres_true = c->h_sqs[SS_REL];
        info->t_solve_ms = ms;
    }
    if (apst[3] != 0) return set_err(c, BILU_ERR_TIMEOUT, "apply kernel: bounded wait gave up");
    return eta <= tol ? BILU_OK : BILU_NOT_CONVERGED;
}
