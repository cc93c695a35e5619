// The C ABI (include/bilu.h): argument checking, call order, host-vector staging.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bilu_internal.h"

extern int g_debug_extra_cta;
extern long long g_debug_spin_limit;
extern long long g_debug_batch_group;
extern long long g_debug_batch_trcap;
extern int g_debug_tc_off;
extern int g_debug_small_pools;
extern int g_debug_poison;
extern int g_debug_no_trunk;
extern int g_debug_trace;
int recip_selftest(int n);

bilu_status set_err(bilu_ctx *c, bilu_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

bilu_status cuda_err(bilu_ctx *c, cudaError_t e, const char *where) {
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BILU_ERR_OOM : BILU_ERR_CUDA;
}

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

bilu_status bilu_params_default(bilu_params *p) {
    if (!p) return BILU_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->blocking = BILU_BLOCKING_FIXED;
    p->max_block = 64;
    p->fixed_block = 32;
    p->tau_analyze = 1e-2;
    p->perturb = 1;
    p->pert_tau = 1e-2;  // Sec. 3.6
    p->pert_rho = 1e-1;  // Sec. 3.6
    p->precision = BILU_PREC_FP64;
    p->skip = BILU_SKIP_NONE;
    return BILU_OK;
}

bilu_status bilu_create(bilu_ctx **ctx, int device, void *cuda_stream) {
    if (!ctx) return BILU_ERR_ARG;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return BILU_ERR_ARG;
    }
    bilu_ctx *c = new (std::nothrow) bilu_ctx();
    if (!c) return BILU_ERR_OOM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete c; return BILU_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) { delete c; return BILU_ERR_CUDA; }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (!coop) { delete c; return BILU_ERR_CUDA; }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        // a private stream: graph capture is not possible on the legacy default stream
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return BILU_ERR_CUDA; }
        c->own_stream = true;
    }
    *ctx = c;
    return BILU_OK;
}

void bilu_destroy(bilu_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    gmres_free(c);
    sqmr_free(c);
    apply_free(c);
    factor_free(c);
    matrix_free(c);
    mlp_free(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

namespace {
thread_local std::string g_host_err;  // last error of this thread's context-free calls
}

const char *bilu_last_error(const bilu_ctx *c) { return c ? c->err.c_str() : g_host_err.c_str(); }

bilu_status bilu_cosine_blocking(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                 int32_t max_block, int32_t *perm, int32_t *bstart, int32_t *nblocks) {
    g_host_err.clear();
    return cosine_blocking_host(n, rowptr, colind, tau, max_block, perm, bstart, nblocks, &g_host_err);
}

bilu_status bilu_partition_ilu1t(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                 double tau, int32_t max_block, int32_t ngroups, const int32_t *gstart,
                                 int32_t *bstart, int32_t *nblocks) {
    g_host_err.clear();
    return partition_ilu1t_host(n, rowptr, colind, val, tau, max_block, ngroups, gstart, bstart, nblocks,
                                &g_host_err);
}

bilu_status bilu_mwm(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val, int32_t *sigma,
                     double *dl, double *dr) {
    g_host_err.clear();
    return mwm_host(n, rowptr, colind, val, sigma, dl, dr, &g_host_err);
}

bilu_status bilu_cosine_blocking_units(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                      int32_t max_block, int32_t nunits, const int32_t *ustart, int32_t *perm,
                                      int32_t *bstart, int32_t *nblocks) {
    g_host_err.clear();
    return cosine_blocking_units_host(n, rowptr, colind, tau, max_block, nunits, ustart, perm, bstart, nblocks,
                                      &g_host_err);
}

bilu_status bilu_sym_mwm(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val, int32_t *perm,
                         double *ds, int32_t *ustart, int32_t *nunits) {
    g_host_err.clear();
    return sym_mwm_host(n, rowptr, colind, val, perm, ds, ustart, nunits, &g_host_err);
}

bilu_status bilu_scale_permute_csr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                   const int32_t *rowperm, const int32_t *colperm, const double *dl,
                                   const double *dr, int64_t *out_rowptr, int32_t *out_colind, double *out_val) {
    g_host_err.clear();
    return scale_permute_csr_host(n, rowptr, colind, val, rowperm, colperm, dl, dr, out_rowptr, out_colind,
                                  out_val, &g_host_err);
}

bilu_status bilu_nd_order(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nblocks,
                          const int32_t *bstart, int32_t leaf, int32_t *perm, int32_t *bstart_out,
                          int32_t *block_order) {
    g_host_err.clear();
    return nd_order_host(n, rowptr, colind, nblocks, bstart, leaf, perm, bstart_out, block_order, &g_host_err);
}

bilu_status bilu_block_etree(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nblocks,
                             const int32_t *bstart, int32_t *parent, int32_t *height) {
    g_host_err.clear();
    return block_etree_host(n, rowptr, colind, nblocks, bstart, parent, height, &g_host_err);
}

bilu_status bilu_permute_csr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                             const int32_t *perm, int64_t *out_rowptr, int32_t *out_colind, double *out_val) {
    g_host_err.clear();
    return permute_csr_host(n, rowptr, colind, val, perm, out_rowptr, out_colind, out_val, &g_host_err);
}

bilu_status bilu_analyze(bilu_ctx *c, int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                         int32_t on_device, const bilu_params *p) {
    if (!c) return BILU_ERR_ARG;
    c->err.clear();
    BILU_CUDA(c, cudaSetDevice(c->device));
    return analyze_run(c, n, rowptr, colind, val, on_device, p);
}

bilu_status bilu_analyze_partition(bilu_ctx *c, int64_t n, const int64_t *rowptr, const int32_t *colind,
                                   const double *val, int32_t on_device, const bilu_params *p, int32_t nblocks,
                                   const int32_t *bstart) {
    if (!c) return BILU_ERR_ARG;
    c->err.clear();
    if (nblocks < 0) return set_err(c, BILU_ERR_ARG, "nblocks < 0");
    BILU_CUDA(c, cudaSetDevice(c->device));
    return analyze_run(c, n, rowptr, colind, val, on_device, p, bstart, nblocks);
}

bilu_status bilu_factor(bilu_ctx *c, double droptol) {
    if (!c) return BILU_ERR_ARG;
    c->err.clear();
    if (c->state < 1) return set_err(c, BILU_ERR_STATE, "bilu_factor before bilu_analyze");
    if (!(droptol >= 0.0) || !std::isfinite(droptol)) return set_err(c, BILU_ERR_ARG, "droptol must be finite and >= 0");
    if (c->p.skip == BILU_SKIP_LEARNED && !c->d_mlp_w && c->rec_cap == 0)
        return set_err(c, BILU_ERR_STATE, "BILU_SKIP_LEARNED needs a model (bilu_set_skip_model)");
    BILU_CUDA(c, cudaSetDevice(c->device));
    c->state = 1;
    gmres_drop_graph(c);  // captured graphs refer to the previous factor
    sqmr_drop_graph(c);
    if (c->p.symmetric && c->rec_cap > 0)
        return set_err(c, BILU_ERR_ARG, "the symmetric variant records no samples");
    bilu_status st = factor_run(c, droptol);
    if (st < 0) return st;
    factor_remember_pools(c);
    bilu_status sg = aggregate_run(c);
    if (sg < 0) return sg;
    bilu_status sa = apply_alloc(c);
    if (sa != BILU_OK) return sa;
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    c->state = 2;
    return st;
}

bilu_status bilu_apply(bilu_ctx *c, const double *r, double *z) {
    if (!c) return BILU_ERR_ARG;
    if (c->state < 2) return set_err(c, BILU_ERR_STATE, "bilu_apply before bilu_factor");
    if (c->n > 0 && (!r || !z)) return set_err(c, BILU_ERR_ARG, "null vector");
    if (c->n == 0) return BILU_OK;
    if (r == z) return set_err(c, BILU_ERR_ARG, "r and z must not overlap");
    BILU_CUDA(c, cudaSetDevice(c->device));
    const bool dr = is_device_ptr(r), dz = is_device_ptr(z);
    if (dr && dz) return apply_run(c, r, z);
    if (!c->d_stage_in) {
        BILU_CUDA(c, cudaMalloc((void **)&c->d_stage_in, c->n * sizeof(double)));
        BILU_CUDA(c, cudaMalloc((void **)&c->d_stage_out, c->n * sizeof(double)));
    }
    const double *rin = r;
    if (!dr) {
        BILU_CUDA(c, cudaMemcpyAsync(c->d_stage_in, r, c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        rin = c->d_stage_in;
    }
    double *zout = dz ? z : c->d_stage_out;
    bilu_status st = apply_run(c, rin, zout);
    if (st != BILU_OK) return st;
    if (!dz) {
        BILU_CUDA(c, cudaMemcpyAsync(z, zout, c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return BILU_OK;
}

bilu_status gmres_solve(bilu_ctx *c, const double *b, double *x, double tol, int32_t restart, int32_t maxit,
                        gmres_info *info) {
    if (!c) return BILU_ERR_ARG;
    c->err.clear();
    if (c->state < 2) return set_err(c, BILU_ERR_STATE, "gmres_solve before bilu_factor");
    if (c->n > 0 && (!b || !x)) return set_err(c, BILU_ERR_ARG, "null vector");
    if (info) std::memset(info, 0, sizeof(*info));
    if (c->n == 0) return BILU_OK;
    BILU_CUDA(c, cudaSetDevice(c->device));
    return gmres_run(c, b, x, tol, restart, maxit, info);
}

bilu_status sqmr_solve(bilu_ctx *c, const double *b, double *x, double tol, int32_t maxit, sqmr_info *info) {
    if (!c) return BILU_ERR_ARG;
    c->err.clear();
    if (c->state < 2) return set_err(c, BILU_ERR_STATE, "sqmr_solve before bilu_factor");
    if (c->n > 0 && (!b || !x)) return set_err(c, BILU_ERR_ARG, "null vector");
    if (info) std::memset(info, 0, sizeof(*info));
    if (c->n == 0) return BILU_OK;
    BILU_CUDA(c, cudaSetDevice(c->device));
    return sqmr_run(c, b, x, tol, maxit, info);
}

bilu_status bilu_factor_batch(bilu_ctx *const *ctxs, int32_t count, double droptol) {
    if (!ctxs || count < 1) return BILU_ERR_ARG;
    bilu_ctx *c0 = ctxs[0];
    if (!c0) return BILU_ERR_ARG;
    for (int32_t i = 0; i < count; ++i) {
        bilu_ctx *c = ctxs[i];
        if (!c) return set_err(c0, BILU_ERR_ARG, "null context in batch");
        c->err.clear();
        if (c->state < 1) return set_err(c0, BILU_ERR_STATE, "bilu_factor_batch: a context has no analysis");
        if (c->device != c0->device) return set_err(c0, BILU_ERR_ARG, "bilu_factor_batch: contexts on different devices");
        if (c->p.precision != c0->p.precision || c->p.skip != c0->p.skip || c->p.perturb != c0->p.perturb)
            return set_err(c0, BILU_ERR_ARG, "bilu_factor_batch: contexts need the same precision, skip and perturbation settings");
        for (int32_t k = 0; k < i; ++k)
            if (ctxs[k] == c) return set_err(c0, BILU_ERR_ARG, "bilu_factor_batch: a context appears twice");
    }
    if (!(droptol >= 0.0) || !std::isfinite(droptol)) return set_err(c0, BILU_ERR_ARG, "droptol must be finite and >= 0");
    for (int32_t i = 0; i < count; ++i)
        if (ctxs[i]->p.skip == BILU_SKIP_LEARNED && !ctxs[i]->d_mlp_w && ctxs[i]->rec_cap == 0)
            return set_err(c0, BILU_ERR_STATE, "BILU_SKIP_LEARNED needs a model on every context (bilu_set_skip_model)");
    BILU_CUDA(c0, cudaSetDevice(c0->device));
    for (int32_t i = 0; i < count; ++i) {
        ctxs[i]->state = 1;
        gmres_drop_graph(ctxs[i]);
        sqmr_drop_graph(ctxs[i]);
    }
    double ms = 0.0;
    bilu_status st = factor_batch_run(ctxs, count, droptol, &ms);
    if (st < 0) return st;
    for (int32_t i = 0; i < count; ++i) {
        bilu_status sg = aggregate_run(ctxs[i]);
        if (sg < 0) return sg;
        bilu_status sa = apply_alloc(ctxs[i]);
        if (sa != BILU_OK) return sa;
    }
    BILU_CUDA(c0, cudaDeviceSynchronize());
    for (int32_t i = 0; i < count; ++i) ctxs[i]->state = 2;
    return st;
}

bilu_status gmres_solve_batch(bilu_ctx *const *ctxs, int32_t count, const double *const *b, double *const *x,
                              double tol, int32_t restart, int32_t maxit, gmres_info *info) {
    if (!ctxs || count < 1 || !b || !x) return BILU_ERR_ARG;
    bilu_ctx *c0 = ctxs[0];
    if (!c0) return BILU_ERR_ARG;
    for (int32_t i = 0; i < count; ++i) {
        bilu_ctx *c = ctxs[i];
        if (!c) return set_err(c0, BILU_ERR_ARG, "null context in batch");
        if (c->state < 2) return set_err(c0, BILU_ERR_STATE, "gmres_solve_batch: a context has no factor");
        if (c->device != c0->device) return set_err(c0, BILU_ERR_ARG, "gmres_solve_batch: contexts on different devices");
        if (c->n == 0 || !b[i] || !x[i]) return set_err(c0, BILU_ERR_ARG, "gmres_solve_batch: empty system or null vector");
    }
    if (info) std::memset(info, 0, sizeof(gmres_info) * (size_t)count);
    BILU_CUDA(c0, cudaSetDevice(c0->device));
    return gmres_batch_run(ctxs, count, b, x, tol, restart, maxit, info);
}

bilu_status bilu_stats(bilu_ctx *c, bilu_stats_t *o) {
    if (!c || !o) return BILU_ERR_ARG;
    if (c->state < 1) return set_err(c, BILU_ERR_STATE, "no analysis");
    std::memset(o, 0, sizeof(*o));
    o->n = c->n;
    o->nnz_a = c->nnz;
    o->nblocks = c->nb;
    o->max_bsize = c->bmax;
    double s = 0.0, s2 = 0.0;
    for (int32_t K = 0; K < c->nb; ++K) {
        const double b = c->h_bstart[K + 1] - c->h_bstart[K];
        s += b;
        s2 += b * b;
    }
    o->avg_bsize = c->nb ? s / c->nb : 0.0;
    o->std_bsize = c->nb ? std::sqrt(std::max(0.0, s2 / c->nb - o->avg_bsize * o->avg_bsize)) : 0.0;
    o->nnz_d = c->h_Dptr.empty() ? 0 : c->h_Dptr.back();
    o->t_analyze_ms = c->t_analyze_ms;
    o->agg_max_bsize = c->bmax;
    o->kernel_launches = c->launches;
    o->schedule = c->p.schedule;
    if (c->p.schedule == BILU_SCHED_TREE) {
        o->tree_height = c->tree_height;
        o->tree_trunk = c->nb - c->tree_split;
        o->group_ctas = tree_group_ctas(c);
    }
    if (c->state >= 2) {
        // sizes of the factor as exported (after any merges)
        const FactorView v = factor_view(c);
        o->nnz_l = v.nnz_l;
        o->nnz_u = v.nnz_u;
        o->nnz_d = v.nnz_d;
        o->kept_rows = v.kept_rows;
        o->kept_cols = v.kept_cols;
        o->agg_merges = c->agg_merges;
        o->agg_max_bsize = c->agg_merges > 0 ? c->agg_bmax : c->bmax;
        o->t_aggregate_ms = c->t_aggregate_ms;
        o->cand_rows = c->cand_rows;
        o->cand_cols = c->cand_cols;
        o->nperturb = c->nperturb;
        o->t_factor_ms = c->t_factor_ms;
        o->pool_retries = c->pool_retries;
        o->flops_factor = c->flops_factor;
        o->flop_upd_l = c->flop_upd_l;
        o->flop_upd_u = c->flop_upd_u;
        o->flop_scale = c->flop_scale;
        o->flop_norm = c->flop_norm;
        for (int k = 0; k < 8; ++k) o->phase_ms[k] = c->phase_ms[k];
        o->skipped_rows = c->skipped_rows;
        o->skipped_cols = c->skipped_cols;
        o->idle_ms = c->p.schedule == BILU_SCHED_TREE ? c->idle_ms : 0.0;
        o->bound_drops = c->bound_drops;
    }
    return BILU_OK;
}

bilu_status bilu_get_factor_partition(bilu_ctx *c, int32_t *bstart) {
    if (!c || !bstart) return BILU_ERR_ARG;
    if (c->state < 2) return set_err(c, BILU_ERR_STATE, "no factor");
    const std::vector<int32_t> &b = c->agg_merges > 0 ? c->h_ag_bstart : c->h_bstart;
    std::memcpy(bstart, b.data(), b.size() * sizeof(int32_t));
    return BILU_OK;
}

bilu_status bilu_get_partition(bilu_ctx *c, int32_t *bstart) {
    if (!c || !bstart) return BILU_ERR_ARG;
    if (c->state < 1) return set_err(c, BILU_ERR_STATE, "no analysis");
    std::memcpy(bstart, c->h_bstart.data(), c->h_bstart.size() * sizeof(int32_t));
    return BILU_OK;
}

bilu_status bilu_export(bilu_ctx *c, int64_t *Lptr, int32_t *Lrow, double *Lval, int64_t *Uptr, int32_t *Ucol,
                        double *Uval, double *Dinv, double *Pblk) {
    if (!c) return BILU_ERR_ARG;
    if (c->state < 2) return set_err(c, BILU_ERR_STATE, "no factor");
    BILU_CUDA(c, cudaSetDevice(c->device));
    const FactorView v = factor_view(c);  // after any merges
    const int64_t nb1 = c->nb + 1, nd = v.nnz_d;
    auto cp = [&](void *dst, const void *src, int64_t bytes) -> cudaError_t {
        if (!dst || bytes <= 0) return cudaSuccess;
        return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    };
    BILU_CUDA(c, cp(Lptr, v.Lptr, nb1 * sizeof(int64_t)));
    BILU_CUDA(c, cp(Uptr, v.Uptr, nb1 * sizeof(int64_t)));
    BILU_CUDA(c, cp(Lrow, v.Lrow, v.kept_rows * sizeof(int32_t)));
    BILU_CUDA(c, cp(Ucol, v.Ucol, v.kept_cols * sizeof(int32_t)));
    if (c->p.precision == BILU_PREC_FP64) {
        BILU_CUDA(c, cp(Lval, v.Lval, v.nnz_l * sizeof(double)));
        BILU_CUDA(c, cp(Uval, v.Uval, v.nnz_u * sizeof(double)));
    } else {
        // reduced-precision storage: widen to FP64 on the host
        const bool f32 = c->p.precision == BILU_PREC_FP32;
        const size_t es = f32 ? 4 : 2;
        auto widen = [&](double *dst, const void *src, int64_t cnt) -> cudaError_t {
            if (!dst || cnt <= 0) return cudaSuccess;
            std::vector<unsigned char> tmp((size_t)cnt * es);
            cudaError_t e = cudaMemcpy(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return e;
            for (int64_t i = 0; i < cnt; ++i) {
                if (f32) {
                    float v;
                    std::memcpy(&v, tmp.data() + i * 4, 4);
                    dst[i] = v;
                } else {
                    uint16_t h;
                    std::memcpy(&h, tmp.data() + i * 2, 2);
                    const uint32_t w = (uint32_t)h << 16;
                    float v;
                    std::memcpy(&v, &w, 4);
                    dst[i] = v;
                }
            }
            return cudaSuccess;
        };
        BILU_CUDA(c, widen(Lval, v.Lval, v.nnz_l));
        BILU_CUDA(c, widen(Uval, v.Uval, v.nnz_u));
    }
    BILU_CUDA(c, cp(Dinv, v.Dinv, nd * sizeof(double)));
    BILU_CUDA(c, cp(Pblk, v.Pblk, nd * sizeof(double)));
    return BILU_OK;
}

bilu_status bilu_debug_set(bilu_ctx *c, int32_t what, int64_t value) {
    if (!c) return BILU_ERR_ARG;
    switch (what) {
        case BILU_DEBUG_EXTRA_CTA: g_debug_extra_cta = value ? 1 : 0; return BILU_OK;
        case BILU_DEBUG_SPIN_LIMIT: g_debug_spin_limit = value; return BILU_OK;
        case BILU_DEBUG_BATCH_GROUP: g_debug_batch_group = value > 0 ? value : 0; return BILU_OK;
        case BILU_DEBUG_NO_TENSOR: g_debug_tc_off = value ? 1 : 0; return BILU_OK;
        case BILU_DEBUG_BATCH_TRCAP: g_debug_batch_trcap = value > 0 ? std::max<int64_t>(4, value) : 0; return BILU_OK;
        case BILU_DEBUG_SMALL_POOLS: g_debug_small_pools = value ? 1 : 0; return BILU_OK;
        case BILU_DEBUG_POISON: g_debug_poison = value ? 1 : 0; return BILU_OK;
        case BILU_DEBUG_NO_TRUNK: g_debug_no_trunk = value ? 1 : 0; return BILU_OK;
        case BILU_DEBUG_TRACE: g_debug_trace = value ? 1 : 0; return BILU_OK;
        case BILU_DEBUG_SELFTEST_RECIP: {
            cudaSetDevice(c->device);
            const int bad = recip_selftest((int)value);
            if (bad == 0) return BILU_OK;
            return set_err(c, BILU_ERR_CUDA, "reciprocal self-test: " + std::to_string(bad) + " results off by more than one ulp");
        }
        default: return set_err(c, BILU_ERR_ARG, "unknown debug setting");
    }
}

}  // extern "C"
