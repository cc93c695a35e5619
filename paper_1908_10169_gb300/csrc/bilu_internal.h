// Internal state of a bilu context (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bilu.h"

// Device-side status codes of the persistent kernels (host maps them to bilu_status).
enum {
    DEV_OK = 0,
    DEV_POOL_OVERFLOW = 1,   // L/U value or index pool full: host grows it and re-runs
    DEV_PROD_OVERFLOW = 2,   // a producer list is full: host grows it and re-runs
    DEV_TIMEOUT = 3,         // a bounded wait gave up
    DEV_SINGULAR = 4,        // singular diagonal block, perturbation off or not curing it
    DEV_INTERNAL = 5,        // an index check failed (never expected)
};

// Slots of the device info array written by the factor kernel.
enum {
    INFO_FAIL_BLOCK = 0,     // block at which a failure was recorded
    INFO_NPERTURB = 1,       // perturbed entries
    INFO_CAND_ROWS = 2,      // candidate rows (outside the pivot block), summed
    INFO_CAND_COLS = 3,
    INFO_MAX_PROD = 4,       // longest producer list seen
    INFO_TIMEOUT_SITE = 5,   // which wait timed out
    INFO_FLOP_UPD_L = 6,     // 2 m n b_J over the L-side updates
    INFO_FLOP_UPD_U = 7,     // 2 m n b_J over the U-side updates
    INFO_FLOP_SCALE = 8,     // 2 b_K^2 per candidate row / column
    INFO_FLOP_NORM = 9,      // 2 b_K per candidate row / column
    INFO_PHASE_NS = 10,      // 6 slots: time of the phases A, B, C, C2, D, E (CTA 0)
    INFO_C2_WORK_NS = 16,    // time CTA 0 spends inside the pivot LU
    INFO_B_WORK_NS = 17,     // time CTA 0 waits for the pivot-row tiles
    INFO_SKIP_ROWS = 18,     // candidate rows skipped (norm bound or classifier)
    INFO_SKIP_COLS = 19,     // candidate columns skipped
    INFO_IDLE_NS = 20,       // tree schedule: time the groups wait for a ready block (summed)
    INFO_BOUND_DROPS = 21,   // candidates dropped by the norm bound of phase D, unscaled
    INFO_COUNT = 24
};

struct bilu_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nsm = 0;
    int apply_grid = 0;  // CTAs of the apply sweeps (0: two per SM); batched solves use a share
    std::string err;
    int state = 0;  // 0 created, 1 analyzed, 2 factored
    bilu_params p{};

    // matrix (device copies; int32 row pointers internally, nnz < 2^31 is checked)
    int64_t n = 0, nnz = 0;
    int32_t *d_rowptr = nullptr, *d_colind = nullptr;
    double *d_val = nullptr;
    int32_t *d_colptr = nullptr, *d_rowind = nullptr;
    double *d_cval = nullptr;
    double alpha = 0.0;  // max |a_ij| (Sec. 3.6)

    // partition
    int32_t nb = 0, bmax = 0, bmin = 0;
    std::vector<int32_t> h_bstart;
    int32_t *d_bstart = nullptr, *d_blkof = nullptr;
    int64_t *d_Dptr = nullptr;
    std::vector<int64_t> h_Dptr;

    // factor pools
    int64_t capLrow = 0, capLval = 0, capUcol = 0, capUval = 0;
    int64_t *d_Lptr = nullptr, *d_Lvptr = nullptr, *d_Uptr = nullptr, *d_Uvptr = nullptr;
    int32_t *d_Lrow = nullptr, *d_Ucol = nullptr;
    double *d_Lval = nullptr, *d_Uval = nullptr;
    double *d_Uhval = nullptr;     // D_K U-breve_K, the layout of d_Uval (read by the backward sweep)
    double *d_Dinv = nullptr, *d_Pblk = nullptr;
    double *d_Lnrm = nullptr, *d_Unrm = nullptr;  // norms of the kept rows of L / columns of U-breve

    // producer lists (blocks J whose kept U columns / L rows hit block K)
    int32_t prodcap = 0;
    int32_t *d_prodL = nullptr, *d_prodLcnt = nullptr, *d_prodU = nullptr, *d_prodUcnt = nullptr;
    int32_t *d_lastL = nullptr, *d_lastU = nullptr;

    // factor scratch
    int64_t capT = 0;
    double *d_TL = nullptr, *d_TU = nullptr, *d_TUh = nullptr;
    double *d_TLP = nullptr;       // partial accumulators of the pivot rows (4 x 64 x 64)
    int32_t *d_rowsL = nullptr, *d_rowsU = nullptr;
    int32_t *d_keepL = nullptr, *d_keepU = nullptr;
    uint32_t *d_bmL = nullptr, *d_bmU = nullptr;
    int32_t *d_wbL = nullptr, *d_wbU = nullptr;        // bitmap word prefix counts
    int32_t *d_xslotL = nullptr, *d_xslotU = nullptr;  // candidate slot per producer entry
    int64_t *d_pinfoL = nullptr, *d_pinfoU = nullptr;  // per-producer update plan
    int64_t capXS = 0;
    double *d_LU = nullptr;
    double *d_nrmL = nullptr, *d_nrmU = nullptr, *d_dcolsq = nullptr;
    uint32_t *d_pivdone = nullptr;
    int32_t *d_perm = nullptr;
    int32_t *d_kstate = nullptr;   // per-step scalars (candidate counts, pivot status)
    int32_t *d_status = nullptr;
    int64_t *d_info = nullptr;
    uint32_t *d_bar = nullptr;     // grid barrier counter + generation

    // tree schedule (BILU_SCHED_TREE): block elimination tree, the ready queue, the scratch of
    // the CTA groups after group 0 (group 0 uses the scratch above) and the chunked pools
    // ("arena") that the groups fill before the closing copy into the block-ordered pools
    std::vector<int32_t> h_parent;  // parent block (-1: root)
    int32_t tree_split = 0;         // blocks [tree_split, nb) form the trunk
    int32_t tree_height = 0;
    int32_t *d_parent = nullptr;
    int32_t tree_nleaves = 0;
    int32_t tree_init_split = -1;   // the trunk start d_tree0 was built for
    char *d_grp_big = nullptr;      // per-group scratch of every group
    char *d_grp_reset = nullptr;    // per-group state cleared before every run
    size_t grp_big_bytes = 0, grp_reset_bytes = 0;  // per group
    int32_t grp_n = 0;              // groups the scratch was carved for
    int64_t grp_key[3] = {0, 0, 0}; // capT, prodcap, capXS it was carved for
    int32_t *d_tree0 = nullptr, *d_tree = nullptr;  // initial / live: pending, queue, control words
    int64_t capA[4] = {0, 0, 0, 0}; // arena capacities (rows L, values L, columns U, values U)
    // capacities a factorization ended with, kept across re-analysis: a matrix of the same
    // size, nonzero count, partition and mode starts from them instead of re-running to grow
    int64_t hint_key[5] = {-1, -1, -1, -1, -1};
    int64_t hint_cap[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int32_t hint_prodcap = 0;
    int32_t *d_aLrow = nullptr, *d_aUcol = nullptr;
    double *d_aLval = nullptr, *d_aUval = nullptr, *d_aUhval = nullptr, *d_aLnrm = nullptr, *d_aUnrm = nullptr;
    int64_t *d_aptr = nullptr;      // 6 x nb: L begin, L end, L value begin, U begin, U end, U value begin
    double idle_ms = 0.0;           // last tree factorization: time its groups waited for ready blocks

    // progressive aggregation (Sec. 3.5): the merged copy of the last factor, which the sweeps,
    // the solves and the export read when agg_merges > 0 (see factor_view)
    int32_t agg_merges = 0, agg_bmax = 0, agg_prodcap = 0;
    int64_t agg_rows = 0, agg_cols = 0, agg_nnz_l = 0, agg_nnz_u = 0, agg_nnz_d = 0;
    double t_aggregate_ms = 0.0;
    std::vector<int32_t> h_ag_bstart;
    int64_t ag_cap[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // allocated sizes of the buffers below
    int32_t *d_ag_bstart = nullptr, *d_ag_blkof = nullptr, *d_ag_Lrow = nullptr, *d_ag_Ucol = nullptr;
    int32_t *d_ag_prodU = nullptr, *d_ag_prodUcnt = nullptr, *d_ag_grp = nullptr;
    int64_t *d_ag_ptr = nullptr;   // 5 x (nb + 1): Lptr, Lvptr, Uptr, Uvptr, Dptr
    void *d_ag_Lval = nullptr, *d_ag_Uval = nullptr, *d_ag_Uhval = nullptr;
    double *d_ag_Dinv = nullptr, *d_ag_Pblk = nullptr;

    // apply
    int32_t *d_flagF = nullptr, *d_flagB = nullptr;
    int2 *d_planF = nullptr;       // per (block, forward producer): L rows inside the block
    int32_t *d_apst = nullptr;     // epoch, forward ticket, backward ticket
    double *d_stage_in = nullptr, *d_stage_out = nullptr;  // host-vector staging

    // gmres workspace
    int gm_restart = 0;
    double *d_V = nullptr, *d_w = nullptr, *d_z = nullptr, *d_r = nullptr, *d_u = nullptr;
    double *d_gb = nullptr, *d_gx = nullptr;   // right-hand side and iterate
    double *d_part = nullptr;      // reduction partials
    double *d_gm = nullptr;        // H, g, cs, sn, y, scalars
    int32_t *d_gmi = nullptr;      // integer gmres state
    double *h_gm_pinned = nullptr;
    int32_t *h_gmi_pinned = nullptr;
    cudaGraphExec_t gm_graph = nullptr;
    int gm_graph_restart = 0;
    const double *gm_graph_b = nullptr;
    double *gm_graph_x = nullptr;

    // sqmr workspace: r, t, q, d, u, residual, b, x; partials; scalar / integer state
    int64_t sq_n = -1;
    double *d_sq = nullptr, *d_sqpart = nullptr, *d_sqs = nullptr;
    int32_t *d_sqi = nullptr;
    double *h_sqs = nullptr;
    int32_t *h_sqi = nullptr;
    cudaGraphExec_t sq_graph = nullptr;
    int64_t sq_graph_kernels = 0;

    // learned skip: classifier (FP32 normalisation, FP16 weights) and sample recording
    float *d_mlp_norm = nullptr;
    void *d_mlp_w = nullptr;       // __half[MW]
    double mlp_logit_hi = 0.0;
    int64_t rec_cap = 0;           // > 0: recording samples
    uint32_t rec_thresh = 0;       // a candidate is taken when its hash (32 bits) < rec_thresh
    uint64_t rec_seed = 0;
    float *d_rec_x = nullptr, *d_rec_y = nullptr;
    int64_t *d_rec_tag = nullptr;
    unsigned long long *d_rec_count = nullptr;
    unsigned long long rec_base = 0;  // samples held before the current factorization
    float *d_featL = nullptr, *d_featU = nullptr;  // capT x F features of the current block's candidates
    int64_t feat_cap = 0;

    // results of the last factorization
    int64_t kept_rows = 0, kept_cols = 0, nnz_l = 0, nnz_u = 0, cand_rows = 0, cand_cols = 0;
    int64_t nperturb = 0, skipped_rows = 0, skipped_cols = 0, bound_drops = 0;
    int32_t pool_retries = 0;
    int64_t launches = 0;          // kernels of this library launched on the context (graph nodes included)
    int64_t gm_graph_kernels = 0;  // kernel nodes of the captured GMRES cycle
    double flops_factor = 0.0, t_analyze_ms = 0.0, t_factor_ms = 0.0;
    int64_t flop_upd_l = 0, flop_upd_u = 0, flop_scale = 0, flop_norm = 0;
    double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// The factor as the sweeps, the solves and the export read it: the factorization's own arrays,
// or, after progressive aggregation merged blocks, the merged copy.  Value arrays hold the
// storage type of the precision (FP64, FP32 or BF16).
struct FactorView {
    int32_t nb = 0, prodcap = 0;
    const int32_t *bstart = nullptr, *blkof = nullptr, *Lrow = nullptr, *Ucol = nullptr;
    const int32_t *prodU = nullptr, *prodUcnt = nullptr;
    const int64_t *Lptr = nullptr, *Lvptr = nullptr, *Uptr = nullptr, *Uvptr = nullptr, *Dptr = nullptr;
    const void *Lval = nullptr, *Uval = nullptr, *Uhval = nullptr;
    const double *Dinv = nullptr, *Pblk = nullptr;
    int64_t kept_rows = 0, kept_cols = 0, nnz_l = 0, nnz_u = 0, nnz_d = 0;
};
FactorView factor_view(const bilu_ctx *c);

// helpers shared by the translation units of the library
bilu_status set_err(bilu_ctx *c, bilu_status st, const std::string &msg);
bilu_status cuda_err(bilu_ctx *c, cudaError_t e, const char *where);
#define BILU_CUDA(ctx, call)                                       \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return cuda_err((ctx), _e, #call);  \
    } while (0)

template <class T>
cudaError_t dev_alloc(T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc((void **)p, (size_t)count * sizeof(T));
}
template <class T>
void dev_free(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// Library-internal entry points implemented in the .cu files.
bilu_status factor_run(bilu_ctx *c, double droptol);
bilu_status factor_alloc(bilu_ctx *c);
void factor_remember_pools(bilu_ctx *c);
void factor_free(bilu_ctx *c);
bilu_status apply_run(bilu_ctx *c, const double *d_r, double *d_z);
bilu_status apply_launch(bilu_ctx *c, const double *d_r, double *d_z, const int32_t *skip);
bilu_status apply_alloc(bilu_ctx *c);
void apply_free(bilu_ctx *c);
bilu_status gmres_run(bilu_ctx *c, const double *d_b, double *d_x, double tol, int restart,
                      int maxit, gmres_info *info);
void gmres_free(bilu_ctx *c);
void gmres_drop_graph(bilu_ctx *c);
void sqmr_drop_graph(bilu_ctx *c);
bilu_status sqmr_run(bilu_ctx *c, const double *b, double *x, double tol, int maxit, sqmr_info *info);
void sqmr_free(bilu_ctx *c);
bilu_status aggregate_run(bilu_ctx *c);
void aggregate_free(bilu_ctx *c);
bilu_status gmres_batch_run(bilu_ctx *const *ctxs, int count, const double *const *b, double *const *x, double tol,
                            int m, int maxit, gmres_info *info);
bilu_status factor_batch_run(bilu_ctx *const *ctxs, int count, double droptol, double *ms_out);
bilu_status analyze_run(bilu_ctx *c, int64_t n, const int64_t *rowptr, const int32_t *colind,
                        const double *val, int on_device, const bilu_params *p,
                        const int32_t *given_bstart = nullptr, int32_t given_nb = -1);
// host-only analysis helpers (no context, no device): Sec. 3.2 cosine blocking and the
// symmetric permutation of a CSR matrix; the message goes to *err
bilu_status cosine_blocking_host(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                 int32_t max_block, int32_t *perm, int32_t *bstart, int32_t *nblocks,
                                 std::string *err);
bilu_status partition_ilu1t_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                 double tau, int32_t max_block, int32_t ngroups, const int32_t *gstart,
                                 int32_t *bstart, int32_t *nblocks, std::string *err);
bilu_status mwm_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                     int32_t *sigma, double *dl, double *dr, std::string *err);
bilu_status sym_mwm_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val, int32_t *perm,
                         double *ds, int32_t *ustart, int32_t *nunits, std::string *err);
bilu_status cosine_blocking_units_host(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                       int32_t max_block, int32_t nunits, const int32_t *ustart, int32_t *perm,
                                       int32_t *bstart, int32_t *nblocks, std::string *err);
bilu_status scale_permute_csr_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                   const int32_t *rowperm, const int32_t *colperm, const double *dl,
                                   const double *dr, int64_t *out_rowptr, int32_t *out_colind, double *out_val,
                                   std::string *err);
bilu_status tree_init(bilu_ctx *c, int32_t split);
int tree_group_ctas(const bilu_ctx *c);
bilu_status nd_order_host(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nb,
                          const int32_t *bstart, int32_t leaf, int32_t *perm, int32_t *bstart_out,
                          int32_t *order_out, std::string *err);
bilu_status block_etree_host(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nb,
                             const int32_t *bstart, int32_t *parent, int32_t *height, std::string *err);
bilu_status permute_csr_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                             const int32_t *perm, int64_t *out_rowptr, int32_t *out_colind, double *out_val,
                             std::string *err);
void matrix_free(bilu_ctx *c);
void mlp_free(bilu_ctx *c);
