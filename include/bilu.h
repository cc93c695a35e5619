/*
 * bilu.h -- C ABI of the GB300 (sm_103a) block incomplete LU library.
 *
 * Method: Bollhoefer, Schenk, Verbosio, "High Performance Block Incomplete LU
 * Factorization", arXiv:1908.10169.  The library computes the Crout-type block ILU
 * A ~ L D^{-1} U of a sparse matrix (Sec. 2.2), applies it as a preconditioner by block
 * forward / backward substitution, and solves A x = b with right-preconditioned
 * restarted GMRES (Sec. 4); for a symmetric A it also computes the incomplete block
 * L D L^T of the symmetric variant and solves with simplified QMR (Sec. 4.2).  Every
 * numerical step runs in CUDA kernels on one GPU.
 *
 * Conventions (all entry points):
 *   - The caller owns every array it passes; the library copies what it keeps and
 *     never frees caller memory.  A context owns all device memory it allocates.
 *   - Vectors passed to bilu_apply / gmres_solve / sqmr_solve may be device pointers or
 *     host pointers (pageable or pinned); host vectors are staged through device buffers.
 *     Work is issued on the context's stream; the calls that return numerical status
 *     (bilu_factor, gmres_solve, sqmr_solve) synchronize that stream before returning.
 *   - Call order: bilu_create -> bilu_analyze -> bilu_factor -> bilu_apply /
 *     gmres_solve / sqmr_solve.  A call out of order returns BILU_ERR_STATE.  bilu_factor may be
 *     repeated (new drop tolerance); bilu_analyze may be repeated (new matrix).
 *   - Status < 0 is an error (the context stays destroyable, bilu_last_error says
 *     why); status > 0 is a warning with a valid result.  No exception, exit() or
 *     device trap crosses this interface.
 *   - A context is not thread-safe: use one per host thread.
 *   - Real FP64 values, int32 column indices, int64 row pointers, 0-based.
 */
#ifndef BILU_H
#define BILU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bilu_ctx bilu_ctx;

typedef enum {
    BILU_OK = 0,
    BILU_NOT_CONVERGED = 1, /* gmres_solve reached maxit; x holds the last iterate      */
    BILU_PERTURBED = 2,     /* some diagonal blocks were perturbed (Sec. 3.6)           */
    BILU_ERR_ARG = -1,      /* invalid argument (bad CSR, NaN, size, null pointer)      */
    BILU_ERR_OOM = -2,      /* device allocation failed                                 */
    BILU_ERR_CUDA = -3,     /* a CUDA runtime call failed                               */
    BILU_ERR_SINGULAR = -4, /* singular diagonal block with perturbation switched off   */
    BILU_ERR_TIMEOUT = -5,  /* a device-side wait exceeded its iteration bound          */
    BILU_ERR_STATE = -6     /* call out of order                                        */
} bilu_status;

enum { BILU_BLOCKING_FIXED = 0, BILU_BLOCKING_ILU1T = 1 };
enum { BILU_PREC_FP64 = 0, BILU_PREC_FP32 = 1, BILU_PREC_BF16 = 2 };
enum { BILU_SKIP_NONE = 0, BILU_SKIP_BOUND = 1, BILU_SKIP_LEARNED = 2 };
enum { BILU_SCHED_CHAIN = 0, BILU_SCHED_TREE = 1 };

/* Maximum diagonal block size supported by the kernels. */
#define BILU_MAX_BLOCK 64

typedef struct {
    int32_t blocking;    /* BILU_BLOCKING_FIXED: consecutive blocks of fixed_block;
                            BILU_BLOCKING_ILU1T: the simplified ILU(1,tau) guess of Sec. 3.4 */
    int32_t max_block;   /* cap on the block size, 1..BILU_MAX_BLOCK (the paper asks for a
                            limit, Sec. 3, without fixing one)                                 */
    int32_t fixed_block; /* block size for BILU_BLOCKING_FIXED                                 */
    double tau_analyze;  /* tau of the ILU(1,tau) simulation                                    */
    int32_t perturb;     /* 1: perturb singular diagonal blocks (Sec. 3.6); 0: report singular */
    double pert_tau;     /* absolute perturbation tolerance tau (paper: 1e-2)                  */
    double pert_rho;     /* relative perturbation tolerance rho (paper: 1e-1)                  */
    int32_t precision;   /* BILU_PREC_*: arithmetic of the Schur updates and panel scaling.
                            BILU_PREC_BF16: BF16 storage of L and U-breve; the Schur updates of
                            the candidate rows run on the tensor cores (tcgen05 MMA, BF16
                            operands, FP32 accumulation in tensor memory) unless a skip mode or
                            sample recording is on                                              */
    int32_t skip;        /* BILU_SKIP_*: candidate-row skipping in the factorization.
                            BILU_SKIP_BOUND: after D_K is known, a candidate row i is skipped
                            when (||A(i,B_K)|| + sum_J ||L_J(i,:)|| ||U_J(:,B_K)||_F) ||D_K||_F
                            <= tau (1 - 1e-10), which proves ||l_i|| <= tau (triangle inequality,
                            ||D_K||_2 <= ||D_K||_F); columns likewise.  Same factor as without.
                            BILU_SKIP_LEARNED: a classifier decides before the updates (see
                            bilu_set_skip_model); needs a model.                                */
    int32_t schedule;    /* BILU_SCHED_CHAIN: the blocks are factored one after another by the
                            whole GPU.  BILU_SCHED_TREE: the block elimination tree of the
                            partition (see bilu_block_etree) is built by bilu_analyze, and groups
                            of group_ctas CTAs factor independent subtrees side by side, each
                            block after all of its children (every block that updates K lies in
                            K's subtree, Sec. 3.3); the chain of single-child blocks at the top
                            of the tree (the trunk) is then factored by the whole GPU.  Same
                            factor, bit for bit, as BILU_SCHED_CHAIN on the same ordering.  It
                            pays off on an ordering with independent subtrees (nested
                            dissection, bilu_nd_order); in natural order the tree is a chain.
                            Not with BILU_SKIP_LEARNED or sample recording (BILU_ERR_ARG).      */
    int32_t group_ctas;  /* CTAs per group of BILU_SCHED_TREE, 1..number of SMs (0: by A's
                            coupling: 8 groups when its rows hold >= 32 entries on average, else
                            15 groups, 19 with BF16 storage; a size that does not divide the SM
                            count leaves the remaining CTAs to the trunk)                       */
    int32_t aggregate_max; /* progressive aggregation (Sec. 3.5), 0 (off) or 2..BILU_MAX_BLOCK:
                            consecutive finished blocks k-1, k are merged into one block of at
                            most this many columns whenever the merge test of Sec. 3.5 holds
                            (nu <= 1.2 mu or nu <= mu + 2 (p + q), mu / nu the stored values
                            before / after); block k-1 becomes void (size 0) and block k holds
                            both.  The merged block stores the union of the rows (columns) and
                            L-hat = L_{:,G} L_GG^{-1}, U-hat = L_GG U-breve_{G,:}, P-hat = L_GG T_GG,
                            D-hat = P-hat^{-1} for the merged group G (L_GG its unit lower part,
                            T_GG its upper part with the pivot blocks): the product of the factors
                            is unchanged, so the preconditioner is the same operator.  Applied
                            after the factorization, in block order, to the finished factor
                            (every schedule); the sweeps, the solves and bilu_export then use
                            the merged blocks (bilu_get_factor_partition).                    */
    int32_t symmetric;   /* 1: BILDL, the symmetric variant (Sec. 4.2): A must equal A^T entry
                            by entry (BILU_ERR_ARG otherwise).  The factor is an incomplete block
                            L D L^T: only the block columns of L are computed (the row blocks of
                            U-breve are their transposes, half the update and scaling work), the
                            pivot block is the lower triangle of P_K mirrored, perturbed on its
                            diagonal only (Sec. 3.6), and D_K = (X + X^T) / 2 for the computed
                            inverse X, so that M = L P L^T and the sweeps apply a symmetric
                            M^{-1}.  Same storage as BILU (U-breve's column i holds L's
                            unnormalised row i).  Not with a skip mode, sample recording or
                            aggregation (BILU_ERR_ARG).  0: BILU.                                */
} bilu_params;

typedef struct {
    int32_t iters;          /* SQMR steps taken (one product with A, one with M^{-1})    */
    int32_t breakdown;      /* 1: sigma = q^T A q or rho = r^T M^{-1} r vanished          */
    double backward_error;  /* ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) at exit */
    double relres_true;     /* ||b - A x||_2 / ||b||_2 at exit                            */
    double t_solve_ms;      /* device time of the solve                                   */
} sqmr_info;

typedef struct {
    int32_t iters;       /* inner Arnoldi steps taken                                  */
    int32_t restarts;    /* completed restart cycles                                  */
    double relres_true;  /* ||b - A x|| / ||b|| at exit                                */
    double relres_est;   /* last Givens residual estimate |g_{j+1}| / ||b||            */
    double t_solve_ms;   /* device time of the solve                                   */
} gmres_info;

typedef struct {
    int64_t n, nnz_a;         /* matrix size and nonzeros                              */
    int32_t nblocks;          /* number of diagonal blocks                             */
    int32_t max_bsize;        /* largest block                                         */
    double avg_bsize, std_bsize;
    int64_t nnz_l, nnz_u;     /* stored values of L and U-breve (kept rows x block)    */
    int64_t nnz_d;            /* sum of b_K^2                                          */
    int64_t kept_rows, kept_cols;   /* kept scalar rows of L / columns of U            */
    int64_t cand_rows, cand_cols;   /* candidate rows / columns before dropping        */
    int64_t nperturb;         /* perturbed entries (Sec. 3.6)                          */
    double flops_factor;      /* algorithmic flops of the last factorization: the sum of
                                 the four counts below plus 2 b_K^3 per block (getrf 2/3,
                                 inverse 4/3)                                           */
    int64_t flop_upd_l;       /* 2 m n b_J summed over the L-side block updates        */
    int64_t flop_upd_u;       /* 2 m n b_J summed over the U-side block updates        */
    int64_t flop_scale;       /* 2 b_K^2 per candidate row and column (D_K products),
                                 skipped and bound-dropped candidates excluded          */
    int64_t flop_norm;        /* 2 b_K per candidate row and column (drop norms), ditto */
    double t_analyze_ms, t_factor_ms;
    int32_t pool_retries;     /* factor re-runs after growing the L/U pools             */
    int64_t kernel_launches;  /* kernels of this library launched on the context so far
                                 (each node of a launched CUDA graph counts once)       */
    double phase_ms[8];       /* factorization time by phase, each up to the end of its
                                 grid barrier (tree schedule: summed over the groups): candidate sets; pivot-row updates + pivot
                                 LU (other updates overlap); inverse; bound-tested
                                 updates (norm-bound skip only); scaling + dropping;
                                 compaction.  Then CTA 0's time inside the pivot LU and
                                 waiting for the pivot-row updates                      */
    int64_t skipped_rows;     /* candidate rows / columns skipped (norm bound proved them */
    int64_t skipped_cols;     /* dropped, or the classifier predicted it): not computed  */
    int32_t schedule;         /* BILU_SCHED_* of the analysis                            */
    int32_t tree_height;      /* BILU_SCHED_TREE: blocks on the longest leaf-to-root path */
    int32_t tree_trunk;       /*   blocks of the trunk (factored by the whole GPU)        */
    int32_t group_ctas;       /*   CTAs per group                                         */
    double idle_ms;           /*   time the groups waited for a ready block, summed over
                                   the groups (0 for the chain schedule)                 */
    int64_t bound_drops;      /* candidates dropped unscaled: the upper bound
                                 sum_k |T_ik| ||D_K(k,:)|| of the norm (columns: with the
                                 column norms of D_K) was already <= tau, so the product
                                 would have dropped them too; the factor is unchanged    */
    int32_t agg_merges;       /* progressive aggregation: blocks merged into their
                                 successor (void blocks of the factor); 0 when off       */
    int32_t agg_max_bsize;    /* largest block of the factor after the merges            */
    double t_aggregate_ms;    /* host + device time of the merges (part of bilu_factor)  */
} bilu_stats_t;

/* Fills *p with the defaults: FIXED blocking of 32 (max 64), tau_analyze 1e-2,
 * perturbation on with tau 1e-2 and rho 1e-1 (Sec. 3.6), FP64, no skipping, the chain
 * schedule (group_ctas 0: chosen by the library), no aggregation, BILU (symmetric 0).
 * Errors: BILU_ERR_ARG (p NULL). */
bilu_status bilu_params_default(bilu_params *p);

/* Creates a context (the library's runtime state; no counterpart in the paper) on CUDA
 * device `device`, issuing work on `cuda_stream` (a cudaStream_t).  NULL makes the context create and own a private non-blocking stream
 * (the solver captures CUDA graphs, which the legacy default stream does not allow).
 * Errors: BILU_ERR_ARG (no such device), BILU_ERR_CUDA (device lacks cooperative launch). */
bilu_status bilu_create(bilu_ctx **ctx, int device, void *cuda_stream);

/*
 * Analysis (Sec. 2.2 setting up the structures; Sec. 3.4 blocking): validates and copies
 * A (n x n CSR: rowptr[n+1] int64, colind[nnz] int32 sorted and unique within each row,
 * val[nnz] finite FP64; host pointers if on_device == 0, device pointers otherwise),
 * builds its CSC copy (access by columns, Sec. 2.1), computes the block partition and
 * sizes the factor's memory.  Errors: BILU_ERR_ARG for a malformed matrix or
 * parameters, BILU_ERR_OOM, BILU_ERR_CUDA.
 */
bilu_status bilu_analyze(bilu_ctx *ctx, int64_t n, const int64_t *rowptr, const int32_t *colind,
                         const double *val, int32_t on_device, const bilu_params *p);

/*
 * Numeric factorization (Algorithm 1 with blocks, Sec. 2.2): for each diagonal block K,
 * the block column of L and block row of U are loaded from A, updated by the earlier
 * blocks (dense products scattered into the target rows), the diagonal block is
 * factored with partial pivoting inside the block and inverted (perturbed if singular,
 * Sec. 3.6), the off-diagonal rows l_i = T[i,:] D_K and columns D_K u_j are computed,
 * and a scalar row / column is dropped when its Euclidean norm is <= droptol.
 * Returns BILU_OK, BILU_PERTURBED, BILU_ERR_SINGULAR (perturb == 0), BILU_ERR_TIMEOUT,
 * BILU_ERR_OOM, BILU_ERR_CUDA, BILU_ERR_STATE (no analysis), BILU_ERR_ARG (droptol < 0).
 * BILU_ERR_OOM also reports a block updated by more than 1024 earlier blocks (the kernels'
 * per-block producer list lives in shared memory): a partition whose blocks do not follow the
 * matrix's structure (for instance fixed blocks after a matching that scrambled the order)
 * needs a blocking or reordering first (Sec. 3.2-3.4).
 */
bilu_status bilu_factor(bilu_ctx *ctx, double droptol);

/*
 * z = M^{-1} r with M = L D^{-1} U (Sec. 2.2: block forward substitution with unit L,
 * then block backward substitution multiplying by the stored inverses D_K).
 * r and z hold n doubles and must not overlap.  Stream-ordered; does not synchronize
 * for device pointers.  Errors: BILU_ERR_STATE (no factor), BILU_ERR_ARG, BILU_ERR_CUDA.
 */
bilu_status bilu_apply(bilu_ctx *ctx, const double *r, double *z);

/*
 * Restarted GMRES(restart), right preconditioned with M (Sec. 4 uses GMRES(30)):
 * solves A x = b; x holds x0 on entry and the solution on exit.  Stops when the Givens
 * residual estimate is <= tol ||b|| and the true residual ||b - A x|| <= tol ||b||, or
 * after maxit inner steps (BILU_NOT_CONVERGED).  info may be NULL.  b and x hold n doubles,
 * device or host memory.  Errors: BILU_ERR_STATE (no factor), BILU_ERR_ARG (null vector,
 * restart outside 1..1000, maxit < 0, tol < 0 or NaN), BILU_ERR_OOM, BILU_ERR_CUDA,
 * BILU_ERR_TIMEOUT (a device-side wait gave up).
 */
bilu_status gmres_solve(bilu_ctx *ctx, const double *b, double *x, double tol, int32_t restart,
                        int32_t maxit, gmres_info *info);

/*
 * Simplified QMR (Freund and Nachtigal), the solver the paper pairs with BILDL (Sec. 4.2),
 * preconditioned with the context's factor (symmetric when it was made with
 * params.symmetric = 1; A must then be symmetric as well).  No look-ahead.  With the BCG
 * residual r, direction q and rho = r^T M^{-1} r, one step takes sigma = q^T A q,
 * alpha = rho / sigma, r -= alpha A q, theta' = ||r|| / tau, c = (1 + theta'^2)^{-1/2},
 * tau = tau theta' c, d = c^2 theta^2 d + c^2 alpha q, x += d, u = M^{-1} r,
 * rho' = r^T u, q = u + (rho' / rho) q.  Stops when the normwise backward error of x,
 * ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), is <= tol (the paper uses 1e-6),
 * checked after every step; after maxit steps (BILU_NOT_CONVERGED); or at a breakdown
 * (sigma or rho zero: BILU_NOT_CONVERGED with info->breakdown = 1).  x holds x0 on entry
 * and the last iterate on exit; b and x hold n doubles, device or host memory; info may be
 * NULL.  The steps run as CUDA graphs of 8 steps each; a step after convergence returns at
 * once.  Errors: BILU_ERR_STATE (no factor), BILU_ERR_ARG (null vector, maxit < 0, tol < 0
 * or NaN), BILU_ERR_OOM, BILU_ERR_CUDA, BILU_ERR_TIMEOUT (a sweep's bounded wait gave up).
 */
bilu_status sqmr_solve(bilu_ctx *ctx, const double *b, double *x, double tol, int32_t maxit, sqmr_info *info);

/*
 * Batched factorization of many independent matrices in one persistent launch.  Every
 * context holds one analysed matrix (bilu_analyze); all must live on the same device and
 * share precision, skip and perturbation settings; work is issued on ctxs[0]'s stream.
 * The grid is split into groups of CTAs; each group takes the next matrix from a device
 * work queue (largest first) and runs the block recurrence of Algorithm 1 (Sec. 2.2) on
 * it.  The group size is tuned by timing candidates on the second call for a given (matrix
 * count, largest block, precision) and cached process-wide (the cache is locked, so
 * batches on disjoint contexts may be factored from different host threads); the first
 * call uses a size from the count.  Each context ends as after bilu_factor on it;
 * statuses as bilu_factor (the worst one is returned, details in bilu_last_error of ctxs[0]).
 * Allocates and frees small device buffers per call.  Synchronizes the device.
 */
bilu_status bilu_factor_batch(bilu_ctx *const *ctxs, int32_t count, double droptol);

/*
 * Restarted GMRES(restart) on the systems of a batch (Sec. 4), as gmres_solve on each
 * context: b[i], x[i] (device or host) of ctxs[i]'s size; info (count entries) may be NULL.
 * One CUDA graph holds a restart cycle of every system as a parallel branch; converged
 * systems are stopped between cycles.  Returns BILU_NOT_CONVERGED if any system did not
 * converge within maxit inner steps.  Work on ctxs[0]'s stream; synchronizes it.
 */
bilu_status gmres_solve_batch(bilu_ctx *const *ctxs, int32_t count, const double *const *b, double *const *x,
                              double tol, int32_t restart, int32_t maxit, gmres_info *info);

/* Statistics of the last analysis / factorization (fill, block sizes, the algorithmic work
 * of Algorithm 1 with blocks, Sec. 2.2, as counted on the device) into *out (caller-owned).
 * Errors: BILU_ERR_ARG (NULL), BILU_ERR_STATE (no analysis). */
bilu_status bilu_stats(bilu_ctx *ctx, bilu_stats_t *out);

/* Copies the block partition (Sec. 3.4 or fixed) to host memory: bstart[nblocks + 1]
 * (caller-owned; nblocks from bilu_stats).  Errors: BILU_ERR_ARG (NULL), BILU_ERR_STATE. */
bilu_status bilu_get_partition(bilu_ctx *ctx, int32_t *bstart);

/* Copies the block boundaries of the factor (nblocks + 1 entries, caller-owned host memory):
 * the analysis partition, or after progressive aggregation (aggregate_max) the merged one,
 * void blocks having bstart[K] == bstart[K+1] (Sec. 3.5).  The export's per-block arrays
 * (Lptr, Uptr, the value layouts) follow these boundaries.
 * Errors: BILU_ERR_ARG (NULL), BILU_ERR_STATE (no factor), BILU_ERR_CUDA. */
bilu_status bilu_get_factor_partition(bilu_ctx *ctx, int32_t *bstart);

/*
 * Copies the factor to host memory in the layout:
 *   Lptr[nb+1] kept-row offsets; Lrow[kept_rows] global rows (sorted per block);
 *   Lval[nnz_l] per block kept_rows_K x b_K row-major (rows of unit L);
 *   Uptr[nb+1]; Ucol[kept_cols]; Uval[nnz_u] per block kept_cols_K x b_K, entry (q,t) =
 *   U-breve(s_K + t, Ucol[q]); Dinv[nnz_d] per block b_K x b_K row-major (D_K = P_K^{-1});
 *   Pblk[nnz_d] the updated pivot blocks P_K.  Any pointer may be NULL.  All host arrays,
 *   caller-owned, sized from bilu_stats; the factor is A ~ L D^{-1} U of Sec. 2.2 with
 *   L D^{-1} U = L U-breve.  Reduced-precision factors are widened to FP64.  With
 *   progressive aggregation the blocks are those of bilu_get_factor_partition.
 * Errors: BILU_ERR_ARG (NULL context), BILU_ERR_STATE (no factor), BILU_ERR_CUDA.
 */
bilu_status bilu_export(bilu_ctx *ctx, int64_t *Lptr, int32_t *Lrow, double *Lval, int64_t *Uptr,
                        int32_t *Ucol, double *Uval, double *Dinv, double *Pblk);

/* Human-readable description of the last error on this context ("" if none).  With
 * ctx == NULL: the last error of this host thread's context-free calls
 * (bilu_cosine_blocking, bilu_cosine_blocking_units, bilu_partition_ilu1t, bilu_mwm, bilu_sym_mwm,
 * bilu_scale_permute_csr,
 * bilu_nd_order, bilu_block_etree, bilu_permute_csr). */
const char *bilu_last_error(const bilu_ctx *ctx);

/*
 * Cosine-based blocking (Sec. 3.2), host only: no context, no device, no allocation visible
 * to the caller.  Rows i and j of A (n x n CSR as in bilu_analyze; the values are not read)
 * are grouped when their 0/1 patterns c_i, c_j satisfy |c_i n c_j|^2 >= tau |c_i| |c_j|
 * (the paper uses tau = 0.8), checked over the pairs j > i that share a column and are not
 * yet in a block.  Rows are visited in increasing order; a row not yet in a block leads a new
 * block and takes its passing partners in increasing order, up to max_block (1..64) rows.
 * An index whose row or column holds more than mu + 2 sigma entries (mu = nnz / n, sigma
 * the standard deviation of the row, resp. column, counts; decided in exact integer
 * arithmetic) takes no part and forms a block of its own.
 * Outputs (caller-owned host arrays): perm[n], the original index at every new position
 * (the symmetric permutation Q with A~ = Q^T A Q, A~[k][l] = A[perm[k]][perm[l]]; the blocks
 * in the order of their leaders, each as leader then members ascending); bstart[n + 1], of
 * which the first *nblocks + 1 entries are the block starts of A~; *nblocks.
 * Errors: BILU_ERR_ARG (malformed pattern, tau < 0 or not finite, max_block out of range,
 * null output), message in bilu_last_error(NULL).
 */
bilu_status bilu_cosine_blocking(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                 int32_t max_block, int32_t *perm, int32_t *bstart, int32_t *nblocks);

/*
 * The simplified ILU(1,tau) block-pattern guess of Sec. 3.4 on the host (the partition that
 * bilu_analyze builds with BILU_BLOCKING_ILU1T), no context or device.  A as in bilu_analyze
 * (host arrays, values read); tau >= 0 the analysis threshold; max_block 1..64.  With
 * gstart == NULL columns join a block one at a time; otherwise gstart[ngroups + 1]
 * (0 = gstart[0] < ... < gstart[ngroups] = n, groups of 1..max_block) are the units of growth,
 * for instance the cosine blocks of Sec. 3.2: a group joins (or starts) a block as a whole, by
 * the same rule with its columns' pattern unions and scalar counts.  bstart[n + 1] (caller-
 * owned) receives the block starts, *nblocks their number.  Errors: BILU_ERR_ARG, message in
 * bilu_last_error(NULL).
 */
bilu_status bilu_partition_ilu1t(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                 double tau, int32_t max_block, int32_t ngroups, const int32_t *gstart,
                                 int32_t *bstart, int32_t *nblocks);

/*
 * Maximum weight matching with scaling (Sec. 3.1), host only: no context or device.  With
 * costs c_ij = log a_j - log|a_ij| on the stored nonzeros of A (a_j = max_k |a_kj|), finds a
 * perfect matching sigma (row i -> column sigma[i]) of least total cost, i.e. of largest
 * product of |a_{i sigma(i)}| (a maximum product transversal), by shortest augmenting paths,
 * and dual variables u, v (u_i + v_j <= c_ij, equal on the matching).  Outputs (caller-owned
 * host arrays of n entries): sigma; dl[i] = e^{u_i}; dr[j] = e^{v_j} / a_j.  Then
 * A^ = D_l A D_r Pi (column sigma[i] moved to position i, see bilu_scale_permute_csr) has
 * |a^_ij| <= 1 and |a^_ii| = 1.  To solve A x = b: solve A^ y = D_l b, then
 * x[sigma[l]] = dr[sigma[l]] y[l].
 * Errors: BILU_ERR_ARG (malformed CSR, non-finite value, null array), BILU_ERR_SINGULAR (no
 * perfect matching on the nonzeros: A is structurally singular); message in
 * bilu_last_error(NULL).
 */
bilu_status bilu_mwm(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val, int32_t *sigma,
                     double *dl, double *dr);

/*
 * Cosine blocking of the compressed matrix (Sec. 4.2: after the symmetrised matching the
 * 2 x 2 pivots are merged before the cosine test), host only.  The consecutive units
 * [ustart[p], ustart[p + 1]), p < nunits (sizes 1..max_block, from 0 to n), are the indices of
 * the compressed pattern, whose row p holds the units of the columns of A's rows in unit p;
 * the blocking of bilu_cosine_blocking runs on it with one change: a unit adds its size to its
 * block, which holds at most max_block indices of A (a partner that passes the test but does
 * not fit is passed over).  Outputs as in bilu_cosine_blocking, over the indices of A: perm[n]
 * (the units of each block in the block's order, the indices of a unit in theirs) and
 * bstart[nblocks + 1] (every block made of whole units).  Errors: BILU_ERR_ARG (malformed CSR
 * or units, tau < 0 or not finite, max_block outside 1..64, null array).
 */
bilu_status bilu_cosine_blocking_units(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                      int32_t max_block, int32_t nunits, const int32_t *ustart, int32_t *perm,
                                      int32_t *bstart, int32_t *nblocks);

/*
 * The symmetrised matching of the symmetric variant (Sec. 4.2; Duff and Pralet), host only.
 * A must equal A^T entry by entry (n x n CSR as in bilu_analyze).  With the matching sigma and
 * the scalings d_l, d_r of bilu_mwm, ds = sqrt(d_l d_r) is a symmetric scaling with
 * |ds_i a_ij ds_j| <= 1, and the cycles of sigma give pivot units: a cycle of one index is a
 * 1 x 1 unit (|a^_ii| = 1), of two indices a 2 x 2 unit (|a^_{i,i+1}| = 1); a longer cycle
 * c_0 .. c_{k-1} is cut into pairs of neighbours (c_t, c_{t+1}), whose coupling is a matched
 * entry -- for even k the cut starting at c_0 or c_1 with the larger sum of log |a_pair|, for
 * odd k the cut leaving c_s alone that maximises log |a_{c_s c_s}| + sum log |a_pair| (the first
 * on ties, a zero diagonal counting as -inf).  Units are ordered by their smallest index, the
 * indices of a unit increasing.  Outputs (caller-owned host arrays): perm[n], the original
 * index at each new position; ds[n], indexed by original index; ustart[n + 1] and *nunits:
 * the units in the new order, [ustart[u], ustart[u + 1]).  A^ = P^T D A D P is then
 * bilu_scale_permute_csr(rowperm = colperm = perm, dl = dr = ds), exactly symmetric; to solve
 * A x = b: solve A^ y = (ds b)[perm], then x[perm] = ds[perm] y.  A partition whose
 * boundaries are unit boundaries keeps every 2 x 2 pivot inside one diagonal block.
 * Errors: BILU_ERR_ARG (malformed CSR, A not symmetric, null array), BILU_ERR_SINGULAR (no
 * perfect matching); message in bilu_last_error(NULL).
 */
bilu_status bilu_sym_mwm(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val, int32_t *perm,
                         double *ds, int32_t *ustart, int32_t *nunits);

/*
 * B[k][l] = A[r_k][c_l] * (dl[r_k] * dr[c_l]) on the host (one product of the two scalings, so
 * that dl = dr keeps a symmetric A symmetric bit for bit), with r_k = rowperm[k] and
 * c_l = colperm[l] (a NULL permutation is the identity, a NULL scaling is 1): rowperm = NULL,
 * colperm = sigma and the scalings of bilu_mwm give A^ = D_l A D_r Pi; rowperm = colperm = Q
 * and no scaling give Q^T A Q (the reorderings of Sec. 3.1-3.3).  Output arrays as in
 * bilu_permute_csr (rows sorted).
 * Errors: BILU_ERR_ARG (malformed CSR, a permutation that is not one, null array).
 */
bilu_status bilu_scale_permute_csr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                   const int32_t *rowperm, const int32_t *colperm, const double *dl,
                                   const double *dr, int64_t *out_rowptr, int32_t *out_colind, double *out_val);

/*
 * Block nested dissection (Sec. 3.3), host only: the blocks bstart[nblocks + 1] of A (pattern
 * only) are compressed to the companion graph (K ~ L when A couples B_K and B_L, either
 * direction), which is reordered by George's level-structure dissection (in place of the
 * paper's METIS): a connected set of more than `leaf` (>= 1) blocks is split by the middle
 * level of a breadth-first level structure from a pseudo-peripheral block, ordered as first
 * part, second part, separator; sets with fewer than 3 levels stay in increasing order.  The
 * block order is expanded to the unknowns with every block kept whole.  Outputs (caller-
 * owned): perm[n] (original index at each new position; A' = P^T A P, see bilu_permute_csr),
 * bstart_out[nblocks + 1] (the blocks of A'), block_order[nblocks] (the original block at each
 * new block position).  Errors: BILU_ERR_ARG, message in bilu_last_error(NULL).
 */
bilu_status bilu_nd_order(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nblocks,
                          const int32_t *bstart, int32_t leaf, int32_t *perm, int32_t *bstart_out,
                          int32_t *block_order);

/*
 * Block elimination tree, host only: parent[K] (-1 for a root) for the blocks bstart of A in
 * their given order, from the symmetrised companion graph with the fill of block elimination
 * (each block's later neighbours become a clique; its parent is the first of them).
 * Outputs caller-owned (parent[nblocks], *height).  Errors: BILU_ERR_ARG (malformed pattern or
 * partition, NULL output), message in bilu_last_error(NULL).  Every
 * block J whose factor entries update block K (a kept row of L_J or column of U-breve_J
 * inside B_K, Algorithm 1 with blocks, Sec. 2.2) is a descendant of K, so K depends only on
 * its subtree; *height is the number of blocks on the longest leaf-to-root path (the critical
 * path of a factorization that runs independent subtrees side by side).
 */
bilu_status bilu_block_etree(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nblocks,
                             const int32_t *bstart, int32_t *parent, int32_t *height);

/*
 * Symmetric permutation A~ = Q^T A Q of a CSR matrix on the host (the reordering step of
 * Sec. 3.2): row k of A~ is row perm[k] of A, every column index j renamed to the position of
 * j in perm, each row sorted.  out_rowptr[n + 1], out_colind[nnz], out_val[nnz] are caller-
 * owned host arrays of A's sizes.  A right-hand side b becomes b[perm[k]] at position k and
 * a solution x~ of A~ maps back by x[perm[k]] = x~[k].
 * Errors: BILU_ERR_ARG (malformed CSR, perm not a permutation of 0..n-1, null array), message
 * in bilu_last_error(NULL).
 */
bilu_status bilu_permute_csr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                             const int32_t *perm, int64_t *out_rowptr, int32_t *out_colind, double *out_val);

/*
 * bilu_analyze with the block partition given by the caller (for instance the one from
 * bilu_cosine_blocking on the permuted matrix): bstart[nblocks + 1] with
 * 0 = bstart[0] < ... < bstart[nblocks] = n and every block of 1..p->max_block indices
 * (host array, copied).  With p->blocking == BILU_BLOCKING_ILU1T the given blocks are groups
 * that the Sec. 3.4 growth rule merges (as bilu_partition_ilu1t with gstart = bstart, threshold
 * p->tau_analyze); otherwise they are used as they are (p->fixed_block is not used).  Errors
 * as bilu_analyze, BILU_ERR_ARG for an invalid partition.
 */
bilu_status bilu_analyze_partition(bilu_ctx *ctx, int64_t n, const int64_t *rowptr, const int32_t *colind,
                                   const double *val, int32_t on_device, const bilu_params *p, int32_t nblocks,
                                   const int32_t *bstart);

/*
 * Test hooks for the failure paths (not for production use).  Settings are global to the
 * process and stay until changed.
 *   BILU_DEBUG_EXTRA_CTA (value 0/1): the factorization's grid barrier waits for one CTA
 *       more than the launch has, so every bounded wait expires and bilu_factor returns
 *       BILU_ERR_TIMEOUT with the GPU still usable.
 *   BILU_DEBUG_SPIN_LIMIT (value > 0): polls of one barrier wait before it gives up
 *       (0 restores the default).
 *   BILU_DEBUG_SELFTEST_RECIP (value = sample count): checks the kernels' Newton-Raphson
 *       reciprocal against the IEEE quotient 1/p on that many values over 200 binades;
 *       BILU_OK when every result is within one ulp.
 *   BILU_DEBUG_BATCH_GROUP (value >= 0): bilu_factor_batch uses groups of this many CTAs
 *       (capped at the SM count) instead of the tuned size; 0 restores tuning.
 *   BILU_DEBUG_SMALL_POOLS (value 0/1): factor storage allocated from then on starts at
 *       1024 entries per pool and 4 producers per block, so that the factorization runs
 *       again with grown storage several times (the result does not change).
 *   BILU_DEBUG_POISON (value 0/1): every factorization first fills the factor's value
 *       arrays and work arrays with NaN, so that a value the kernels fail to write shows.
 *   BILU_DEBUG_NO_TRUNK (value 0/1): the tree schedule factors every block in its CTA
 *       groups, the trunk included (same factor), instead of the trunk on the whole grid.
 *   BILU_DEBUG_TRACE (value 0/1): the tree schedule prints one line per factorization run
 *       (status, storage sizes) to stderr.
 *   BILU_DEBUG_BATCH_TRCAP (value >= 0): bilu_factor_batch's update tiles hold at most this
 *       many candidate rows (values below 4 count as 4, above 16 as 16) instead of the tuned
 *       cap; 0 restores tuning.  The factor does not change.
 *   BILU_DEBUG_NO_TENSOR (value 0/1): BF16 factorizations compute their update tiles on the
 *       FP32 units instead of the tensor cores (for comparison; the results agree within the
 *       FP32 accumulation rounding).
 */
enum {
    BILU_DEBUG_EXTRA_CTA = 1,
    BILU_DEBUG_SPIN_LIMIT = 2,
    BILU_DEBUG_SELFTEST_RECIP = 3,
    BILU_DEBUG_BATCH_GROUP = 4,
    BILU_DEBUG_SMALL_POOLS = 5,
    BILU_DEBUG_POISON = 6,
    BILU_DEBUG_NO_TRUNK = 7,
    BILU_DEBUG_TRACE = 8,
    BILU_DEBUG_BATCH_TRCAP = 9,
    BILU_DEBUG_NO_TENSOR = 10
};
bilu_status bilu_debug_set(bilu_ctx *ctx, int32_t what, int64_t value);

/*
 * bilu_apply's result without any device allocation.  The paper has no counterpart: the
 * method does not deal with memory allocation.  This entry point serves callers that cannot
 * allocate device memory at the moment they apply the preconditioner: programs whose device
 * memory belongs to a fixed pool or to another framework's allocator, and real-time loops
 * that must not enter the allocator.  bilu_apply itself allocates nothing per call, but it
 * relies on buffers created with the factor and stages host vectors through buffers
 * allocated on first use.
 *
 * z = M^{-1} r as bilu_apply computes it (the same operations; the backward sweep's sums are
 * grouped differently, so results agree to rounding), FP64 factors and device pointers only
 * (host pointers, reduced-precision factors: BILU_ERR_ARG).  Its scratch (per-block
 * completion flags and sweep state) is one fixed array of 512 KB in device memory that every
 * GPU loading the library holds until the process exits; it serves factors of at most 65536
 * diagonal blocks (more: BILU_ERR_ARG).  The first call on a device looks up that array's
 * device address (a CUDA runtime query, no allocation): make the first call on each device
 * before any stream capture.  All calls on a device share the array and each call clears
 * the part it uses: calls whose work overlaps on the GPU (other streams, other contexts)
 * race and must be ordered by the caller.  Stream-ordered on the context's stream; does not
 * synchronize.  A device-side wait that gives up (bounded; never expected) fills z with NaN.
 * Calls no cudaMalloc / cudaFree.
 */
bilu_status bilu_apply_noalloc(bilu_ctx *ctx, const double *r, double *z);

/*
 * ---- Learned skip (BILU_SKIP_LEARNED) ----------------------------------------------------
 * The paper drops a row of L (a column of U) after computing it, when its norm is <= tau
 * (Sec. 3).  The learned skip predicts that outcome before the row's Schur updates are
 * computed: a classifier maps features of candidate row i of block K (column j on the U
 * side) to a logit z of P(dropped); rows with z >= logit_hi are neither updated nor scaled
 * and count as dropped, all others are computed and tested exactly.  The paper has no such
 * predictor; a wrong "drop" changes the factor (a row that would have been kept is lost),
 * so logit_hi is chosen for a small false-drop rate on training data.
 *
 * Features (FP32, BILU_MLP_FEATURES per candidate), with lg(x) = log10(max(x, 1e-30)), the
 * candidate's producers J (blocks whose kept rows of L (columns of U-breve) contain it) and
 * X_J = its row of L_J (column of U-breve_J), Y_J = L_J's rows in B_K / U-breve_J's columns
 * in B_K:
 *   0 lg a, a = ||A(i, B_K)||           1 1 if A(i, B_K) has a nonzero, else 0
 *   2 lg s, s = sum_J ||X_J|| ||Y_J||_F   3 lg max_J ||X_J|| ||Y_J||_F
 *   4 log2(1 + number of producers)      5 lg d, d = ||D_{K-1}||_F (1/alpha for K = 0)
 *   6 lg ((a + s) d)                     7 lg tau
 *   8 b_K / 64                           9 mean b_J over the producers / 64 (0 if none)
 *   10 log2(1 + max(0, i - s_K) / 64)    11 side: 0 row of L, 1 column of U
 * Classifier: x' = (x - mean) / std, h1 = relu(W1 x' + b1), h2 = relu(W2 h1 + b2),
 * z = w3 . h2 + b3; 64 hidden units per layer; weights and biases stored in FP16, products
 * accumulated in FP32.  Model array (FP32, BILU_MLP_PARAMS entries, host memory):
 *   mean[F] std[F] W1[64][F] b1[64] W2[64][64] b2[64] w3[64] b3   (F = BILU_MLP_FEATURES)
 * the weights are rounded to FP16 wherever they are used.
 */
#define BILU_MLP_FEATURES 12
#define BILU_MLP_HIDDEN 64
#define BILU_MLP_PARAMS (2 * BILU_MLP_FEATURES + BILU_MLP_HIDDEN * BILU_MLP_FEATURES + BILU_MLP_HIDDEN + \
                         BILU_MLP_HIDDEN * BILU_MLP_HIDDEN + BILU_MLP_HIDDEN + BILU_MLP_HIDDEN + 1)

typedef struct {
    int32_t epochs;      /* passes over the samples                                     */
    int32_t batch;       /* samples per Adam step (drawn with replacement), 1..65536   */
    float lr;            /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8)           */
    uint64_t seed;       /* initial weights and sample draws                            */
} bilu_mlp_train_cfg;

/*
 * Records training samples during the following factorizations of ctx (exact ones: no
 * skipping while recording): each candidate row / column is taken with probability `rate`
 * (a counter-based hash of seed, K and slot decides), its features and its label (1 dropped,
 * 0 kept) appended until `capacity` samples are held.  capacity 0 stops recording and frees
 * the buffer.  bilu_get_samples copies up to cap samples (x: cap x F row-major, y: cap, tags:
 * cap or NULL; host or device memory) and the number held in *count.  A tag identifies the
 * candidate: K * 2^33 + side * 2^32 + its global row (side 0) or column (side 1) index.
 * Sample order is not deterministic; a factorization that re-runs with grown storage keeps
 * only the samples of its final run.  (The paper computes every candidate; the learned skip
 * predicts its drop rule, Sec. 2.2.)  Errors: BILU_ERR_ARG (capacity < 0, rate outside
 * [0, 1]; count NULL, cap < 0, or x / y NULL with cap > 0), BILU_ERR_OOM, BILU_ERR_CUDA.
 */
bilu_status bilu_record_samples(bilu_ctx *ctx, int64_t capacity, double rate, uint64_t seed);
bilu_status bilu_get_samples(bilu_ctx *ctx, float *x, float *y, int64_t *tags, int64_t cap, int64_t *count);

/*
 * Trains the classifier on n samples (x: n x F row-major, y: n labels in {0, 1}; host or
 * device memory) with the binary cross-entropy of the logits, mean over each batch: feature
 * mean / std from the samples, weights uniform in +-1/sqrt(fan-in), Adam on FP32 master
 * weights whose FP16 roundings are used in the forward and backward passes.  Deterministic
 * for a given seed.  Writes the model (host, BILU_MLP_PARAMS) and, if final_loss is not NULL,
 * the mean cross-entropy over all n samples at the end.  Runs on ctx's device and stream
 * (ctx needs no matrix); synchronizes.  Errors: BILU_ERR_ARG (NULL array, n < 1, a
 * configuration out of range), BILU_ERR_OOM, BILU_ERR_CUDA.
 */
bilu_status bilu_mlp_train(bilu_ctx *ctx, const float *x, const float *y, int64_t n, const bilu_mlp_train_cfg *cfg,
                           float *model, double *final_loss);

/* Logits of n samples (x host or device; logits host or device, n entries).
 * Errors: BILU_ERR_ARG (NULL array, n < 0, a model with non-finite entries or std <= 0),
 * BILU_ERR_OOM, BILU_ERR_CUDA. */
bilu_status bilu_mlp_forward(bilu_ctx *ctx, const float *model, const float *x, int64_t n, float *logits);

/* Gradient of the mean cross-entropy over n samples with respect to the model entries
 * (host, BILU_MLP_PARAMS; zero for mean and std), at the FP16-rounded weights.
 * Errors: BILU_ERR_ARG (NULL array, n outside 1..65536, an invalid model), BILU_ERR_OOM,
 * BILU_ERR_CUDA. */
bilu_status bilu_mlp_grad(bilu_ctx *ctx, const float *model, const float *x, const float *y, int64_t n, float *grad);

/* Installs the model used by BILU_SKIP_LEARNED factorizations of ctx: a candidate is skipped
 * when its logit is >= logit_hi (the pivot rows of a block are never skipped).  The model
 * (host, BILU_MLP_PARAMS) is copied.  Errors: BILU_ERR_ARG (NULL model, non-finite logit_hi,
 * an invalid model), BILU_ERR_OOM, BILU_ERR_CUDA. */
bilu_status bilu_set_skip_model(bilu_ctx *ctx, const float *model, double logit_hi);

/* Releases the context and all device memory it owns (synchronizing its stream first).
 * NULL is ignored; no status. */
void bilu_destroy(bilu_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* BILU_H */
