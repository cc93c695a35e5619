/*
 * FP64 CPU oracle for the block incomplete LU (BILU) factorization, its
 * preconditioner application and restarted GMRES.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library, and never calls it.
 *
 * Source: Bollhoefer, Schenk, Verbosio, "High Performance Block Incomplete LU
 * Factorization" (arXiv:1908.10169).
 *   - Crout ILU, Algorithm 1 (Sec. 2.1); its block version (Sec. 2.2): drop
 *     l_ik when ||l_ik l_kk^{-1}|| <= tau and u_ki when ||u_kk^{-1} u_ki|| <= tau,
 *     l_ik <- l_ik l_kk^{-1}; hybrid storage: block columns of L and block rows
 *     of U with scalar row / column index arrays, dense diagonal blocks in D.
 *   - A ~ L D^{-1} U with L, U^T unit block lower triangular, the diagonal
 *     blocks factored (LU with pivoting inside the block only) and inverted
 *     (Sec. 2.2, end).
 *   - Perturbation of singular diagonal blocks (Sec. 3.6).
 *   - Progressive aggregation of consecutive blocks during the factorization (Sec. 3.5).
 *   - Simplified ILU(1,tau) block-pattern guess (Sec. 3.4).
 *   - Restarted GMRES(30) (Sec. 4, Example setup).
 *   - The symmetric variant BILDL and simplified QMR with a backward-error stop (Sec. 4.2).
 *
 * Readings where the paper is silent or garbled (all listed in the design notes):
 *   R1 drop norm = Euclidean norm of one scalar row (1 x b_K) of the normalised
 *      L block column, resp. one column (b_K x 1) of D_K * U;
 *   R2 drop iff norm <= tau (so exact zeros are dropped even at tau = 0);
 *   R3 L is stored normalised (unit), U is stored unnormalised (U-breve), D_K = P_K^{-1};
 *   R4 getrf pivot = first index of the largest |.| in the column;
 *   R5 perturbation: beta_j := 1, sign(0) := +1; triggers on an all-zero column
 *      or row, and on a pivot with |u_jj| <= 1e-14 * max|P_K|;
 *   R6 the candidate rows/cols are the structural union of touched indices;
 *   R7 updates from earlier blocks J are applied in increasing J;
 *   R8 GMRES: right preconditioning, modified Gram-Schmidt, Givens rotations,
 *      stop when the Givens residual <= tol * ||b|| and the true residual agrees.
 *   R9 ILU(1,tau) blocking bookkeeping: see orc_partition_ilu1t.
 *   R22 BILDL pivot block: the mirrored lower triangle, LU with pivoting as in step 3,
 *      perturbations on the diagonal, D_K = (X + X^T) / 2 for the computed inverse X;
 *   R23 BILDL storage: l_i in L, the unnormalised t_i as column i of U-breve;
 *   R24 SQMR: no look-ahead, normwise backward error in the infinity norm, checked after
 *      every step, x0 = 0.
 */
#ifndef BILU_ORACLE_H
#define BILU_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_factor orc_factor;

/* Status codes (same meaning as the library's, defined independently here). */
#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_PERTURBED 2
#define ORC_BREAKDOWN 3 /* SQMR: sigma or rho vanished */
#define ORC_ERR_ARG (-1)
#define ORC_ERR_SINGULAR (-4)

/* Counters filled by the factorization (algorithmic work, no padding). */
enum {
    ORC_C_FLOP_UPD_L = 0,   /* 2*m*n*b_J summed over L-side updates              */
    ORC_C_FLOP_UPD_U,       /* 2*m*n*b_J summed over U-side updates              */
    ORC_C_FLOP_GETRF,       /* (2/3) b_K^3 per diagonal block (nominal)          */
    ORC_C_FLOP_INV,         /* (4/3) b_K^3 per diagonal block (nominal)          */
    ORC_C_FLOP_SCALE,       /* 2 b_K^2 per candidate row and per candidate col   */
    ORC_C_FLOP_NORM,        /* 2 b_K per candidate row and per candidate col     */
    ORC_C_CAND_ROWS,        /* candidate (pre-drop) L rows outside the pivot     */
    ORC_C_CAND_COLS,        /* candidate (pre-drop) U cols                       */
    ORC_C_PANEL_READ_BYTES, /* 8*(m*b_J + n*b_J) per update: producer operands   */
    ORC_C_NPAIRS_L,         /* number of (J,K) L-side updates                    */
    ORC_C_NPAIRS_U,         /* number of (J,K) U-side updates                    */
    ORC_C_NPERTURB,         /* perturbed entries                                 */
    ORC_C_COUNT = 16
};

/* Partition into consecutive blocks of size b (the last one may be smaller).
 * bstart must hold n/b + 2 entries; returns the number of blocks. */
int32_t orc_partition_fixed(int64_t n, int32_t b, int32_t *bstart);

/* Simplified ILU(1,tau) block-pattern guess, Sec. 3.4.  bstart holds n+1 entries;
 * returns the number of blocks (< 0 on error). */
int32_t orc_partition_ilu1t(int64_t n, const int64_t *rowptr, const int32_t *colind,
                            const double *val, double tau, int32_t max_block,
                            int32_t *bstart);

/* The same growth rule over whole groups of columns gstart[ngroups+1] (0 = gstart[0] < ...
 * < gstart[ngroups] = n, groups of 1..max_block columns, for instance cosine blocks): a group
 * joins or starts a block as a whole.  bstart holds n+1 entries; returns the number of
 * blocks (< 0 on error). */
int32_t orc_partition_ilu1t_groups(int64_t n, const int64_t *rowptr, const int32_t *colind,
                                   const double *val, double tau, int32_t max_block, int32_t ngroups,
                                   const int32_t *gstart, int32_t *bstart);

/* Numeric Crout BILU.  A is CSR with sorted column indices.  On success (status >= 0)
 * *out receives the factor, to be freed with orc_factor_free. */
int32_t orc_bilu_factor(int64_t n, const int64_t *rowptr, const int32_t *colind,
                        const double *val, int32_t nb, const int32_t *bstart, double droptol,
                        int32_t perturb, double pert_tau, double pert_rho, orc_factor **out);

/* The same with progressive aggregation (Sec. 3.5) when agg_max > 0: after block K is
 * finished it is merged with block K-1 when the merge test holds and the merged block has at
 * most agg_max columns; block K-1 then becomes void (size 0) and block K holds both.  The
 * factor's block boundaries are then those of orc_factor_bstart.  agg_max = 0: no merging
 * (orc_bilu_factor). */
int32_t orc_bilu_factor_agg(int64_t n, const int64_t *rowptr, const int32_t *colind,
                            const double *val, int32_t nb, const int32_t *bstart, double droptol,
                            int32_t perturb, double pert_tau, double pert_rho, int32_t agg_max,
                            orc_factor **out);

/* Sec. 3.5 merge test for the counts it names (see bilu_oracle.c); 1 = merge. */
int32_t orc_agg_rule(int64_t p, int64_t q, int64_t r, int64_t s, int64_t rp, int64_t sp, int64_t t,
                     int64_t tp, int64_t u, int64_t v);

/* The factor's block boundaries (nb + 1 entries): the partition given, with merged blocks
 * (void blocks have bstart[K] == bstart[K+1]). */
void orc_factor_bstart(const orc_factor *F, int32_t *bstart);

/* sizes[0] = kept L rows, [1] = kept U cols, [2] = L values, [3] = U values,
 * [4] = sum b_K^2, [5] = number of blocks, [6] = perturbations, [7] = merges */
void orc_factor_sizes(const orc_factor *F, int64_t sizes[8]);

/* Exports the factor in the layout shared by the tests:
 *   Lptr[nb+1]   kept-row offsets; Lrow[]: global row indices (sorted per block)
 *   Lval[]       per block nL_K x b_K row-major (rows of unit L)
 *   Uptr[nb+1]   kept-col offsets; Ucol[]: global column indices (sorted per block)
 *   Uval[]       per block nU_K x b_K: entry (q, t) = U-breve(s_K + t, Ucol[q])
 *   Dinv[]       per block b_K x b_K row-major, D_K = P_K^{-1}
 *   Pblk[]       per block b_K x b_K row-major, the updated pivot block P_K
 *   LUblk[]      per block: the getrf factors of P_K (unit L below, U on and above)
 *   piv[]        per block b_K entries: row piv[i] of P_K is row i of P*P_K
 * Any pointer may be NULL to skip that array. */
void orc_factor_export(const orc_factor *F, int64_t *Lptr, int32_t *Lrow, double *Lval,
                       int64_t *Uptr, int32_t *Ucol, double *Uval, double *Dinv,
                       double *Pblk, double *LUblk, int32_t *piv);

void orc_factor_counters(const orc_factor *F, double c[ORC_C_COUNT]);
void orc_factor_free(orc_factor *F);

/* z = M^{-1} r with M = L D^{-1} U (block forward then block backward substitution). */
void orc_bilu_apply(const orc_factor *F, const double *r, double *z);

/* y = A x (plain CSR). */
void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
              const double *x, double *y);

/* Right-preconditioned restarted GMRES(restart) with MGS.  M may be NULL (no
 * preconditioner).  x holds x0 on entry.  hist (optional, maxit+1 entries) receives
 * the Givens residual estimate |g_{j+1}| / ||b|| after each inner step.
 * Returns ORC_OK or ORC_NOT_CONVERGED. */
int32_t orc_gmres(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                  const orc_factor *M, const double *b, double *x, double tol, int32_t restart,
                  int32_t maxit, int32_t *iters, double *relres_true, double *hist);

/* BILDL (Sec. 4.2): incomplete block L D L^T of a symmetric A (A must equal A^T entry by
 * entry, column indices sorted in each row; else ORC_ERR_ARG).  The factor has the BILU
 * layout: U-breve's column i holds the unnormalised row t_i of L, so orc_bilu_apply applies
 * M^{-1} = (L P L^T)^{-1}. */
int32_t orc_bildl_factor(int64_t n, const int64_t *rowptr, const int32_t *colind,
                         const double *val, int32_t nb, const int32_t *bstart, double droptol,
                         int32_t perturb, double pert_tau, double pert_rho, orc_factor **out);

/* Simplified QMR with the symmetric preconditioner M (NULL: none), stopped on the normwise
 * backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol (Sec. 4.2).
 * Returns ORC_OK, ORC_NOT_CONVERGED (maxit) or ORC_BREAKDOWN; hist (maxit + 1 entries, or
 * NULL) receives the backward error after every step. */
int32_t orc_sqmr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                 const orc_factor *M, const double *b, double *x, double tol, int32_t maxit,
                 int32_t *iters, double *berr, double *hist);

#ifdef __cplusplus
}
#endif
#endif
