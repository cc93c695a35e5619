/*
 * FP64 CPU oracle: Crout-type block ILU, its application, GMRES(m), and the
 * ILU(1,tau) block-pattern guess.  TEST INFRASTRUCTURE ONLY (see bilu_oracle.h).
 *
 * Written for clarity, not speed: single-threaded, no BLAS, every step in the
 * order of the paper's description.  Every function names the passage it follows.
 */
#include "bilu_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ helpers */

static void *xmalloc(size_t nbytes) {
    void *p = malloc(nbytes ? nbytes : 1);
    if (!p) abort();
    return p;
}
static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n ? n : 1, sz ? sz : 1);
    if (!p) abort();
    return p;
}
static void *xrealloc(void *p, size_t nbytes) {
    void *q = realloc(p, nbytes ? nbytes : 1);
    if (!q) abort();
    return q;
}

/* first position in sorted a[lo..hi) with a[pos] >= key */
static int64_t lower_bound_i32(const int32_t *a, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* growable arrays */
typedef struct { int32_t *a; int64_t n, cap; } vec_i32;
typedef struct { double *a; int64_t n, cap; } vec_f64;
static void vi_push(vec_i32 *v, int32_t x) {
    if (v->n == v->cap) { v->cap = v->cap ? 2 * v->cap : 64; v->a = xrealloc(v->a, (size_t)v->cap * sizeof(int32_t)); }
    v->a[v->n++] = x;
}
static void vd_reserve(vec_f64 *v, int64_t extra) {
    if (v->n + extra > v->cap) {
        int64_t c = v->cap ? v->cap : 256;
        while (c < v->n + extra) c *= 2;
        v->a = xrealloc(v->a, (size_t)c * sizeof(double));
        v->cap = c;
    }
}

/* CSC copy (transpose) of a CSR matrix: column j holds rows sorted increasingly. */
typedef struct { int64_t *colptr; int32_t *rowind; double *val; } csc_t;
static csc_t csr_to_csc(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val) {
    csc_t t;
    int64_t nnz = rowptr[n];
    t.colptr = xcalloc((size_t)n + 1, sizeof(int64_t));
    t.rowind = xmalloc((size_t)nnz * sizeof(int32_t));
    t.val = xmalloc((size_t)nnz * sizeof(double));
    for (int64_t e = 0; e < nnz; ++e) t.colptr[colind[e] + 1]++;
    for (int64_t j = 0; j < n; ++j) t.colptr[j + 1] += t.colptr[j];
    int64_t *fill = xmalloc((size_t)n * sizeof(int64_t));
    memcpy(fill, t.colptr, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t pos = fill[colind[e]]++;
            t.rowind[pos] = (int32_t)i;
            t.val[pos] = val[e];
        }
    free(fill);
    return t;
}
static void csc_free(csc_t *t) { free(t->colptr); free(t->rowind); free(t->val); }

static double entry(const int64_t *ptr, const int32_t *ind, const double *v, int64_t row, int32_t col) {
    int64_t p = lower_bound_i32(ind, ptr[row], ptr[row + 1], col);
    return (p < ptr[row + 1] && ind[p] == col) ? v[p] : 0.0;
}

/* ------------------------------------------------------------ partitioning */

int32_t orc_partition_fixed(int64_t n, int32_t b, int32_t *bstart) {
    if (n < 0 || b < 1) return ORC_ERR_ARG;
    int32_t nb = 0;
    for (int64_t s = 0; s < n; s += b) bstart[nb++] = (int32_t)s;
    bstart[nb] = (int32_t)n;
    return nb;
}

/*
 * Sec. 3.4, simplified local ILU(1,tau) simulation.
 * For column k:  I~_k = { i > k : a_ik != 0, |a_ik| >= tau |a_kk| }
 *                     u { i > k : a_ij != 0, a_jk != 0, j < k, |a_ij a_jk| >= tau |a_jj a_kk| }
 * and J~_k the same with rows and columns exchanged.
 * A block [k, k+l) with r rows below it in L and s columns right of it in U holds
 * f_l = (r + s + l) l entries; its scalar count grows by |I~| + |J~| + 1 per column.
 * Column k+l joins while f_{l+1} <= (4/3) s_{l+1} or f_{l+1} <= s_{l+1} + 4 (l+1),
 * and l+1 <= max_block (the paper asks for a limit without giving one).
 * Reading: the indices of the sets that fall inside the block are not counted in r, s.
 */
static void ilu1t_sets(int64_t k, const int64_t *rowptr, const int32_t *colind, const double *val,
                       const csc_t *c, double tau, int32_t *stamp, int32_t stampval,
                       vec_i32 *Iout, vec_i32 *Jout) {
    double akk = entry(rowptr, colind, val, k, (int32_t)k);
    Iout->n = 0;
    Jout->n = 0;
    /* rows: original entries of column k */
    for (int64_t e = c->colptr[k]; e < c->colptr[k + 1]; ++e) {
        int32_t i = c->rowind[e];
        if (i > k && fabs(c->val[e]) >= tau * fabs(akk) && stamp[i] != stampval) {
            stamp[i] = stampval; vi_push(Iout, i);
        }
    }
    /* rows: fill a_ik = -a_ij a_jk / a_jj from original entries, j < k < i */
    for (int64_t e = c->colptr[k]; e < c->colptr[k + 1]; ++e) {
        int32_t j = c->rowind[e];
        if (j >= k) continue;
        double ajk = c->val[e];
        double ajj = entry(rowptr, colind, val, j, j);
        for (int64_t f = c->colptr[j]; f < c->colptr[j + 1]; ++f) {
            int32_t i = c->rowind[f];
            if (i <= k) continue;
            if (fabs(c->val[f] * ajk) >= tau * fabs(ajj * akk) && stamp[i] != stampval) {
                stamp[i] = stampval; vi_push(Iout, i);
            }
        }
    }
    /* columns: the same on rows (stamp value negated keeps the two sets apart) */
    int32_t sv = -stampval;
    for (int64_t e = rowptr[k]; e < rowptr[k + 1]; ++e) {
        int32_t j = colind[e];
        if (j > k && fabs(val[e]) >= tau * fabs(akk) && stamp[j] != sv) {
            stamp[j] = sv; vi_push(Jout, j);
        }
    }
    for (int64_t e = rowptr[k]; e < rowptr[k + 1]; ++e) {
        int32_t j = colind[e];
        if (j >= k) continue;
        double akj = val[e];
        double ajj = entry(rowptr, colind, val, j, j);
        for (int64_t f = rowptr[j]; f < rowptr[j + 1]; ++f) {
            int32_t i = colind[f];
            if (i <= k) continue;
            if (fabs(akj * val[f]) >= tau * fabs(ajj * akk) && stamp[i] != sv) {
                stamp[i] = sv; vi_push(Jout, i);
            }
        }
    }
}

/*
 * The union of the sets of the columns of one group [g0, g1) (deduplicated with the stamp
 * value gsv) and its scalar count: the sum over its columns of |I~_k| + |J~_k| + 1.
 */
static int64_t ilu1t_group_sets(int64_t g0, int64_t g1, const int64_t *rowptr, const int32_t *colind,
                                const double *val, const csc_t *c, double tau, int32_t *stamp,
                                int32_t *colstamp, int32_t *inI, int32_t *inJ, int32_t gsv,
                                vec_i32 *I, vec_i32 *J, vec_i32 *GI, vec_i32 *GJ) {
    int64_t scal = 0;
    GI->n = 0;
    GJ->n = 0;
    for (int64_t k = g0; k < g1; ++k) {
        ilu1t_sets(k, rowptr, colind, val, c, tau, stamp, ++*colstamp, I, J);
        scal += I->n + J->n + 1;
        for (int64_t t = 0; t < I->n; ++t)
            if (inI[I->a[t]] != gsv) { inI[I->a[t]] = gsv; vi_push(GI, I->a[t]); }
        for (int64_t t = 0; t < J->n; ++t)
            if (inJ[J->a[t]] != gsv) { inJ[J->a[t]] = gsv; vi_push(GJ, J->a[t]); }
    }
    return scal;
}

/*
 * Sec. 3.4 growth rule over whole groups of columns (a group is never split): a block
 * [s, s+l) with r rows at or after its end in L and s' columns at or after its end in U
 * stores f = (r + s' + l) l entries; its scalar count is the sum over its columns of
 * |I~_k| + |J~_k| + 1.  The next group [e, e+g) joins while f_{l+g} <= (4/3) s_{l+g} or
 * f_{l+g} <= s_{l+g} + 4 (l+g), and l+g <= max_block.  With groups of one column this is the
 * column-by-column rule of orc_partition_ilu1t.
 */
int32_t orc_partition_ilu1t_groups(int64_t n, const int64_t *rowptr, const int32_t *colind,
                                   const double *val, double tau, int32_t max_block, int32_t ngroups,
                                   const int32_t *gstart, int32_t *bstart) {
    if (n < 0 || max_block < 1 || tau < 0 || ngroups < 0) return ORC_ERR_ARG;
    if (gstart[0] != 0 || gstart[ngroups] != n || (n > 0 && ngroups == 0)) return ORC_ERR_ARG;
    for (int32_t g = 0; g < ngroups; ++g)
        if (gstart[g + 1] - gstart[g] < 1 || gstart[g + 1] - gstart[g] > max_block) return ORC_ERR_ARG;
    csc_t c = csr_to_csc(n, rowptr, colind, val);
    int32_t *stamp = xcalloc((size_t)n + 1, sizeof(int32_t));
    int32_t *inR = xcalloc((size_t)n + 1, sizeof(int32_t));
    int32_t *inC = xcalloc((size_t)n + 1, sizeof(int32_t));
    int32_t *inI = xcalloc((size_t)n + 1, sizeof(int32_t));
    int32_t *inJ = xcalloc((size_t)n + 1, sizeof(int32_t));
    vec_i32 I = {0}, J = {0}, GI = {0}, GJ = {0}, R = {0}, C = {0};
    int32_t nb = 0, colstamp = 0, gsv = 0;
    int32_t g = 0;
    while (g < ngroups) {
        int64_t start = gstart[g];
        int32_t blk = nb + 1; /* membership stamp of this block */
        int64_t scal = ilu1t_group_sets(start, gstart[g + 1], rowptr, colind, val, &c, tau, stamp, &colstamp,
                                        inI, inJ, ++gsv, &I, &J, &GI, &GJ);
        R.n = 0; C.n = 0;
        for (int64_t t = 0; t < GI.n; ++t) { inR[GI.a[t]] = blk; vi_push(&R, GI.a[t]); }
        for (int64_t t = 0; t < GJ.n; ++t) { inC[GJ.a[t]] = blk; vi_push(&C, GJ.a[t]); }
        int64_t l = gstart[g + 1] - start;
        ++g;
        while (g < ngroups) {
            int64_t gs = gstart[g + 1] - gstart[g];
            if (l + gs > max_block) break;
            int64_t end = gstart[g + 1];
            int64_t gscal = ilu1t_group_sets(gstart[g], end, rowptr, colind, val, &c, tau, stamp, &colstamp,
                                             inI, inJ, ++gsv, &I, &J, &GI, &GJ);
            int64_t r2 = 0, s2 = 0;
            for (int64_t t = 0; t < R.n; ++t) r2 += (R.a[t] >= end);
            for (int64_t t = 0; t < GI.n; ++t) r2 += (inR[GI.a[t]] != blk && GI.a[t] >= end);
            for (int64_t t = 0; t < C.n; ++t) s2 += (C.a[t] >= end);
            for (int64_t t = 0; t < GJ.n; ++t) s2 += (inC[GJ.a[t]] != blk && GJ.a[t] >= end);
            int64_t l2 = l + gs;
            int64_t f2 = (r2 + s2 + l2) * l2;
            int64_t scal2 = scal + gscal;
            int accept = (3 * f2 <= 4 * scal2) || (f2 <= scal2 + 4 * l2);
            if (!accept) break;
            for (int64_t t = 0; t < GI.n; ++t)
                if (inR[GI.a[t]] != blk) { inR[GI.a[t]] = blk; vi_push(&R, GI.a[t]); }
            for (int64_t t = 0; t < GJ.n; ++t)
                if (inC[GJ.a[t]] != blk) { inC[GJ.a[t]] = blk; vi_push(&C, GJ.a[t]); }
            scal = scal2;
            l = l2;
            ++g;
        }
        bstart[nb++] = (int32_t)start;
    }
    bstart[nb] = (int32_t)n;
    free(stamp); free(inR); free(inC); free(inI); free(inJ);
    free(I.a); free(J.a); free(GI.a); free(GJ.a); free(R.a); free(C.a);
    csc_free(&c);
    return nb;
}

/* Column-by-column growth: every column its own group. */
int32_t orc_partition_ilu1t(int64_t n, const int64_t *rowptr, const int32_t *colind,
                            const double *val, double tau, int32_t max_block, int32_t *bstart) {
    if (n < 0 || max_block < 1 || tau < 0) return ORC_ERR_ARG;
    int32_t *unit = xmalloc(((size_t)n + 1) * sizeof(int32_t));
    for (int64_t k = 0; k <= n; ++k) unit[k] = (int32_t)k;
    int32_t nb = orc_partition_ilu1t_groups(n, rowptr, colind, val, tau, max_block, (int32_t)n, unit, bstart);
    free(unit);
    return nb;
}

/* ------------------------------------------------------------ the factor */

struct orc_factor {
    int64_t n;
    int32_t nb;
    int32_t *bstart;
    int64_t *Lptr, *Lvptr, *Uptr, *Uvptr, *Dptr;
    vec_i32 Lrow, Ucol;
    vec_f64 Lval, Uval;
    double *Dinv, *Pblk, *LUblk;
    int64_t dcap;   /* entries allocated in Dinv, Pblk, LUblk */
    int32_t *piv;
    int64_t merges; /* progressive aggregation: blocks merged into their successor (Sec. 3.5) */
    double counters[ORC_C_COUNT];
};

static double sgn_plus(double x) { return x >= 0.0 ? 1.0 : -1.0; } /* reading R5: sign(0) = +1 */

/*
 * Textbook LU with partial pivoting of a b x b row-major matrix, in place (LAPACK getrf
 * semantics: pivot = first index of the largest |.| in the column, reading R4).
 * perm[i] = original row now at position i.  Returns -1 on success, or the column j at
 * which the pivot magnitude was <= thresh (singular / ill-conditioned block).
 */
static int getrf_plain(double *a, int b, int32_t *perm, double thresh) {
    for (int i = 0; i < b; ++i) perm[i] = i;
    for (int j = 0; j < b; ++j) {
        int p = j;
        double amax = fabs(a[j * b + j]);
        for (int i = j + 1; i < b; ++i)
            if (fabs(a[i * b + j]) > amax) { amax = fabs(a[i * b + j]); p = i; }
        if (amax <= thresh) return j;
        if (p != j) {
            for (int k = 0; k < b; ++k) { double t = a[j * b + k]; a[j * b + k] = a[p * b + k]; a[p * b + k] = t; }
            int32_t t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        }
        for (int i = j + 1; i < b; ++i) a[i * b + j] /= a[j * b + j];
        for (int i = j + 1; i < b; ++i)
            for (int k = j + 1; k < b; ++k) a[i * b + k] -= a[i * b + j] * a[j * b + k];
    }
    return -1;
}

/* D = P^{-1} by solving P X = I column by column with the LU factors (Sec. 2.2: the
 * diagonal blocks are factored and inverted). */
static void inverse_from_lu(const double *lu, const int32_t *perm, int b, double *d) {
    double *y = xmalloc((size_t)b * sizeof(double));
    for (int c = 0; c < b; ++c) {
        for (int i = 0; i < b; ++i) y[i] = (perm[i] == c) ? 1.0 : 0.0;
        for (int i = 0; i < b; ++i)
            for (int k = 0; k < i; ++k) y[i] -= lu[i * b + k] * y[k];
        for (int i = b - 1; i >= 0; --i) {
            for (int k = i + 1; k < b; ++k) y[i] -= lu[i * b + k] * y[k];
            y[i] /= lu[i * b + i];
        }
        for (int i = 0; i < b; ++i) d[i * b + c] = y[i];
    }
    free(y);
}

/* Sec. 3.6: d_kj <- d_kj (1 + rho beta_j) + sign(d_kj) tau alpha, beta_j := 1 (reading R5). */
static double perturbed(double d, double ptau, double prho, double alpha) {
    return d * (1.0 + prho) + sgn_plus(d) * ptau * alpha;
}

/*
 * Factor and invert the pivot block P (b x b, row-major, modified in place when
 * perturbed).  Sec. 3.6: an all-zero column j is perturbed at its largest entry, the
 * diagonal entry taking precedence when 2|d_jj| >= |d_kj|; rows likewise.  A pivot
 * breakdown during the LU perturbs the breaking column the same way and restarts.
 * With sym (BILDL) the breaking column is perturbed at its diagonal entry.
 * Returns the number of perturbations, or -1 when singular and perturbation is off
 * (or did not cure the block).
 */
static int factor_pivot_block(double *P, int b, int perturb, double ptau, double prho, double alpha, int sym,
                              double *lu, int32_t *perm, double *dinv) {
    int count = 0;
    if (perturb) {
        for (int j = 0; j < b; ++j) {
            int zero = 1;
            for (int i = 0; i < b; ++i) zero &= (P[i * b + j] == 0.0);
            if (zero) { P[j * b + j] = perturbed(P[j * b + j], ptau, prho, alpha); ++count; }
        }
        for (int i = 0; i < b; ++i) {
            int zero = 1;
            for (int j = 0; j < b; ++j) zero &= (P[i * b + j] == 0.0);
            if (zero) { P[i * b + i] = perturbed(P[i * b + i], ptau, prho, alpha); ++count; }
        }
    }
    for (int attempt = 0; attempt <= 2 * b; ++attempt) {
        double pmax = 0.0;
        for (int e = 0; e < b * b; ++e) pmax = fmax(pmax, fabs(P[e]));
        memcpy(lu, P, (size_t)b * b * sizeof(double));
        int bad = getrf_plain(lu, b, perm, 1e-14 * pmax);
        if (bad < 0) {
            inverse_from_lu(lu, perm, b, dinv);
            return count;
        }
        if (!perturb) return -1;
        int k = 0;
        for (int i = 1; i < b; ++i)
            if (fabs(P[i * b + bad]) > fabs(P[k * b + bad])) k = i;
        if (2.0 * fabs(P[bad * b + bad]) >= fabs(P[k * b + bad])) k = bad;
        if (sym) k = bad; /* symmetric variant: the diagonal entry, so that P stays symmetric (reading R22) */
        P[k * b + bad] = perturbed(P[k * b + bad], ptau, prho, alpha);
        ++count;
    }
    return -1;
}

/* sort helper: slots ordered by their global index */
static const int32_t *g_sort_keys;
static int cmp_slot(const void *a, const void *b) {
    int32_t x = g_sort_keys[*(const int32_t *)a], y = g_sort_keys[*(const int32_t *)b];
    return (x > y) - (x < y);
}

/* sparse accumulator: a dense buffer of b values per touched index */
typedef struct {
    int32_t *slot_of; /* n entries, -1 when untouched */
    int32_t *idx;     /* global index per slot */
    double *buf;      /* nslot x b */
    int64_t nslot, cap;
    int b;
} spa_t;

static int32_t spa_slot(spa_t *s, int32_t i) {
    if (s->slot_of[i] >= 0) return s->slot_of[i];
    if (s->nslot == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 256;
        s->idx = xrealloc(s->idx, (size_t)s->cap * sizeof(int32_t));
        s->buf = xrealloc(s->buf, (size_t)s->cap * (size_t)s->b * sizeof(double));
    }
    int32_t sl = (int32_t)s->nslot++;
    s->slot_of[i] = sl;
    s->idx[sl] = i;
    memset(s->buf + (size_t)sl * s->b, 0, (size_t)s->b * sizeof(double));
    return sl;
}
static void spa_reset(spa_t *s, int b) {
    for (int64_t t = 0; t < s->nslot; ++t) s->slot_of[s->idx[t]] = -1;
    s->nslot = 0;
    if (b != s->b) { s->b = b; s->buf = xrealloc(s->buf, (size_t)(s->cap ? s->cap : 1) * (size_t)b * sizeof(double)); }
}

/* ------------------------------------------------------------ progressive aggregation */

/*
 * Sec. 3.5 merge test.  Block k-1 has p columns, block k has q; L_{k,k-1}, L_{k+1,k-1},
 * L_{k+1,k} have r, s, t stored rows and U_{k-1,k}, U_{k-1,k+1}, U_{k,k+1} have rp, sp, tp
 * stored columns; u (v) counts the rows (columns) of the merged block column of L (row of
 * U) beyond block k.  Before merging mu = p (p + r + s + rp + sp) + q (q + t + tp) values
 * are stored, after it nu = (p + q)(p + q + u + v) (the diagonal block dense).  Merge iff
 * nu <= 1.2 mu or nu <= mu + 2 (p + q); 1.2 mu is compared exactly as 5 nu <= 6 mu.
 */
int32_t orc_agg_rule(int64_t p, int64_t q, int64_t r, int64_t s, int64_t rp, int64_t sp, int64_t t,
                     int64_t tp, int64_t u, int64_t v) {
    const int64_t mu = p * (p + r + s + rp + sp) + q * (q + t + tp);
    const int64_t nu = (p + q) * (p + q + u + v);
    return (5 * nu <= 6 * mu) || (nu <= mu + 2 * (p + q));
}

/* sorted union of two sorted index lists (no duplicates inside either); out may be NULL */
static int64_t sorted_union(const int32_t *a, int64_t na, const int32_t *b, int64_t nb, int32_t *out) {
    int64_t i = 0, j = 0, m = 0;
    while (i < na || j < nb) {
        int32_t x;
        if (j == nb || (i < na && a[i] < b[j])) x = a[i++];
        else if (i == na || b[j] < a[i]) x = b[j++];
        else { x = a[i]; ++i; ++j; }
        if (out) out[m] = x;
        ++m;
    }
    return m;
}

/* position of x in the sorted list a[0..n), or -1 */
static int64_t find_i32(const int32_t *a, int64_t n, int32_t x) {
    int64_t k = lower_bound_i32(a, 0, n, x);
    return (k < n && a[k] == x) ? k : -1;
}

/* the last two producers appended to a later block's list are k-1 and / or k: after the
 * merge only k remains (block k-1 is void) */
static void fix_producers(vec_i32 *list, int32_t k) {
    if (list->n >= 2 && list->a[list->n - 1] == k && list->a[list->n - 2] == k - 1) {
        list->a[list->n - 2] = k;
        list->n -= 1;
    } else if (list->n >= 1 && list->a[list->n - 1] == k - 1) {
        list->a[list->n - 1] = k;
    }
}

/*
 * After block k is finished: test the merge of the (possibly already merged) block k-1
 * with k, Sec. 3.5, and on success rewrite both as one block k of p + q columns and make
 * k-1 void (size 0).  With L21 = L_{k,k-1} (q x p, zero rows where nothing is stored) and
 * U12 = U-breve_{k-1,k} (p x q), the product of the factors is unchanged when
 *   L-hat_{i,:}   = [ L_{i,k-1} - L_{i,k} L21 ,  L_{i,k} ]         for rows i beyond B_k,
 *   U-hat_{:,j}   = [ U_{k-1,j} ; L21 U_{k-1,j} + U_{k,j} ]         for columns j beyond B_k,
 *   P-hat         = [ P_{k-1}  U12 ; L21 P_{k-1}  L21 U12 + P_k ],
 *   D-hat = P-hat^{-1} = [ D_{k-1} + (D_{k-1} U12) D_k L21   -(D_{k-1} U12) D_k ;
 *                          -D_k L21                           D_k ],
 * the rows (columns) of the merged block being the union of both blocks' (the common
 * pattern the paper asks for), absent entries taken as zero.
 */
static void aggregate_step(orc_factor *F, int32_t k, int32_t agg_max, vec_i32 *prodL, vec_i32 *prodU,
                           int32_t *blk_of) {
    const int32_t a0 = F->bstart[k - 1], s0 = F->bstart[k], s1 = F->bstart[k + 1];
    const int64_t p = s0 - a0, q = s1 - s0, w = p + q;
    if (p == 0 || q == 0 || w > agg_max) return;
    const int64_t L0 = F->Lptr[k - 1], L1 = F->Lptr[k], L2 = F->Lptr[k + 1];
    const int64_t U0 = F->Uptr[k - 1], U1 = F->Uptr[k], U2 = F->Uptr[k + 1];
    /* rows of L_{:,k-1} are all >= s0: those inside B_k come first */
    const int64_t Lm = lower_bound_i32(F->Lrow.a, L0, L1, s1), Um = lower_bound_i32(F->Ucol.a, U0, U1, s1);
    const int64_t r = Lm - L0, s = L1 - Lm, t = L2 - L1;
    const int64_t rp = Um - U0, sp = U1 - Um, tp = U2 - U1;
    const int64_t u = sorted_union(F->Lrow.a + Lm, s, F->Lrow.a + L1, t, NULL);
    const int64_t v = sorted_union(F->Ucol.a + Um, sp, F->Ucol.a + U1, tp, NULL);
    if (!orc_agg_rule(p, q, r, s, rp, sp, t, tp, u, v)) return;

    const double *Lv0 = F->Lval.a + F->Lvptr[k - 1], *Lv1 = F->Lval.a + F->Lvptr[k];
    const double *Uv0 = F->Uval.a + F->Uvptr[k - 1], *Uv1 = F->Uval.a + F->Uvptr[k];
    const double *P1 = F->Pblk + F->Dptr[k - 1], *P2 = F->Pblk + F->Dptr[k];
    const double *D1 = F->Dinv + F->Dptr[k - 1], *D2 = F->Dinv + F->Dptr[k];

    double *L21 = xcalloc((size_t)(q * p + 1), sizeof(double));
    double *U12 = xcalloc((size_t)(p * q + 1), sizeof(double));
    for (int64_t e = L0; e < Lm; ++e)
        for (int64_t c = 0; c < p; ++c) L21[(F->Lrow.a[e] - s0) * p + c] = Lv0[(e - L0) * p + c];
    for (int64_t e = U0; e < Um; ++e)
        for (int64_t c = 0; c < p; ++c) U12[c * q + (F->Ucol.a[e] - s0)] = Uv0[(e - U0) * p + c];

    /* merged diagonal block and its inverse */
    double *Ph = xcalloc((size_t)(w * w), sizeof(double));
    double *Dh = xcalloc((size_t)(w * w), sizeof(double));
    double *DU = xcalloc((size_t)(p * q + 1), sizeof(double)); /* D_{k-1} U12 */
    double *DL = xcalloc((size_t)(q * p + 1), sizeof(double)); /* D_k L21 */
    for (int64_t i = 0; i < p; ++i)
        for (int64_t j = 0; j < p; ++j) Ph[i * w + j] = P1[i * p + j];
    for (int64_t i = 0; i < p; ++i)
        for (int64_t j = 0; j < q; ++j) Ph[i * w + p + j] = U12[i * q + j];
    for (int64_t i = 0; i < q; ++i) {
        for (int64_t j = 0; j < p; ++j) {
            double acc = 0.0;
            for (int64_t m = 0; m < p; ++m) acc += L21[i * p + m] * P1[m * p + j];
            Ph[(p + i) * w + j] = acc;
        }
        for (int64_t j = 0; j < q; ++j) {
            double acc = P2[i * q + j];
            for (int64_t m = 0; m < p; ++m) acc += L21[i * p + m] * U12[m * q + j];
            Ph[(p + i) * w + p + j] = acc;
        }
    }
    for (int64_t i = 0; i < p; ++i)
        for (int64_t j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int64_t m = 0; m < p; ++m) acc += D1[i * p + m] * U12[m * q + j];
            DU[i * q + j] = acc;
        }
    for (int64_t i = 0; i < q; ++i)
        for (int64_t j = 0; j < p; ++j) {
            double acc = 0.0;
            for (int64_t m = 0; m < q; ++m) acc += D2[i * q + m] * L21[m * p + j];
            DL[i * p + j] = acc;
        }
    for (int64_t i = 0; i < p; ++i) {
        for (int64_t j = 0; j < p; ++j) {
            double acc = D1[i * p + j];
            for (int64_t m = 0; m < q; ++m) acc += DU[i * q + m] * DL[m * p + j];
            Dh[i * w + j] = acc;
        }
        for (int64_t j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int64_t m = 0; m < q; ++m) acc += DU[i * q + m] * D2[m * q + j];
            Dh[i * w + p + j] = -acc;
        }
    }
    for (int64_t i = 0; i < q; ++i) {
        for (int64_t j = 0; j < p; ++j) Dh[(p + i) * w + j] = -DL[i * p + j];
        for (int64_t j = 0; j < q; ++j) Dh[(p + i) * w + p + j] = D2[i * q + j];
    }

    /* merged rows of L and columns of U-breve */
    int32_t *Rn = xmalloc((size_t)(u + 1) * sizeof(int32_t));
    int32_t *Cn = xmalloc((size_t)(v + 1) * sizeof(int32_t));
    sorted_union(F->Lrow.a + Lm, s, F->Lrow.a + L1, t, Rn);
    sorted_union(F->Ucol.a + Um, sp, F->Ucol.a + U1, tp, Cn);
    double *Lh = xcalloc((size_t)(u * w + 1), sizeof(double));
    double *Uh = xcalloc((size_t)(v * w + 1), sizeof(double));
    for (int64_t e = 0; e < u; ++e) {
        const int64_t ia = find_i32(F->Lrow.a + Lm, s, Rn[e]), ib = find_i32(F->Lrow.a + L1, t, Rn[e]);
        const double *la = ia >= 0 ? Lv0 + (r + ia) * p : NULL, *lb = ib >= 0 ? Lv1 + ib * q : NULL;
        double *out = Lh + e * w;
        for (int64_t j = 0; j < p; ++j) {
            double acc = la ? la[j] : 0.0;
            if (lb)
                for (int64_t m = 0; m < q; ++m) acc -= lb[m] * L21[m * p + j];
            out[j] = acc;
        }
        for (int64_t m = 0; m < q; ++m) out[p + m] = lb ? lb[m] : 0.0;
    }
    for (int64_t e = 0; e < v; ++e) {
        const int64_t ia = find_i32(F->Ucol.a + Um, sp, Cn[e]), ib = find_i32(F->Ucol.a + U1, tp, Cn[e]);
        const double *ua = ia >= 0 ? Uv0 + (rp + ia) * p : NULL, *ub = ib >= 0 ? Uv1 + ib * q : NULL;
        double *out = Uh + e * w;
        for (int64_t j = 0; j < p; ++j) out[j] = ua ? ua[j] : 0.0;
        for (int64_t i = 0; i < q; ++i) {
            double acc = ub ? ub[i] : 0.0;
            if (ua)
                for (int64_t m = 0; m < p; ++m) acc += L21[i * p + m] * ua[m];
            out[p + i] = acc;
        }
    }

    /* producer lists of later blocks: k-1 becomes k (read before the rows are rewritten) */
    int32_t last = -1;
    for (int64_t e = 0; e < u; ++e) {
        int32_t tb = blk_of[Rn[e]];
        if (tb != last) { fix_producers(&prodU[tb], k); last = tb; }
    }
    last = -1;
    for (int64_t e = 0; e < v; ++e) {
        int32_t tb = blk_of[Cn[e]];
        if (tb != last) { fix_producers(&prodL[tb], k); last = tb; }
    }

    /* rewrite the storage: block k-1 void, block k = the merged block */
    F->Lrow.n = L0;
    F->Lval.n = F->Lvptr[k - 1];
    for (int64_t e = 0; e < u; ++e) vi_push(&F->Lrow, Rn[e]);
    vd_reserve(&F->Lval, u * w);
    memcpy(F->Lval.a + F->Lval.n, Lh, (size_t)(u * w) * sizeof(double));
    F->Lval.n += u * w;
    F->Ucol.n = U0;
    F->Uval.n = F->Uvptr[k - 1];
    for (int64_t e = 0; e < v; ++e) vi_push(&F->Ucol, Cn[e]);
    vd_reserve(&F->Uval, v * w);
    memcpy(F->Uval.a + F->Uval.n, Uh, (size_t)(v * w) * sizeof(double));
    F->Uval.n += v * w;
    F->Lptr[k] = L0; F->Lvptr[k] = F->Lvptr[k - 1];
    F->Uptr[k] = U0; F->Uvptr[k] = F->Uvptr[k - 1];
    F->Lptr[k + 1] = F->Lrow.n; F->Lvptr[k + 1] = F->Lval.n;
    F->Uptr[k + 1] = F->Ucol.n; F->Uvptr[k + 1] = F->Uval.n;

    const int64_t d0 = F->Dptr[k - 1];
    if (d0 + w * w > F->dcap) {
        F->dcap = 2 * (d0 + w * w);
        F->Dinv = xrealloc(F->Dinv, (size_t)F->dcap * sizeof(double));
        F->Pblk = xrealloc(F->Pblk, (size_t)F->dcap * sizeof(double));
        F->LUblk = xrealloc(F->LUblk, (size_t)F->dcap * sizeof(double));
    }
    memcpy(F->Dinv + d0, Dh, (size_t)(w * w) * sizeof(double));
    memcpy(F->Pblk + d0, Ph, (size_t)(w * w) * sizeof(double));
    /* the getrf factors of P-hat, for export only (D-hat comes from the identity above) */
    memcpy(F->LUblk + d0, Ph, (size_t)(w * w) * sizeof(double));
    getrf_plain(F->LUblk + d0, (int)w, F->piv + a0, 0.0);
    F->Dptr[k] = d0;
    F->Dptr[k + 1] = d0 + w * w;
    F->bstart[k] = a0;
    for (int32_t i = a0; i < s0; ++i) blk_of[i] = k;
    F->merges += 1;

    free(L21); free(U12); free(Ph); free(Dh); free(DU); free(DL);
    free(Rn); free(Cn); free(Lh); free(Uh);
}

/*
 * Crout-type BILU (Algorithm 1 with blocks, Sec. 2.2).  For K = 0..nb-1 with block
 * B_K = [s0, s1), b = s1 - s0:
 *  1. T_L[i, B_K] = A[i, B_K] for i >= s0 (pivot rows included), T_U[B_K, j] = A[B_K, j]
 *     for j >= s1 (load the sparse columns / rows of A into the block buffers, Sec. 2.2).
 *  2. for every earlier block J (increasing J, reading R7) with kept L rows R_J and kept
 *     U columns C_J:  T_L[i, c] -= L_J(i,:) U_J(:,c) for i in R_J, i >= s0, c in C_J n B_K,
 *     and T_U[r, j] -= L_J(r,:) U_J(:,j) for r in R_J n B_K, j in C_J, j >= s1
 *     (Algorithm 1's two inner loops; gather / GEMM / scatter of Sec. 2.2).
 *  3. P_K = T_L[B_K, B_K]: LU with pivoting inside the block, perturbed if singular
 *     (Sec. 3.6), D_K = P_K^{-1}.
 *  4. l_i = T_L[i, B_K] D_K for candidate rows i >= s1; keep iff ||l_i||_2 > tau.
 *  5. u^_j = D_K T_U[B_K, j] for candidate cols j >= s1; keep iff ||u^_j||_2 > tau; store
 *     the column T_U[B_K, j] unnormalised (readings R1-R3).
 */
static int32_t crout_factor(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                            int32_t nb, const int32_t *bstart, double droptol, int32_t perturb,
                            double pert_tau, double pert_rho, int32_t agg_max, int sym, orc_factor **out);

int32_t orc_bilu_factor(int64_t n, const int64_t *rowptr, const int32_t *colind,
                        const double *val, int32_t nb, const int32_t *bstart, double droptol,
                        int32_t perturb, double pert_tau, double pert_rho, orc_factor **out) {
    return crout_factor(n, rowptr, colind, val, nb, bstart, droptol, perturb, pert_tau, pert_rho, 0, 0, out);
}

int32_t orc_bilu_factor_agg(int64_t n, const int64_t *rowptr, const int32_t *colind,
                            const double *val, int32_t nb, const int32_t *bstart, double droptol,
                            int32_t perturb, double pert_tau, double pert_rho, int32_t agg_max,
                            orc_factor **out) {
    return crout_factor(n, rowptr, colind, val, nb, bstart, droptol, perturb, pert_tau, pert_rho, agg_max, 0, out);
}

/*
 * BILDL, the symmetric variant (incomplete block L D L^T of a symmetric A, Sec. 4.2): the
 * same Crout loop on the lower triangle only.  For symmetric A the row block T_U[B_K, :]
 * of step 1-2 is the transpose of the column block T_L[:, B_K], so step 2b and step 5 are
 * not computed; instead
 *  3'. the pivot block is the lower triangle of T_L[B_K, B_K] mirrored (symmetric by
 *      construction), factored as in step 3 with perturbations on the diagonal only, and
 *      D_K = (X + X^T) / 2 for the computed inverse X (symmetric to the last bit);
 *  4'. a kept row l_i = t_i D_K is stored in L and its unnormalised t_i, as column i, in
 *      U-breve (D_K t_i^T = l_i^T, so the column's drop test is the row's).
 * The preconditioner L U-breve = L P L^T is then symmetric (readings R22, R23).
 */
int32_t orc_bildl_factor(int64_t n, const int64_t *rowptr, const int32_t *colind,
                         const double *val, int32_t nb, const int32_t *bstart, double droptol,
                         int32_t perturb, double pert_tau, double pert_rho, orc_factor **out) {
    if (n < 0 || !rowptr) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) /* A must equal A^T, entry by entry */
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (colind[e] < 0 || colind[e] >= n || entry(rowptr, colind, val, colind[e], (int32_t)i) != val[e])
                return ORC_ERR_ARG;
    return crout_factor(n, rowptr, colind, val, nb, bstart, droptol, perturb, pert_tau, pert_rho, 0, 1, out);
}

static int32_t crout_factor(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                            int32_t nb, const int32_t *bstart, double droptol, int32_t perturb,
                            double pert_tau, double pert_rho, int32_t agg_max, int sym, orc_factor **out) {
    if (n < 0 || nb < 0 || droptol < 0 || agg_max < 0 || !out) return ORC_ERR_ARG;
    if (bstart[0] != 0 || bstart[nb] != n) return ORC_ERR_ARG;
    for (int32_t K = 0; K < nb; ++K)
        if (bstart[K + 1] <= bstart[K]) return ORC_ERR_ARG;

    orc_factor *F = xcalloc(1, sizeof(orc_factor));
    F->n = n; F->nb = nb;
    F->bstart = xmalloc((size_t)(nb + 1) * sizeof(int32_t));
    memcpy(F->bstart, bstart, (size_t)(nb + 1) * sizeof(int32_t));
    F->Lptr = xcalloc((size_t)nb + 1, sizeof(int64_t));
    F->Lvptr = xcalloc((size_t)nb + 1, sizeof(int64_t));
    F->Uptr = xcalloc((size_t)nb + 1, sizeof(int64_t));
    F->Uvptr = xcalloc((size_t)nb + 1, sizeof(int64_t));
    F->Dptr = xcalloc((size_t)nb + 1, sizeof(int64_t));
    /* D blocks are laid out in block order as the blocks are factored (a merge rewrites
     * the last two); the initial capacity is that of the unmerged partition */
    for (int32_t K = 0; K < nb; ++K) {
        int64_t b = bstart[K + 1] - bstart[K];
        F->dcap += b * b;
    }
    F->Dinv = xcalloc((size_t)F->dcap + 1, sizeof(double));
    F->Pblk = xcalloc((size_t)F->dcap + 1, sizeof(double));
    F->LUblk = xcalloc((size_t)F->dcap + 1, sizeof(double));
    F->piv = xcalloc((size_t)n, sizeof(int32_t));

    csc_t csc = csr_to_csc(n, rowptr, colind, val);
    double alpha = 0.0; /* Sec. 3.6: alpha = max |a_ij| */
    for (int64_t e = 0; e < rowptr[n]; ++e) alpha = fmax(alpha, fabs(val[e]));

    /* producer lists (the role of L_head/L_list and U_head/U_list, Sec. 2.1):
     * prodL[K] = blocks J whose kept U columns hit B_K, prodU[K] = blocks J whose
     * kept L rows hit B_K; appended when J is finished, hence increasing in J. */
    vec_i32 *prodL = xcalloc((size_t)nb + 1, sizeof(vec_i32));
    vec_i32 *prodU = xcalloc((size_t)nb + 1, sizeof(vec_i32));
    int32_t *blk_of = xmalloc((size_t)n * sizeof(int32_t) + 1);
    for (int32_t K = 0; K < nb; ++K)
        for (int32_t i = bstart[K]; i < bstart[K + 1]; ++i) blk_of[i] = K;

    spa_t TL = {0}, TU = {0};
    TL.slot_of = xmalloc((size_t)n * sizeof(int32_t) + 1);
    TU.slot_of = xmalloc((size_t)n * sizeof(int32_t) + 1);
    for (int64_t i = 0; i < n; ++i) { TL.slot_of[i] = -1; TU.slot_of[i] = -1; }
    TL.b = TU.b = 1;

    int32_t status = ORC_OK;
    int32_t *order = NULL;
    int64_t order_cap = 0;
    double *P = NULL, *ell = NULL;

    for (int32_t K = 0; K < nb && status >= 0; ++K) {
        const int32_t s0 = bstart[K], s1 = bstart[K + 1];
        const int b = s1 - s0;
        spa_reset(&TL, b);
        spa_reset(&TU, b);

        /* step 1: load A */
        for (int32_t r = s0; r < s1; ++r) spa_slot(&TL, r); /* dense diagonal block */
        for (int32_t c = s0; c < s1; ++c)
            for (int64_t e = csc.colptr[c]; e < csc.colptr[c + 1]; ++e) {
                int32_t i = csc.rowind[e];
                if (i < s0) continue;
                int32_t sl = spa_slot(&TL, i);
                TL.buf[(size_t)sl * b + (c - s0)] = csc.val[e];
            }
        for (int32_t r = s0; r < s1 && !sym; ++r)
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
                int32_t j = colind[e];
                if (j < s1) continue;
                int32_t sl = spa_slot(&TU, j);
                TU.buf[(size_t)sl * b + (r - s0)] = val[e];
            }

        /* step 2a: L side, J with kept U columns in B_K */
        for (int64_t t = 0; t < prodL[K].n; ++t) {
            int32_t J = prodL[K].a[t];
            int bJ = F->bstart[J + 1] - F->bstart[J]; /* a merged producer spans its void predecessor */
            int64_t qs = lower_bound_i32(F->Ucol.a, F->Uptr[J], F->Uptr[J + 1], s0);
            int64_t qe = lower_bound_i32(F->Ucol.a, qs, F->Uptr[J + 1], s1);
            int64_t ps = lower_bound_i32(F->Lrow.a, F->Lptr[J], F->Lptr[J + 1], s0);
            int64_t pe = F->Lptr[J + 1];
            if (qs == qe) continue;
            F->counters[ORC_C_NPAIRS_L] += 1;
            F->counters[ORC_C_FLOP_UPD_L] += 2.0 * (double)(pe - ps) * (double)(qe - qs) * bJ;
            F->counters[ORC_C_PANEL_READ_BYTES] += 8.0 * ((double)(pe - ps) + (double)(qe - qs)) * bJ;
            for (int64_t p = ps; p < pe; ++p) {
                int32_t sl = spa_slot(&TL, F->Lrow.a[p]);
                const double *lrow = F->Lval.a + F->Lvptr[J] + (p - F->Lptr[J]) * bJ;
                for (int64_t q = qs; q < qe; ++q) {
                    const double *ucol = F->Uval.a + F->Uvptr[J] + (q - F->Uptr[J]) * bJ;
                    double sum = 0.0;
                    for (int tt = 0; tt < bJ; ++tt) sum += lrow[tt] * ucol[tt];
                    TL.buf[(size_t)sl * b + (F->Ucol.a[q] - s0)] -= sum;
                }
            }
        }
        /* step 2b: U side, J with kept L rows in B_K (BILDL: the transpose of step 2a) */
        for (int64_t t = 0; t < prodU[K].n && !sym; ++t) {
            int32_t J = prodU[K].a[t];
            int bJ = F->bstart[J + 1] - F->bstart[J];
            int64_t ps = lower_bound_i32(F->Lrow.a, F->Lptr[J], F->Lptr[J + 1], s0);
            int64_t pe = lower_bound_i32(F->Lrow.a, ps, F->Lptr[J + 1], s1);
            int64_t qs = lower_bound_i32(F->Ucol.a, F->Uptr[J], F->Uptr[J + 1], s1);
            int64_t qe = F->Uptr[J + 1];
            if (ps == pe) continue;
            F->counters[ORC_C_NPAIRS_U] += 1;
            F->counters[ORC_C_FLOP_UPD_U] += 2.0 * (double)(pe - ps) * (double)(qe - qs) * bJ;
            F->counters[ORC_C_PANEL_READ_BYTES] += 8.0 * ((double)(pe - ps) + (double)(qe - qs)) * bJ;
            for (int64_t q = qs; q < qe; ++q) {
                int32_t sl = spa_slot(&TU, F->Ucol.a[q]);
                const double *ucol = F->Uval.a + F->Uvptr[J] + (q - F->Uptr[J]) * bJ;
                for (int64_t p = ps; p < pe; ++p) {
                    const double *lrow = F->Lval.a + F->Lvptr[J] + (p - F->Lptr[J]) * bJ;
                    double sum = 0.0;
                    for (int tt = 0; tt < bJ; ++tt) sum += lrow[tt] * ucol[tt];
                    TU.buf[(size_t)sl * b + (F->Lrow.a[p] - s0)] -= sum;
                }
            }
        }

        /* step 3: pivot block */
        F->Dptr[K + 1] = F->Dptr[K] + (int64_t)b * b;
        if (F->Dptr[K + 1] > F->dcap) { /* merges made the D blocks larger than the partition's */
            F->dcap = 2 * F->Dptr[K + 1];
            F->Dinv = xrealloc(F->Dinv, (size_t)F->dcap * sizeof(double));
            F->Pblk = xrealloc(F->Pblk, (size_t)F->dcap * sizeof(double));
            F->LUblk = xrealloc(F->LUblk, (size_t)F->dcap * sizeof(double));
        }
        P = xrealloc(P, (size_t)b * b * sizeof(double));
        for (int r = 0; r < b; ++r)
            for (int c = 0; c < b; ++c) P[r * b + c] = TL.buf[(size_t)r * b + c]; /* slots 0..b-1 = rows s0.. */
        if (sym) /* BILDL: the lower triangle defines the symmetric pivot block */
            for (int r = 0; r < b; ++r)
                for (int c = r + 1; c < b; ++c) P[r * b + c] = P[c * b + r];
        double *D = F->Dinv + F->Dptr[K];
        int np = factor_pivot_block(P, b, perturb, pert_tau, pert_rho, alpha, sym,
                                    F->LUblk + F->Dptr[K], F->piv + s0, D);
        if (np >= 0 && sym)
            for (int r = 0; r < b; ++r)
                for (int c = r + 1; c < b; ++c) {
                    double v = (D[r * b + c] + D[c * b + r]) * 0.5;
                    D[r * b + c] = v;
                    D[c * b + r] = v;
                }
        memcpy(F->Pblk + F->Dptr[K], P, (size_t)b * b * sizeof(double));
        if (np < 0) { status = ORC_ERR_SINGULAR; break; }
        if (np > 0) { F->counters[ORC_C_NPERTURB] += np; }
        F->counters[ORC_C_FLOP_GETRF] += 2.0 / 3.0 * b * (double)b * b;
        F->counters[ORC_C_FLOP_INV] += 4.0 / 3.0 * b * (double)b * b;

        /* step 4: L rows, in increasing row order */
        int64_t ncand = TL.nslot - b;
        if (TL.nslot > order_cap) { order_cap = TL.nslot + TU.nslot + 16; order = xrealloc(order, (size_t)order_cap * sizeof(int32_t)); }
        if (TU.nslot > order_cap) { order_cap = TL.nslot + TU.nslot + 16; order = xrealloc(order, (size_t)order_cap * sizeof(int32_t)); }
        ell = xrealloc(ell, (size_t)b * sizeof(double));
        for (int64_t t = 0; t < ncand; ++t) order[t] = (int32_t)(b + t);
        g_sort_keys = TL.idx;
        qsort(order, (size_t)ncand, sizeof(int32_t), cmp_slot);
        F->counters[ORC_C_CAND_ROWS] += (double)ncand;
        F->counters[ORC_C_FLOP_SCALE] += 2.0 * b * (double)b * ncand;
        F->counters[ORC_C_FLOP_NORM] += 2.0 * b * (double)ncand;
        for (int64_t t = 0; t < ncand; ++t) {
            const double *trow = TL.buf + (size_t)order[t] * b;
            double nrm2 = 0.0;
            for (int c = 0; c < b; ++c) {
                double s = 0.0;
                for (int k = 0; k < b; ++k) s += trow[k] * D[k * b + c];
                ell[c] = s;
                nrm2 += s * s;
            }
            if (sqrt(nrm2) > droptol) {
                vi_push(&F->Lrow, TL.idx[order[t]]);
                vd_reserve(&F->Lval, b);
                memcpy(F->Lval.a + F->Lval.n, ell, (size_t)b * sizeof(double));
                F->Lval.n += b;
                if (sym) { /* BILDL: column i of U-breve is t_i^T */
                    vi_push(&F->Ucol, TL.idx[order[t]]);
                    vd_reserve(&F->Uval, b);
                    memcpy(F->Uval.a + F->Uval.n, trow, (size_t)b * sizeof(double));
                    F->Uval.n += b;
                }
            }
        }
        /* step 5: U columns, in increasing column order (BILDL: taken in step 4) */
        int64_t ncc = sym ? 0 : TU.nslot;
        for (int64_t t = 0; t < ncc; ++t) order[t] = (int32_t)t;
        g_sort_keys = TU.idx;
        qsort(order, (size_t)ncc, sizeof(int32_t), cmp_slot);
        F->counters[ORC_C_CAND_COLS] += (double)ncc;
        F->counters[ORC_C_FLOP_SCALE] += 2.0 * b * (double)b * ncc;
        F->counters[ORC_C_FLOP_NORM] += 2.0 * b * (double)ncc;
        for (int64_t t = 0; t < ncc; ++t) {
            const double *tcol = TU.buf + (size_t)order[t] * b;
            double nrm2 = 0.0;
            for (int r = 0; r < b; ++r) {
                double s = 0.0;
                for (int k = 0; k < b; ++k) s += D[r * b + k] * tcol[k];
                nrm2 += s * s;
            }
            if (sqrt(nrm2) > droptol) {
                vi_push(&F->Ucol, TU.idx[order[t]]);
                vd_reserve(&F->Uval, b);
                memcpy(F->Uval.a + F->Uval.n, tcol, (size_t)b * sizeof(double));
                F->Uval.n += b;
            }
        }
        F->Lptr[K + 1] = F->Lrow.n;
        F->Lvptr[K + 1] = F->Lval.n;
        F->Uptr[K + 1] = F->Ucol.n;
        F->Uvptr[K + 1] = F->Uval.n;

        /* producer lists of later blocks */
        int32_t last = -1;
        for (int64_t p = F->Lptr[K]; p < F->Lptr[K + 1]; ++p) {
            int32_t t = blk_of[F->Lrow.a[p]];
            if (t != last) { vi_push(&prodU[t], K); last = t; }
        }
        last = -1;
        for (int64_t q = F->Uptr[K]; q < F->Uptr[K + 1]; ++q) {
            int32_t t = blk_of[F->Ucol.a[q]];
            if (t != last) { vi_push(&prodL[t], K); last = t; }
        }

        /* Sec. 3.5: merge the finished blocks K-1 and K when the memory grows mildly */
        if (agg_max > 0 && K > 0) aggregate_step(F, K, agg_max, prodL, prodU, blk_of);
    }

    if (status >= 0 && F->counters[ORC_C_NPERTURB] > 0) status = ORC_PERTURBED;
    free(order); free(P); free(ell);
    free(TL.slot_of); free(TL.idx); free(TL.buf);
    free(TU.slot_of); free(TU.idx); free(TU.buf);
    for (int32_t K = 0; K <= nb; ++K) { free(prodL[K].a); free(prodU[K].a); }
    free(prodL); free(prodU); free(blk_of);
    csc_free(&csc);
    if (status < 0) { orc_factor_free(F); *out = NULL; return status; }
    *out = F;
    return status;
}

void orc_factor_bstart(const orc_factor *F, int32_t *bstart) {
    memcpy(bstart, F->bstart, (size_t)(F->nb + 1) * sizeof(int32_t));
}

void orc_factor_sizes(const orc_factor *F, int64_t sizes[8]) {
    memset(sizes, 0, 8 * sizeof(int64_t));
    sizes[7] = F->merges;
    sizes[0] = F->Lrow.n;
    sizes[1] = F->Ucol.n;
    sizes[2] = F->Lval.n;
    sizes[3] = F->Uval.n;
    sizes[4] = F->Dptr[F->nb];
    sizes[5] = F->nb;
    sizes[6] = (int64_t)F->counters[ORC_C_NPERTURB];
}

void orc_factor_export(const orc_factor *F, int64_t *Lptr, int32_t *Lrow, double *Lval,
                       int64_t *Uptr, int32_t *Ucol, double *Uval, double *Dinv,
                       double *Pblk, double *LUblk, int32_t *piv) {
    int32_t nb = F->nb;
    if (Lptr) memcpy(Lptr, F->Lptr, (size_t)(nb + 1) * sizeof(int64_t));
    if (Lrow) memcpy(Lrow, F->Lrow.a, (size_t)F->Lrow.n * sizeof(int32_t));
    if (Lval) memcpy(Lval, F->Lval.a, (size_t)F->Lval.n * sizeof(double));
    if (Uptr) memcpy(Uptr, F->Uptr, (size_t)(nb + 1) * sizeof(int64_t));
    if (Ucol) memcpy(Ucol, F->Ucol.a, (size_t)F->Ucol.n * sizeof(int32_t));
    if (Uval) memcpy(Uval, F->Uval.a, (size_t)F->Uval.n * sizeof(double));
    if (Dinv) memcpy(Dinv, F->Dinv, (size_t)F->Dptr[nb] * sizeof(double));
    if (Pblk) memcpy(Pblk, F->Pblk, (size_t)F->Dptr[nb] * sizeof(double));
    if (LUblk) memcpy(LUblk, F->LUblk, (size_t)F->Dptr[nb] * sizeof(double));
    if (piv) memcpy(piv, F->piv, (size_t)F->n * sizeof(int32_t));
}

void orc_factor_counters(const orc_factor *F, double c[ORC_C_COUNT]) {
    memcpy(c, F->counters, ORC_C_COUNT * sizeof(double));
}

void orc_factor_free(orc_factor *F) {
    if (!F) return;
    free(F->bstart); free(F->Lptr); free(F->Lvptr); free(F->Uptr); free(F->Uvptr); free(F->Dptr);
    free(F->Lrow.a); free(F->Ucol.a); free(F->Lval.a); free(F->Uval.a);
    free(F->Dinv); free(F->Pblk); free(F->LUblk); free(F->piv);
    free(F);
}

/* ------------------------------------------------------------ application */

/*
 * z = M^{-1} r with M = L D^{-1} U = L U-breve (Sec. 2.2):
 *   forward:  y_K = r_K - sum_{J<K} L_J(B_K rows, :) y_J          (unit block lower L)
 *   backward: z_K = D_K ( y_K - U-breve_K(:, C_K) z(C_K) ), K = nb-1 .. 0.
 */
void orc_bilu_apply(const orc_factor *F, const double *r, double *z) {
    int64_t n = F->n;
    double *y = xmalloc((size_t)n * sizeof(double) + 8);
    memcpy(y, r, (size_t)n * sizeof(double));
    for (int32_t J = 0; J < F->nb; ++J) {
        int bJ = F->bstart[J + 1] - F->bstart[J];
        const double *yJ = y + F->bstart[J];
        for (int64_t p = F->Lptr[J]; p < F->Lptr[J + 1]; ++p) {
            const double *lrow = F->Lval.a + F->Lvptr[J] + (p - F->Lptr[J]) * bJ;
            double s = 0.0;
            for (int t = 0; t < bJ; ++t) s += lrow[t] * yJ[t];
            y[F->Lrow.a[p]] -= s;
        }
    }
    int tcap = 64;
    double *t = xmalloc((size_t)tcap * sizeof(double));
    for (int32_t K = F->nb - 1; K >= 0; --K) {
        int32_t s0 = F->bstart[K];
        int b = F->bstart[K + 1] - s0;
        if (b > tcap) { tcap = b; t = xrealloc(t, (size_t)b * sizeof(double)); }
        for (int i = 0; i < b; ++i) t[i] = y[s0 + i];
        for (int64_t q = F->Uptr[K]; q < F->Uptr[K + 1]; ++q) {
            const double *ucol = F->Uval.a + F->Uvptr[K] + (q - F->Uptr[K]) * b;
            double zj = z[F->Ucol.a[q]];
            for (int i = 0; i < b; ++i) t[i] -= ucol[i] * zj;
        }
        const double *D = F->Dinv + F->Dptr[K];
        for (int i = 0; i < b; ++i) {
            double s = 0.0;
            for (int k = 0; k < b; ++k) s += D[i * b + k] * t[k];
            z[s0 + i] = s;
        }
    }
    free(t);
    free(y);
}

/* ------------------------------------------------------------ GMRES */

void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
              const double *x, double *y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[colind[e]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void precond(const orc_factor *M, int64_t n, const double *v, double *out) {
    if (M) orc_bilu_apply(M, v, out);
    else memcpy(out, v, (size_t)n * sizeof(double));
}

/*
 * Restarted GMRES(m) (Saad and Schultz), right preconditioned: A M^{-1} u = b,
 * x = x0 + M^{-1} V y.  Arnoldi by modified Gram-Schmidt, least-squares problem by
 * Givens rotations.  A cycle stops when |g_{j+1}| <= tol ||b||; the true residual
 * ||b - A x|| / ||b|| then decides whether to stop or restart (reading R8).
 * Iterations count inner Arnoldi steps.
 */
int32_t orc_gmres(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                  const orc_factor *M, const double *b, double *x, double tol, int32_t restart,
                  int32_t maxit, int32_t *iters, double *relres_true, double *hist) {
    int m = restart;
    double *V = xmalloc((size_t)(m + 1) * (size_t)n * sizeof(double) + 8);
    double *H = xcalloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = xmalloc((size_t)m * sizeof(double)), *sn = xmalloc((size_t)m * sizeof(double));
    double *g = xmalloc((size_t)(m + 1) * sizeof(double)), *y = xmalloc((size_t)m * sizeof(double));
    double *w = xmalloc((size_t)n * sizeof(double) + 8), *zt = xmalloc((size_t)n * sizeof(double) + 8);
    double *r = xmalloc((size_t)n * sizeof(double) + 8);
    int32_t its = 0, status = ORC_NOT_CONVERGED;
    double bnorm = sqrt(dot(n, b, b));
    double rel = 0.0;
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        *iters = 0; *relres_true = 0.0; status = ORC_OK;
        goto done;
    }
    orc_spmv(n, rowptr, colind, val, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double beta = sqrt(dot(n, r, r));
    rel = beta / bnorm;
    if (hist) hist[0] = rel;
    while (rel > tol && its < maxit) {
        for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        memset(g, 0, (size_t)(m + 1) * sizeof(double));
        g[0] = beta;
        int j, jdone = 0;
        for (j = 0; j < m && its < maxit; ++j) {
            double *vj = V + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            precond(M, n, vj, zt);
            orc_spmv(n, rowptr, colind, val, zt, w);
            for (int i = 0; i <= j; ++i) {
                double h = dot(n, w, V + (size_t)i * n);
                H[i * m + j] = h;
                for (int64_t e = 0; e < n; ++e) w[e] -= h * V[(size_t)i * n + e];
            }
            double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (int64_t e = 0; e < n; ++e) vn[e] = w[e] / hn;
            for (int i = 0; i < j; ++i) {
                double a = H[i * m + j], c2 = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c2;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c2;
            }
            double a = H[j * m + j], c2 = H[(j + 1) * m + j];
            double den = hypot(a, c2);
            cs[j] = (den == 0.0) ? 1.0 : a / den;
            sn[j] = (den == 0.0) ? 0.0 : c2 / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            jdone = j + 1;
            if (hist) hist[its] = fabs(g[j + 1]) / bnorm;
            if (fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
        }
        /* y = H(0:jdone,0:jdone)^{-1} g, x += M^{-1} V y */
        for (int i = jdone - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < jdone; ++k) s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        memset(w, 0, (size_t)n * sizeof(double));
        for (int k = 0; k < jdone; ++k)
            for (int64_t e = 0; e < n; ++e) w[e] += y[k] * V[(size_t)k * n + e];
        precond(M, n, w, zt);
        for (int64_t e = 0; e < n; ++e) x[e] += zt[e];
        orc_spmv(n, rowptr, colind, val, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        beta = sqrt(dot(n, r, r));
        rel = beta / bnorm;
    }
    *iters = its;
    *relres_true = rel;
    status = (rel <= tol) ? ORC_OK : ORC_NOT_CONVERGED;
done:
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(w); free(zt); free(r);
    return status;
}

/* ------------------------------------------------------------ SQMR */

/* Normwise backward error of x (Rigal and Gaches, with the data A and b perturbed):
 * ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)  (reading R24). */
static double backward_error(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                             double anorm, const double *b, const double *x, double *work) {
    orc_spmv(n, rowptr, colind, val, x, work);
    double rmax = 0.0, xmax = 0.0, bmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        rmax = fmax(rmax, fabs(b[i] - work[i]));
        xmax = fmax(xmax, fabs(x[i]));
        bmax = fmax(bmax, fabs(b[i]));
    }
    double den = anorm * xmax + bmax;
    return den > 0.0 ? rmax / den : 0.0;
}

/*
 * Simplified QMR (Freund and Nachtigal; Freund and Jarre) for a symmetric, possibly
 * indefinite A with a symmetric preconditioner M (the solver paired with BILDL, Sec. 4.2).
 * No look-ahead.  With the BCG residual r, direction q, rho = r^T M^{-1} r:
 *   sigma = q^T A q,  alpha = rho / sigma,  r <- r - alpha A q,
 *   theta' = ||r|| / tau,  c = 1 / sqrt(1 + theta'^2),  tau <- tau theta' c,
 *   d <- c^2 theta^2 d + c^2 alpha q,  x <- x + d,
 *   u = M^{-1} r,  rho' = r^T u,  q <- u + (rho' / rho) q,
 * starting from r = b - A x0, tau = ||r||, q = M^{-1} r, theta = 0, d = 0.  Stops when the
 * backward error of x (backward_error above) is <= tol, after maxit steps, or when sigma or
 * rho vanishes (a breakdown).  iters counts steps (one product with A and one with M^{-1}
 * each); hist[k] is the backward error after step k (hist[0]: of x0).
 */
int32_t orc_sqmr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                 const orc_factor *M, const double *b, double *x, double tol, int32_t maxit,
                 int32_t *iters, double *berr, double *hist) {
    double *r = xmalloc((size_t)n * sizeof(double) + 8), *t = xmalloc((size_t)n * sizeof(double) + 8);
    double *q = xmalloc((size_t)n * sizeof(double) + 8), *d = xcalloc((size_t)n + 1, sizeof(double));
    double *u = xmalloc((size_t)n * sizeof(double) + 8), *w = xmalloc((size_t)n * sizeof(double) + 8);
    int32_t its = 0, status = ORC_NOT_CONVERGED;
    double anorm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += fabs(val[e]);
        anorm = fmax(anorm, s);
    }
    double eta = backward_error(n, rowptr, colind, val, anorm, b, x, w);
    if (hist) hist[0] = eta;
    if (eta <= tol) { status = ORC_OK; goto done; }
    orc_spmv(n, rowptr, colind, val, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    double tau = sqrt(dot(n, r, r)), theta = 0.0;
    precond(M, n, r, q);
    double rho = dot(n, r, q);
    while (its < maxit) {
        orc_spmv(n, rowptr, colind, val, q, t);
        double sigma = dot(n, q, t);
        if (sigma == 0.0) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / sigma;
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * t[i];
        double theta1 = sqrt(dot(n, r, r)) / tau;
        double c = 1.0 / sqrt(1.0 + theta1 * theta1);
        tau = tau * theta1 * c;
        for (int64_t i = 0; i < n; ++i) {
            d[i] = c * c * theta * theta * d[i] + c * c * alpha * q[i];
            x[i] += d[i];
        }
        ++its;
        eta = backward_error(n, rowptr, colind, val, anorm, b, x, w);
        if (hist) hist[its] = eta;
        if (eta <= tol) { status = ORC_OK; break; }
        if (rho == 0.0) { status = ORC_BREAKDOWN; break; }
        precond(M, n, r, u);
        double rho1 = dot(n, r, u);
        double beta = rho1 / rho;
        for (int64_t i = 0; i < n; ++i) q[i] = u[i] + beta * q[i];
        rho = rho1;
        theta = theta1;
    }
done:
    *iters = its;
    *berr = eta;
    free(r); free(t); free(q); free(d); free(u); free(w);
    return status;
}
