// Analysis (host side): validation and copy of A, its CSC copy, the block partition, and the
// preprocessing of Sec. 3.
//
// Sec. 2.1: the Crout ILU needs A by rows and by columns, so a CSC copy is built once.
// Sec. 3.4: the block partition is fixed-size, the simplified ILU(1,tau) guess (column by
//           column or over given groups), or the caller's.
// Sec. 3.1: maximum weight matching with scaling (mwm_host) and the scale-and-permute step.
// Sec. 3.2: cosine-based blocking (cosine_blocking_host) and symmetric permutation.
// Sec. 3.3: block nested dissection (nd_order_host) and the block elimination tree.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>
#include <limits>
#include <string>
#include <utility>

#include "bilu_internal.h"

namespace {

struct HostCSR {
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    std::vector<double> val;
};

// Column-major copy: for column j, rows ascending.
void build_csc(const HostCSR &A, std::vector<int32_t> &colptr, std::vector<int32_t> &rowind,
               std::vector<double> &cval) {
    const int64_t n = A.n, nnz = A.rowptr[n];
    colptr.assign(n + 1, 0);
    rowind.resize(nnz);
    cval.resize(nnz);
    for (int64_t e = 0; e < nnz; ++e) colptr[A.colind[e] + 1]++;
    for (int64_t j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
    std::vector<int32_t> next(colptr.begin(), colptr.end() - 1);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
            int32_t pos = next[A.colind[e]]++;
            rowind[pos] = (int32_t)i;
            cval[pos] = A.val[e];
        }
}

double diag_of(const int64_t *ptr, const int32_t *ind, const double *v, int64_t i) {
    const int32_t *b = ind + ptr[i], *e = ind + ptr[i + 1];
    const int32_t *p = std::lower_bound(b, e, (int32_t)i);
    return (p != e && *p == i) ? v[p - ind] : 0.0;
}

// The estimated pattern of column k of L (rows > k) or of row k of U (columns > k) under
// the simplified ILU(1,tau) of Sec. 3.4: the original entries with |a| >= tau |a_kk|, and
// the fill a_ik = -a_ij a_jk / a_jj (j < k < i, all three original) when
// |a_ij a_jk| >= tau |a_jj a_kk|.  `major` is the compressed orientation that lists the
// entries of column k (CSC for L, CSR for U); the fill walks the same orientation at j.
std::vector<int32_t> ilu1t_pattern(int64_t k, const int64_t *ptr, const int32_t *ind,
                                   const double *v, const std::vector<double> &diag, double tau) {
    std::vector<int32_t> out;
    const double akk = diag[k];
    for (int64_t e = ptr[k]; e < ptr[k + 1]; ++e) {
        const int32_t i = ind[e];
        if (i > k && std::fabs(v[e]) >= tau * std::fabs(akk)) out.push_back(i);
    }
    for (int64_t e = ptr[k]; e < ptr[k + 1]; ++e) {
        const int32_t j = ind[e];
        if (j >= k) break;  // sorted: the entries above the diagonal come first
        const double ajk = v[e], ajj = diag[j];
        for (int64_t f = ptr[j]; f < ptr[j + 1]; ++f) {
            const int32_t i = ind[f];
            if (i > k && std::fabs(v[f] * ajk) >= tau * std::fabs(ajj * akk)) out.push_back(i);
        }
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}

// Number of entries of the sorted union of a and b that are > bound.
int64_t union_count_above(const std::vector<int32_t> &a, const std::vector<int32_t> &b, int64_t bound) {
    auto ia = std::upper_bound(a.begin(), a.end(), (int32_t)bound);
    auto ib = std::upper_bound(b.begin(), b.end(), (int32_t)bound);
    int64_t cnt = 0;
    while (ia != a.end() || ib != b.end()) {
        if (ib == b.end() || (ia != a.end() && *ia < *ib)) { ++ia; }
        else if (ia == a.end() || *ib < *ia) { ++ib; }
        else { ++ia; ++ib; }
        ++cnt;
    }
    return cnt;
}

std::vector<int32_t> sorted_union(const std::vector<int32_t> &a, const std::vector<int32_t> &b) {
    std::vector<int32_t> out;
    out.reserve(a.size() + b.size());
    std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
    return out;
}

// Sec. 3.4 growth rule over whole groups of columns (groups of one column: the rule column by
// column): a block [k, k+l) with r rows at or after its end in L and s columns at or after its
// end in U stores f = (r + s + l) l entries; its scalar count is the sum over its columns of
// |I~| + |J~| + 1.  The next group [e, e+g) joins while f_{l+g} <= 4/3 s_{l+g} or
// f_{l+g} <= s_{l+g} + 4(l+g), and l+g <= max_block.  Indices inside the block are not counted
// in r, s.  `groups` holds the group starts and n at the end.
std::vector<int32_t> partition_ilu1t(const HostCSR &A, const std::vector<int32_t> &colptr,
                                     const std::vector<int32_t> &rowind, const std::vector<double> &cval,
                                     double tau, int max_block, const std::vector<int32_t> &groups) {
    const int64_t n = A.n;
    std::vector<double> diag(n);
    for (int64_t i = 0; i < n; ++i) diag[i] = diag_of(A.rowptr.data(), A.colind.data(), A.val.data(), i);
    std::vector<int64_t> cp(colptr.begin(), colptr.end());
    auto colpat = [&](int64_t k) { return ilu1t_pattern(k, cp.data(), rowind.data(), cval.data(), diag, tau); };
    auto rowpat = [&](int64_t k) {
        return ilu1t_pattern(k, A.rowptr.data(), A.colind.data(), A.val.data(), diag, tau);
    };
    // union of the patterns of the columns [g0, g1) and their scalar count
    auto group_sets = [&](int64_t g0, int64_t g1, std::vector<int32_t> &GI, std::vector<int32_t> &GJ) {
        int64_t scal = 0;
        GI.clear();
        GJ.clear();
        for (int64_t k = g0; k < g1; ++k) {
            const std::vector<int32_t> I = colpat(k), J = rowpat(k);
            scal += (int64_t)I.size() + (int64_t)J.size() + 1;
            GI = sorted_union(GI, I);
            GJ = sorted_union(GJ, J);
        }
        return scal;
    };
    std::vector<int32_t> bstart, R, C, GI, GJ;
    const size_t ng = groups.size() - 1;
    size_t g = 0;
    while (g < ng) {
        const int64_t start = groups[g];
        int64_t scalar = group_sets(start, groups[g + 1], R, C);
        int64_t l = groups[g + 1] - start;
        ++g;
        while (g < ng) {
            const int64_t gs = groups[g + 1] - groups[g];
            if (l + gs > max_block) break;
            const int64_t end = groups[g + 1];
            const int64_t gscal = group_sets(groups[g], end, GI, GJ);
            const int64_t r2 = union_count_above(R, GI, end - 1), s2 = union_count_above(C, GJ, end - 1);
            const int64_t l2 = l + gs;
            const int64_t f2 = (r2 + s2 + l2) * l2;
            const int64_t scalar2 = scalar + gscal;
            if (!(3 * f2 <= 4 * scalar2 || f2 <= scalar2 + 4 * l2)) break;
            R = sorted_union(R, GI);
            C = sorted_union(C, GJ);
            scalar = scalar2;
            l = l2;
            ++g;
        }
        bstart.push_back((int32_t)start);
    }
    bstart.push_back((int32_t)n);
    return bstart;
}

std::vector<int32_t> unit_groups(int64_t n) {
    std::vector<int32_t> g(n + 1);
    for (int64_t k = 0; k <= n; ++k) g[k] = (int32_t)k;
    return g;
}

// Pattern checks shared by the host-only helpers: rowptr monotone from 0, column indices in
// range and strictly increasing within each row.  Returns an empty string when valid.
std::string check_pattern(int64_t n, const int64_t *rowptr, const int32_t *colind) {
    if (n < 0 || n >= (int64_t)INT32_MAX) return "n out of range";
    if (n > 0 && (!rowptr || !colind)) return "null CSR array";
    if (n == 0) return "";
    if (rowptr[0] != 0) return "rowptr[0] != 0";
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return "rowptr not monotone";
    if (rowptr[n] >= (int64_t)INT32_MAX) return "nnz >= 2^31 not supported";
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            if (colind[e] < 0 || colind[e] >= n) return "column index out of range";
            if (e > rowptr[i] && colind[e] <= colind[e - 1])
                return "column indices not strictly increasing within a row";
        }
    return "";
}

// count > mu + 2 sigma for each count (mu = nnz / n, sigma the population standard deviation
// of the counts), decided exactly: n count > nnz and (n count - nnz)^2 > 4 (n S - nnz^2),
// S = sum of squared counts.
std::vector<char> above_two_sigma(const std::vector<int64_t> &cnt, int64_t nnz) {
    const __int128 n = (__int128)cnt.size();
    __int128 S = 0;
    for (int64_t v : cnt) S += (__int128)v * v;
    const __int128 var4 = 4 * (n * S - (__int128)nnz * nnz);
    std::vector<char> out(cnt.size(), 0);
    for (size_t i = 0; i < cnt.size(); ++i) {
        const __int128 d = n * cnt[i] - nnz;
        out[i] = d > 0 && d * d > var4;
    }
    return out;
}

}  // namespace

// Sec. 3.2: rows i, j of A with 0/1 patterns c_i, c_j are grouped when
// |c_i n c_j|^2 >= tau |c_i| |c_j|, over the pairs j > i that share a column (the upper part of
// the pattern of A A^T) and are not yet in a block.  Rows are visited in increasing order; an
// unplaced row leads a block and takes its passing partners in increasing order up to
// max_block.  A row or column with more than mu + 2 sigma entries takes no part: its index is
// a block of its own.  perm lists the blocks in the order of their leaders (leader first,
// members ascending); bstart holds the block starts of Q^T A Q.
// The sweep of the cosine blocking over a validated pattern; weight (null: 1 per index) is what
// an index adds to its block, which holds at most max_block of it (a partner that passes the
// test but does not fit is passed over).
static void cosine_core(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau, int32_t max_block,
                        const int32_t *weight, int32_t *perm, int32_t *bstart, int32_t *nblocks) {
    const int64_t nnz = n > 0 ? rowptr[n] : 0;
    // columns of the pattern (rows ascending) and the row / column counts
    std::vector<int64_t> rcnt(n), ccnt(n, 0);
    std::vector<int64_t> cptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) rcnt[i] = rowptr[i + 1] - rowptr[i];
    for (int64_t e = 0; e < nnz; ++e) ccnt[colind[e]]++;
    for (int64_t j = 0; j < n; ++j) cptr[j + 1] = cptr[j] + ccnt[j];
    std::vector<int32_t> crow(nnz);
    {
        std::vector<int64_t> next(cptr.begin(), cptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) crow[next[colind[e]]++] = (int32_t)i;
    }
    const std::vector<char> xr = above_two_sigma(rcnt, nnz), xc = above_two_sigma(ccnt, nnz);
    std::vector<char> placed(n, 0);
    std::vector<int32_t> seen(n, -1), partners;
    int64_t pos = 0;
    int32_t nb = 0;
    bstart[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (placed[i]) continue;
        placed[i] = 1;
        perm[pos++] = (int32_t)i;
        int64_t size = weight ? weight[i] : 1;
        if (!xr[i] && !xc[i]) {
            partners.clear();
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int32_t k = colind[e];
                for (int64_t f = cptr[k]; f < cptr[k + 1]; ++f) {
                    const int32_t j = crow[f];
                    if (j > i && seen[j] != (int32_t)i) {
                        seen[j] = (int32_t)i;
                        partners.push_back(j);
                    }
                }
            }
            std::sort(partners.begin(), partners.end());
            const double ni = (double)rcnt[i];
            for (int32_t j : partners) {
                if (size >= max_block) break;
                const int64_t wj = weight ? weight[j] : 1;
                if (placed[j] || xr[j] || xc[j] || size + wj > max_block) continue;
                // |c_i n c_j| by merging the two sorted rows
                int64_t a = rowptr[i], b = rowptr[j], cnt = 0;
                while (a < rowptr[i + 1] && b < rowptr[j + 1]) {
                    if (colind[a] < colind[b]) ++a;
                    else if (colind[b] < colind[a]) ++b;
                    else { ++cnt; ++a; ++b; }
                }
                if ((double)cnt * (double)cnt >= (tau * ni) * (double)rcnt[j]) {
                    placed[j] = 1;
                    perm[pos++] = j;
                    size += wj;
                }
            }
        }
        bstart[++nb] = (int32_t)pos;
    }
    *nblocks = nb;
}

bilu_status cosine_blocking_host(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                 int32_t max_block, int32_t *perm, int32_t *bstart, int32_t *nblocks,
                                 std::string *err) {
    auto fail = [&](const char *m) { if (err) *err = m; return BILU_ERR_ARG; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(bad.c_str());
    if (!(tau >= 0.0) || !std::isfinite(tau)) return fail("tau must be finite and >= 0");
    if (max_block < 1 || max_block > BILU_MAX_BLOCK) return fail("max_block must be in 1..64");
    if (!bstart || !nblocks || (n > 0 && !perm)) return fail("null output array");
    cosine_core(n, rowptr, colind, tau, max_block, nullptr, perm, bstart, nblocks);
    return BILU_OK;
}

// Sec. 4.2: the cosine blocking of the compressed matrix whose indices are the consecutive
// units [ustart[p], ustart[p + 1]) (the 2 x 2 pivots of the symmetrised matching merged): row p
// of the compressed pattern holds the units of the columns of the rows in unit p; the sweep
// weighs each unit by its size, and the blocks are expanded to the indices of A (units in the
// block's order, the indices of a unit in theirs).
bilu_status cosine_blocking_units_host(int64_t n, const int64_t *rowptr, const int32_t *colind, double tau,
                                       int32_t max_block, int32_t nunits, const int32_t *ustart, int32_t *perm,
                                       int32_t *bstart, int32_t *nblocks, std::string *err) {
    auto fail = [&](const char *m) { if (err) *err = m; return BILU_ERR_ARG; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(bad.c_str());
    if (!(tau >= 0.0) || !std::isfinite(tau)) return fail("tau must be finite and >= 0");
    if (max_block < 1 || max_block > BILU_MAX_BLOCK) return fail("max_block must be in 1..64");
    if (!bstart || !nblocks || (n > 0 && (!perm || !ustart))) return fail("null array");
    if (nunits < 0 || (n > 0 && nunits < 1)) return fail("nunits out of range");
    if (n > 0 && (ustart[0] != 0 || ustart[nunits] != n)) return fail("units must run from 0 to n");
    for (int32_t p = 0; p < nunits; ++p)
        if (ustart[p + 1] <= ustart[p] || ustart[p + 1] - ustart[p] > max_block)
            return fail("unit sizes must be in 1..max_block");
    if (n == 0) {
        bstart[0] = 0;
        *nblocks = 0;
        return BILU_OK;
    }
    std::vector<int32_t> unit_of(n), weight(nunits);
    for (int32_t p = 0; p < nunits; ++p) {
        weight[p] = ustart[p + 1] - ustart[p];
        for (int32_t i = ustart[p]; i < ustart[p + 1]; ++i) unit_of[i] = p;
    }
    std::vector<int64_t> crp(nunits + 1, 0);
    std::vector<int32_t> cci, row;
    for (int32_t p = 0; p < nunits; ++p) {
        row.clear();
        for (int32_t i = ustart[p]; i < ustart[p + 1]; ++i)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) row.push_back(unit_of[colind[e]]);
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        cci.insert(cci.end(), row.begin(), row.end());
        crp[p + 1] = (int64_t)cci.size();
    }
    std::vector<int32_t> uperm(nunits), ub(nunits + 1);
    int32_t nub = 0;
    cosine_core(nunits, crp.data(), cci.data(), tau, max_block, weight.data(), uperm.data(), ub.data(), &nub);
    int64_t pos = 0;
    bstart[0] = 0;
    for (int32_t b = 0; b < nub; ++b) {
        for (int32_t k = ub[b]; k < ub[b + 1]; ++k)
            for (int32_t i = ustart[uperm[k]]; i < ustart[uperm[k] + 1]; ++i) perm[pos++] = i;
        bstart[b + 1] = (int32_t)pos;
    }
    *nblocks = nub;
    return BILU_OK;
}

// The Sec. 3.4 partition on the host: column by column (gstart NULL) or over the given groups.
bilu_status partition_ilu1t_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                 double tau, int32_t max_block, int32_t ngroups, const int32_t *gstart,
                                 int32_t *bstart, int32_t *nblocks, std::string *err) {
    auto fail = [&](const char *m) { if (err) *err = m; return BILU_ERR_ARG; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(bad.c_str());
    if (n > 0 && !val) return fail("null CSR array");
    if (!(tau >= 0.0) || !std::isfinite(tau)) return fail("tau must be finite and >= 0");
    if (max_block < 1 || max_block > BILU_MAX_BLOCK) return fail("max_block must be in 1..64");
    if (!bstart || !nblocks) return fail("null output array");
    HostCSR A;
    A.n = n;
    A.rowptr.assign(rowptr, rowptr + n + 1);
    if (n == 0) A.rowptr.assign(1, 0);
    const int64_t nnz = A.rowptr[n];
    A.colind.assign(colind, colind + nnz);
    A.val.assign(val, val + nnz);
    for (double v : A.val)
        if (!std::isfinite(v)) return fail("non-finite matrix value");
    std::vector<int32_t> groups;
    if (gstart) {
        if (ngroups < 0 || gstart[0] != 0 || gstart[ngroups] != n || (n > 0 && ngroups == 0))
            return fail("groups must run from 0 to n");
        for (int32_t g = 0; g < ngroups; ++g)
            if (gstart[g + 1] - gstart[g] < 1 || gstart[g + 1] - gstart[g] > max_block)
                return fail("group size not in 1..max_block");
        groups.assign(gstart, gstart + ngroups + 1);
    } else {
        groups = unit_groups(n);
    }
    std::vector<int32_t> colptr, rowind;
    std::vector<double> cval;
    build_csc(A, colptr, rowind, cval);
    const std::vector<int32_t> bs = n > 0 ? partition_ilu1t(A, colptr, rowind, cval, tau, max_block, groups)
                                          : std::vector<int32_t>(1, 0);
    std::copy(bs.begin(), bs.end(), bstart);
    *nblocks = (int32_t)bs.size() - 1;
    return BILU_OK;
}

// Sec. 3.1: maximum product transversal and scaling.  Costs c_ij = log a_j - log|a_ij| on the
// stored nonzeros (a_j the largest |a_kj| of column j); a minimum-cost perfect matching sigma by
// one shortest augmenting path per row (Dijkstra on the reduced costs c_ij - u_i - v_j >= 0,
// columns taken by distance, then index); the duals give d_l = e^u, d_r = e^v / a_j, so that
// D_l A D_r has |entries| <= 1 and |entry| = 1 on the matching.
bilu_status mwm_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                     int32_t *sigma, double *dl, double *dr, std::string *err) {
    auto fail = [&](bilu_status st, const char *m) { if (err) *err = m; return st; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(BILU_ERR_ARG, bad.c_str());
    if (n > 0 && (!val || !sigma || !dl || !dr)) return fail(BILU_ERR_ARG, "null array");
    const int64_t nnz = n > 0 ? rowptr[n] : 0;
    std::vector<double> amax(n, 0.0), c(nnz, 0.0);
    for (int64_t e = 0; e < nnz; ++e) {
        if (!std::isfinite(val[e])) return fail(BILU_ERR_ARG, "non-finite matrix value");
        amax[colind[e]] = std::max(amax[colind[e]], std::fabs(val[e]));
    }
    for (int64_t e = 0; e < nnz; ++e)
        if (val[e] != 0.0) c[e] = std::log(amax[colind[e]]) - std::log(std::fabs(val[e]));
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<double> u(n, 0.0), v(n, 0.0), dist(n, inf);
    std::vector<int32_t> row_of(n, -1), col_of(n, -1), prev(n, -1), touched, finished;
    std::vector<char> done(n, 0);
    using Item = std::pair<double, int32_t>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int64_t s = 0; s < n; ++s) {
        auto relax = [&](int32_t i, double base) {
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int32_t k = colind[e];
                if (val[e] == 0.0 || done[k]) continue;
                const double d = base + c[e] - u[i] - v[k];
                if (d < dist[k]) {
                    if (dist[k] == inf) touched.push_back(k);
                    dist[k] = d;
                    prev[k] = i;
                    heap.push({d, k});
                }
            }
        };
        relax((int32_t)s, 0.0);
        int32_t free = -1;
        while (!heap.empty()) {
            const auto [d, j] = heap.top();
            heap.pop();
            if (done[j] || d > dist[j]) continue;
            done[j] = 1;
            finished.push_back(j);
            if (row_of[j] < 0) { free = j; break; }
            relax(row_of[j], dist[j]);
        }
        if (free < 0) return fail(BILU_ERR_SINGULAR, "structurally singular: no perfect matching on the nonzeros");
        const double D = dist[free];
        u[s] += D;
        for (int32_t j : finished)
            if (j != free) {
                u[row_of[j]] += D - dist[j];
                v[j] -= D - dist[j];
            }
        for (int32_t j = free;;) {  // augment along the path
            const int32_t i = prev[j], nxt = col_of[i];
            row_of[j] = i;
            col_of[i] = j;
            if (i == s) break;
            j = nxt;
        }
        for (int32_t k : touched) { dist[k] = inf; done[k] = 0; prev[k] = -1; }
        touched.clear();
        finished.clear();
        heap = decltype(heap)();
    }
    for (int64_t i = 0; i < n; ++i) {
        sigma[i] = col_of[i];
        dl[i] = std::exp(u[i]);
        dr[i] = std::exp(v[i]) / (amax[i] > 0.0 ? amax[i] : 1.0);
    }
    return BILU_OK;
}

// B[k][l] = dl[r_k] A[r_k][c_l] dr[c_l] with r_k = rowperm[k], c_l = colperm[l] (identity or
// unit scaling where a pointer is NULL); each row of B sorted by column.
// Sec. 4.2: the symmetrised matching of the symmetric variant (Duff and Pralet).  The
// unsymmetric matching sigma with its scalings d_l, d_r gives the symmetric scaling
// d = sqrt(d_l d_r) (|d_i a_ij d_j| <= 1 for symmetric A) and, from the cycles of sigma, pivot
// units: a one-index cycle is a 1 x 1 unit, a two-index cycle a 2 x 2 unit; a longer cycle
// c_0 .. c_{k-1} is cut into pairs of neighbours (c_t, c_{t+1}), whose coupling is a matched
// entry: for even k the cut starting at c_0 or at c_1 with the larger sum of log |a_pair|, for
// odd k the cut leaving c_s alone that maximises log |a_{c_s c_s}| + sum log |a_pair| (the first
// on ties; a zero diagonal counts as -inf).  Units are ordered by their smallest index, the
// indices of a unit increasing.
static double abs_entry(const int64_t *rowptr, const int32_t *colind, const double *val, int32_t i, int32_t j) {
    const int32_t *lo = colind + rowptr[i], *hi = colind + rowptr[i + 1];
    const int32_t *p = std::lower_bound(lo, hi, j);
    return (p < hi && *p == j) ? std::fabs(val[rowptr[i] + (p - lo)]) : 0.0;
}

static double log_or_minus_inf(double x) { return x > 0.0 ? std::log(x) : -INFINITY; }

bilu_status sym_mwm_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val, int32_t *perm,
                         double *ds, int32_t *ustart, int32_t *nunits, std::string *err) {
    auto fail = [&](bilu_status st, const char *m) { if (err) *err = m; return st; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(BILU_ERR_ARG, bad.c_str());
    if (!nunits || (n > 0 && (!val || !perm || !ds || !ustart))) return fail(BILU_ERR_ARG, "null array");
    for (int64_t i = 0; i < n; ++i)  // A = A^T entry by entry
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int32_t j = colind[e];
            const int32_t *lo = colind + rowptr[j], *hi = colind + rowptr[j + 1];
            const int32_t *p = std::lower_bound(lo, hi, (int32_t)i);
            if (p == hi || *p != (int32_t)i || val[rowptr[j] + (p - lo)] != val[e])
                return fail(BILU_ERR_ARG, "the symmetric matching needs a symmetric matrix");
        }
    std::vector<int32_t> sigma(std::max<int64_t>(n, 1));
    std::vector<double> dl(std::max<int64_t>(n, 1)), dr(std::max<int64_t>(n, 1));
    const bilu_status st = mwm_host(n, rowptr, colind, val, sigma.data(), dl.data(), dr.data(), err);
    if (st != BILU_OK) return st;
    for (int64_t i = 0; i < n; ++i) ds[i] = std::sqrt(dl[i] * dr[i]);
    std::vector<std::vector<int32_t>> units;
    std::vector<char> seen(std::max<int64_t>(n, 1), 0);
    std::vector<int32_t> cyc;
    auto pair_log = [&](int64_t t, int64_t k) {
        return log_or_minus_inf(abs_entry(rowptr, colind, val, cyc[t % k], cyc[(t + 1) % k]));
    };
    auto add_pair = [&](int32_t a, int32_t b) { units.push_back({std::min(a, b), std::max(a, b)}); };
    for (int64_t i = 0; i < n; ++i) {
        if (seen[i]) continue;
        cyc.clear();
        for (int32_t j = (int32_t)i; !seen[j]; j = sigma[j]) {
            seen[j] = 1;
            cyc.push_back(j);
        }
        const int64_t k = (int64_t)cyc.size();
        if (k == 1) {
            units.push_back({cyc[0]});
        } else if (k == 2) {
            add_pair(cyc[0], cyc[1]);
        } else if (k % 2 == 0) {
            double best = 0.0;
            int64_t first = 0;
            for (int64_t start = 0; start < 2; ++start) {
                double score = 0.0;
                for (int64_t t = start; t < start + k; t += 2) score += pair_log(t, k);
                if (start == 0 || score > best) { best = score; first = start; }
            }
            for (int64_t t = first; t < first + k; t += 2) add_pair(cyc[t % k], cyc[(t + 1) % k]);
        } else {
            double best = 0.0;
            int64_t alone = 0;
            for (int64_t sx = 0; sx < k; ++sx) {
                double score = log_or_minus_inf(abs_entry(rowptr, colind, val, cyc[sx], cyc[sx]));
                for (int64_t t = sx + 1; t < sx + k; t += 2) score += pair_log(t, k);
                if (sx == 0 || score > best) { best = score; alone = sx; }
            }
            units.push_back({cyc[alone]});
            for (int64_t t = alone + 1; t < alone + k; t += 2) add_pair(cyc[t % k], cyc[(t + 1) % k]);
        }
    }
    std::sort(units.begin(), units.end(), [](const auto &x, const auto &y) { return x[0] < y[0]; });
    int64_t pos = 0;
    ustart[0] = 0;
    for (size_t u = 0; u < units.size(); ++u) {
        for (int32_t v : units[u]) perm[pos++] = v;
        ustart[u + 1] = (int32_t)pos;
    }
    *nunits = (int32_t)units.size();
    return BILU_OK;
}

bilu_status scale_permute_csr_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                   const int32_t *rowperm, const int32_t *colperm, const double *dl,
                                   const double *dr, int64_t *out_rowptr, int32_t *out_colind, double *out_val,
                                   std::string *err) {
    auto fail = [&](const char *m) { if (err) *err = m; return BILU_ERR_ARG; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(bad.c_str());
    if (!out_rowptr || (n > 0 && (!val || !out_colind || !out_val))) return fail("null array");
    auto inverse = [&](const int32_t *p, std::vector<int32_t> &inv) {
        inv.assign(n, -1);
        for (int64_t k = 0; k < n; ++k) {
            if (p[k] < 0 || p[k] >= n || inv[p[k]] >= 0) return false;
            inv[p[k]] = (int32_t)k;
        }
        return true;
    };
    std::vector<int32_t> icol, irow;
    if (rowperm && !inverse(rowperm, irow)) return fail("rowperm is not a permutation");
    if (colperm && !inverse(colperm, icol)) return fail("colperm is not a permutation");
    out_rowptr[0] = 0;
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t k = 0; k < n; ++k) {
        const int32_t i = rowperm ? rowperm[k] : (int32_t)k;
        row.clear();
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int32_t j = colind[e];
            double a = val[e];
            // one product of the two scalings: with dl = dr a symmetric A stays symmetric bit for bit
            if (dl || dr) a *= (dl ? dl[i] : 1.0) * (dr ? dr[j] : 1.0);
            row.emplace_back(colperm ? icol[j] : j, a);
        }
        std::sort(row.begin(), row.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        int64_t o = out_rowptr[k];
        for (const auto &rv : row) { out_colind[o] = rv.first; out_val[o] = rv.second; ++o; }
        out_rowptr[k + 1] = o;
    }
    return BILU_OK;
}

namespace {

// Symmetrised companion graph of a block partition: K ~ L when A couples B_K and B_L in either
// direction (sorted, unique adjacency lists).
std::vector<std::vector<int32_t>> block_graph(int64_t n, const int64_t *rowptr, const int32_t *colind,
                                              int32_t nb, const int32_t *bstart) {
    std::vector<int32_t> blk(n);
    for (int32_t K = 0; K < nb; ++K)
        for (int32_t i = bstart[K]; i < bstart[K + 1]; ++i) blk[i] = K;
    std::vector<std::vector<int32_t>> adj(nb);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int32_t K = blk[i], L = blk[colind[e]];
            if (K != L) {
                adj[K].push_back(L);
                adj[L].push_back(K);
            }
        }
    for (auto &a : adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    return adj;
}

// George's level-structure nested dissection of the block graph (Sec. 3.3 with a dissection
// written here in place of METIS).  A connected set of more than `leaf` nodes is split by the
// breadth-first level structure from a pseudo-peripheral node (from the set's smallest node,
// move to a least-degree node of the last level, ties by index, while the level count grows):
// the middle level (L / 2 of L levels) is the separator, the levels before and after it the
// two parts; order = first part, second part, separator (ascending).  Fewer than 3 levels, or
// at most `leaf` nodes: ascending order.  A disconnected set: its components by smallest node.
struct Dissection {
    const std::vector<std::vector<int32_t>> &adj;
    int leaf;
    std::vector<int32_t> mark, seen, out;
    int32_t marks = 0, seens = 0;

    Dissection(const std::vector<std::vector<int32_t>> &a, int lf)
        : adj(a), leaf(lf), mark(a.size(), 0), seen(a.size(), 0) {}

    std::vector<std::vector<int32_t>> levels(int32_t sid, int32_t root) {
        ++seens;
        seen[root] = seens;
        std::vector<std::vector<int32_t>> L{{root}};
        for (;;) {
            std::vector<int32_t> nxt;
            for (int32_t v : L.back())
                for (int32_t w : adj[v])
                    if (mark[w] == sid && seen[w] != seens) {
                        seen[w] = seens;
                        nxt.push_back(w);
                    }
            if (nxt.empty()) return L;
            std::sort(nxt.begin(), nxt.end());
            L.push_back(std::move(nxt));
        }
    }

    int degree(int32_t v, int32_t sid) const {
        int d = 0;
        for (int32_t w : adj[v]) d += mark[w] == sid;
        return d;
    }

    void dissect(std::vector<int32_t> nodes) {
        const int32_t sid = ++marks;
        for (int32_t v : nodes) mark[v] = sid;
        std::sort(nodes.begin(), nodes.end());
        // components, by smallest node
        std::vector<std::vector<int32_t>> comps;
        ++seens;
        const int32_t cs = seens;
        for (int32_t v : nodes) {
            if (seen[v] == cs) continue;
            std::vector<int32_t> comp{v};
            seen[v] = cs;
            for (size_t q = 0; q < comp.size(); ++q)
                for (int32_t w : adj[comp[q]])
                    if (mark[w] == sid && seen[w] != cs) {
                        seen[w] = cs;
                        comp.push_back(w);
                    }
            comps.push_back(std::move(comp));
        }
        for (auto &comp : comps) {
            std::sort(comp.begin(), comp.end());
            if ((int)comp.size() <= leaf) {
                out.insert(out.end(), comp.begin(), comp.end());
                continue;
            }
            const int32_t cid = ++marks;
            for (int32_t v : comp) mark[v] = cid;
            int32_t root = comp[0];
            auto L = levels(cid, root);
            for (;;) {
                int32_t cand = -1, cdeg = 0;
                for (int32_t v : L.back()) {
                    const int d = degree(v, cid);
                    if (cand < 0 || d < cdeg || (d == cdeg && v < cand)) { cand = v; cdeg = d; }
                }
                auto L2 = levels(cid, cand);
                if (L2.size() <= L.size()) break;
                root = cand;
                L = std::move(L2);
            }
            if (L.size() < 3) {
                out.insert(out.end(), comp.begin(), comp.end());
                continue;
            }
            const size_t m = L.size() / 2;
            std::vector<int32_t> first, second;
            for (size_t k = 0; k < m; ++k) first.insert(first.end(), L[k].begin(), L[k].end());
            for (size_t k = m + 1; k < L.size(); ++k) second.insert(second.end(), L[k].begin(), L[k].end());
            const std::vector<int32_t> sep = L[m];
            dissect(std::move(first));
            dissect(std::move(second));
            out.insert(out.end(), sep.begin(), sep.end());
        }
    }
};

std::string check_partition(int64_t n, int32_t nb, const int32_t *bstart) {
    if (nb < 0 || !bstart) return "invalid partition";
    if (bstart[0] != 0 || bstart[nb] != n || (n > 0 && nb == 0)) return "partition must run from 0 to n";
    for (int32_t K = 0; K < nb; ++K)
        if (bstart[K + 1] <= bstart[K]) return "partition not strictly increasing";
    return "";
}

}  // namespace

bilu_status nd_order_host(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nb,
                          const int32_t *bstart, int32_t leaf, int32_t *perm, int32_t *bstart_out,
                          int32_t *order_out, std::string *err) {
    auto fail = [&](const std::string &m) { if (err) *err = m; return BILU_ERR_ARG; };
    std::string bad = check_pattern(n, rowptr, colind);
    if (bad.empty()) bad = check_partition(n, nb, bstart);
    if (!bad.empty()) return fail(bad);
    if (leaf < 1) return fail("leaf must be >= 1");
    if (!bstart_out || (n > 0 && (!perm || !order_out))) return fail("null output array");
    const auto adj = block_graph(n, rowptr, colind, nb, bstart);
    Dissection d(adj, leaf);
    std::vector<int32_t> all(nb);
    std::iota(all.begin(), all.end(), 0);
    d.dissect(all);
    int64_t pos = 0;
    bstart_out[0] = 0;
    for (int32_t k = 0; k < nb; ++k) {
        const int32_t K = d.out[k];
        order_out[k] = K;
        for (int32_t i = bstart[K]; i < bstart[K + 1]; ++i) perm[pos++] = i;
        bstart_out[k + 1] = (int32_t)pos;
    }
    return BILU_OK;
}

// Elimination tree of the symmetrised block graph: eliminating the blocks in order, each one's
// later neighbours become a clique, so they are handed to its first later neighbour, its parent.
bilu_status block_etree_host(int64_t n, const int64_t *rowptr, const int32_t *colind, int32_t nb,
                             const int32_t *bstart, int32_t *parent, int32_t *height, std::string *err) {
    auto fail = [&](const std::string &m) { if (err) *err = m; return BILU_ERR_ARG; };
    std::string bad = check_pattern(n, rowptr, colind);
    if (bad.empty()) bad = check_partition(n, nb, bstart);
    if (!bad.empty()) return fail(bad);
    if (!height || (nb > 0 && !parent)) return fail("null output array");
    const auto adj = block_graph(n, rowptr, colind, nb, bstart);
    std::vector<std::vector<int32_t>> later(nb);
    for (int32_t K = 0; K < nb; ++K)
        for (int32_t w : adj[K])
            if (w > K) later[K].push_back(w);
    std::vector<int32_t> h(nb, 1);
    for (int32_t K = 0; K < nb; ++K) {
        parent[K] = -1;
        if (later[K].empty()) continue;
        const int32_t p = later[K][0];
        parent[K] = p;
        std::vector<int32_t> merged;
        std::set_union(later[p].begin(), later[p].end(), later[K].begin() + 1, later[K].end(),
                       std::back_inserter(merged));
        later[p] = std::move(merged);
        std::vector<int32_t>().swap(later[K]);
        h[p] = std::max(h[p], h[K] + 1);
    }
    *height = nb > 0 ? *std::max_element(h.begin(), h.end()) : 0;
    return BILU_OK;
}

// A~ = Q^T A Q: row k of A~ is row perm[k] of A with every column j renamed iperm[j] and the
// row re-sorted.
bilu_status permute_csr_host(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                             const int32_t *perm, int64_t *out_rowptr, int32_t *out_colind, double *out_val,
                             std::string *err) {
    auto fail = [&](const char *m) { if (err) *err = m; return BILU_ERR_ARG; };
    const std::string bad = check_pattern(n, rowptr, colind);
    if (!bad.empty()) return fail(bad.c_str());
    if (!out_rowptr || (n > 0 && (!perm || !val || !out_colind || !out_val))) return fail("null array");
    std::vector<int32_t> iperm(n, -1);
    for (int64_t k = 0; k < n; ++k) {
        if (perm[k] < 0 || perm[k] >= n || iperm[perm[k]] >= 0) return fail("perm is not a permutation");
        iperm[perm[k]] = (int32_t)k;
    }
    out_rowptr[0] = 0;
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t k = 0; k < n; ++k) {
        const int32_t i = perm[k];
        row.clear();
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) row.emplace_back(iperm[colind[e]], val[e]);
        std::sort(row.begin(), row.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        int64_t o = out_rowptr[k];
        for (const auto &rv : row) { out_colind[o] = rv.first; out_val[o] = rv.second; ++o; }
        out_rowptr[k + 1] = o;
    }
    return BILU_OK;
}

void matrix_free(bilu_ctx *c) {
    dev_free(c->d_parent);
    dev_free(c->d_tree0);
    dev_free(c->d_tree);
    c->h_parent.clear();
    c->tree_split = c->tree_height = c->tree_nleaves = 0;
    dev_free(c->d_rowptr);
    dev_free(c->d_colind);
    dev_free(c->d_val);
    dev_free(c->d_colptr);
    dev_free(c->d_rowind);
    dev_free(c->d_cval);
    dev_free(c->d_bstart);
    dev_free(c->d_blkof);
    dev_free(c->d_Dptr);
}

// The tree schedule's static data (Sec. 3.3: each block depends only on its subtree): the
// block elimination tree of the partition and the trunk (the longest run of blocks at the end
// in which every block's only child is the block before it, down to the first block with
// another child count: factored by the whole grid).  The device copy of the initial queue
// state is built by tree_init (below) for the trunk the factorization uses.
bilu_status tree_setup(bilu_ctx *c, const HostCSR &A) {
    const int32_t nb = c->nb;
    std::vector<int32_t> parent(std::max(nb, 1), -1);
    int32_t height = 0;
    std::string err;
    if (nb > 0) {
        const bilu_status st = block_etree_host(A.n, A.rowptr.data(), A.colind.data(), nb, c->h_bstart.data(),
                                                parent.data(), &height, &err);
        if (st != BILU_OK) return set_err(c, st, "block elimination tree: " + err);
    }
    std::vector<int32_t> nchild(std::max(nb, 1), 0);
    for (int32_t K = 0; K < nb; ++K)
        if (parent[K] >= 0) nchild[parent[K]]++;
    int32_t split = nb;
    if (nb > 0 && parent[nb - 1] < 0) {
        split = nb - 1;
        while (split > 0 && nchild[split] == 1 && parent[split - 1] == split) --split;
    }
    c->h_parent.assign(parent.begin(), parent.begin() + nb);
    c->tree_split = split;
    c->tree_height = height;
    c->tree_init_split = -1;
    cudaError_t e;
    if ((e = dev_alloc(&c->d_parent, std::max(nb, 1))) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_parent, parent.data(), std::max(nb, 1) * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? set_err(c, BILU_ERR_OOM, "device allocation failed in analyze")
                                              : cuda_err(c, e, "tree upload");
    return BILU_OK;
}

// Initial queue state of a tree factorization whose trunk starts at block `split` (d_tree0;
// copied to d_tree before every run).  Int32 words: [0, 8) four 64-bit pool cursors, [8, 12)
// the whole-grid barrier, [12, 14) queue head and tail, [14, 14 + nsm) the group slots, then
// pending[nb] (children of every block below the trunk not finished yet) and queue[nb] (the
// leaves below the trunk first, those farthest from the trunk first; -1 elsewhere).
bilu_status tree_init(bilu_ctx *c, int32_t split) {
    if (c->tree_init_split == split && c->d_tree0 && c->d_tree) return BILU_OK;
    const int32_t nb = c->nb;
    const std::vector<int32_t> &parent = c->h_parent;
    std::vector<int32_t> nchild(std::max(nb, 1), 0), depth(std::max(nb, 1), 0);
    for (int32_t K = 0; K < split; ++K)
        if (parent[K] >= 0 && parent[K] < split) nchild[parent[K]]++;
    for (int32_t K = split - 1; K >= 0; --K)
        depth[K] = (parent[K] >= 0 && parent[K] < split) ? depth[parent[K]] + 1 : 0;
    std::vector<int32_t> leaves;
    for (int32_t K = 0; K < split; ++K)
        if (nchild[K] == 0) leaves.push_back(K);
    std::stable_sort(leaves.begin(), leaves.end(), [&](int32_t x, int32_t y) { return depth[x] > depth[y]; });
    const int64_t words = 14 + (int64_t)c->nsm + 2 * (int64_t)std::max(nb, 1);
    std::vector<int32_t> t0(words, 0);
    t0[13] = (int32_t)leaves.size();
    int32_t *pending = t0.data() + 14 + c->nsm, *queue = pending + std::max(nb, 1);
    for (int32_t K = 0; K < std::max(nb, 1); ++K) queue[K] = -1;
    for (int32_t K = 0; K < split; ++K) pending[K] = nchild[K];
    for (size_t i = 0; i < leaves.size(); ++i) queue[i] = leaves[i];
    dev_free(c->d_tree0);
    dev_free(c->d_tree);
    c->tree_init_split = -1;
    cudaError_t e;
    if ((e = dev_alloc(&c->d_tree0, words)) != cudaSuccess || (e = dev_alloc(&c->d_tree, words)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_tree0, t0.data(), words * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? set_err(c, BILU_ERR_OOM, "device allocation failed in factor")
                                              : cuda_err(c, e, "tree queue upload");
    c->tree_init_split = split;
    c->tree_nleaves = (int32_t)leaves.size();
    return BILU_OK;
}

bilu_status analyze_run(bilu_ctx *c, int64_t n, const int64_t *rowptr, const int32_t *colind,
                        const double *val, int on_device, const bilu_params *p,
                        const int32_t *given_bstart, int32_t given_nb) {
    if (!p) return set_err(c, BILU_ERR_ARG, "params is NULL");
    if (n < 0 || n >= (int64_t)INT32_MAX) return set_err(c, BILU_ERR_ARG, "n out of range");
    if (p->max_block < 1 || p->max_block > BILU_MAX_BLOCK)
        return set_err(c, BILU_ERR_ARG, "max_block must be in 1..64");
    const bool given = given_nb >= 0;
    if (!given && p->blocking == BILU_BLOCKING_FIXED && (p->fixed_block < 1 || p->fixed_block > p->max_block))
        return set_err(c, BILU_ERR_ARG, "fixed_block must be in 1..max_block");
    if (!given && p->blocking != BILU_BLOCKING_FIXED && p->blocking != BILU_BLOCKING_ILU1T)
        return set_err(c, BILU_ERR_ARG, "unknown blocking");
    if (given) {  // a caller's partition: 0 = s_0 < s_1 < ... < s_nb = n, blocks <= max_block
        if (!given_bstart) return set_err(c, BILU_ERR_ARG, "null partition");
        if (given_bstart[0] != 0 || given_bstart[given_nb] != n || (n > 0 && given_nb == 0))
            return set_err(c, BILU_ERR_ARG, "partition must run from 0 to n");
        for (int32_t K = 0; K < given_nb; ++K) {
            const int64_t b = (int64_t)given_bstart[K + 1] - given_bstart[K];
            if (b < 1 || b > p->max_block) return set_err(c, BILU_ERR_ARG, "partition block size not in 1..max_block");
        }
    }
    if (!(p->tau_analyze >= 0.0) || !(p->pert_tau >= 0.0) || !(p->pert_rho >= 0.0))
        return set_err(c, BILU_ERR_ARG, "negative or NaN tolerance");
    if (p->precision != BILU_PREC_FP64 && p->precision != BILU_PREC_FP32 && p->precision != BILU_PREC_BF16)
        return set_err(c, BILU_ERR_ARG, "unknown precision");
    if (p->skip != BILU_SKIP_NONE && p->skip != BILU_SKIP_BOUND && p->skip != BILU_SKIP_LEARNED)
        return set_err(c, BILU_ERR_ARG, "unknown skip mode");
    if (n > 0 && (!rowptr || !colind || !val)) return set_err(c, BILU_ERR_ARG, "null CSR array");
    if (p->schedule != BILU_SCHED_CHAIN && p->schedule != BILU_SCHED_TREE)
        return set_err(c, BILU_ERR_ARG, "unknown schedule");
    if (p->group_ctas < 0 || p->group_ctas > c->nsm)
        return set_err(c, BILU_ERR_ARG, "group_ctas must be in 0..number of SMs");
    if (p->aggregate_max != 0 && (p->aggregate_max < 2 || p->aggregate_max > BILU_MAX_BLOCK))
        return set_err(c, BILU_ERR_ARG, "aggregate_max must be 0 or in 2..BILU_MAX_BLOCK");
    if (p->symmetric != 0 && p->symmetric != 1) return set_err(c, BILU_ERR_ARG, "symmetric must be 0 or 1");
    if (p->symmetric && (p->skip != BILU_SKIP_NONE || p->aggregate_max != 0))
        return set_err(c, BILU_ERR_ARG, "the symmetric variant takes no skip mode and no aggregation");

    const auto t_start = std::chrono::steady_clock::now();

    HostCSR A;
    A.n = n;
    A.rowptr.assign(n + 1, 0);
    if (n > 0) {
        if (on_device) {
            BILU_CUDA(c, cudaMemcpy(A.rowptr.data(), rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(A.rowptr.data(), rowptr, (n + 1) * sizeof(int64_t));
        }
    }
    if (A.rowptr[0] != 0) return set_err(c, BILU_ERR_ARG, "rowptr[0] != 0");
    for (int64_t i = 0; i < n; ++i)
        if (A.rowptr[i + 1] < A.rowptr[i]) return set_err(c, BILU_ERR_ARG, "rowptr not monotone");
    const int64_t nnz = A.rowptr[n];
    if (nnz >= (int64_t)INT32_MAX) return set_err(c, BILU_ERR_ARG, "nnz >= 2^31 not supported");
    A.colind.resize(nnz);
    A.val.resize(nnz);
    if (nnz > 0) {
        if (on_device) {
            BILU_CUDA(c, cudaMemcpy(A.colind.data(), colind, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
            BILU_CUDA(c, cudaMemcpy(A.val.data(), val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(A.colind.data(), colind, nnz * sizeof(int32_t));
            std::memcpy(A.val.data(), val, nnz * sizeof(double));
        }
    }
    double alpha = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
            if (A.colind[e] < 0 || A.colind[e] >= n) return set_err(c, BILU_ERR_ARG, "column index out of range");
            if (e > A.rowptr[i] && A.colind[e] <= A.colind[e - 1])
                return set_err(c, BILU_ERR_ARG, "column indices not strictly increasing within a row");
            if (!std::isfinite(A.val[e])) return set_err(c, BILU_ERR_ARG, "non-finite matrix value");
            alpha = std::max(alpha, std::fabs(A.val[e]));
        }

    std::vector<int32_t> colptr, rowind;
    std::vector<double> cval;
    build_csc(A, colptr, rowind, cval);
    if (p->symmetric) {
        // with strictly increasing columns in every row, A = A^T exactly when its column
        // storage equals its row storage
        for (int64_t i = 0; i <= n; ++i)
            if ((int64_t)colptr[i] != A.rowptr[i]) return set_err(c, BILU_ERR_ARG, "symmetric variant: A is not symmetric");
        for (int64_t e = 0; e < nnz; ++e)
            if (rowind[e] != A.colind[e] || cval[e] != A.val[e])
                return set_err(c, BILU_ERR_ARG, "symmetric variant: A is not symmetric");
    }

    std::vector<int32_t> bstart;
    if (given && p->blocking == BILU_BLOCKING_ILU1T && n > 0) {
        // the given blocks are groups that the Sec. 3.4 growth rule merges
        const std::vector<int32_t> groups(given_bstart, given_bstart + given_nb + 1);
        bstart = partition_ilu1t(A, colptr, rowind, cval, p->tau_analyze, p->max_block, groups);
    } else if (given) {
        bstart.assign(given_bstart, given_bstart + given_nb + 1);
    } else if (p->blocking == BILU_BLOCKING_FIXED) {
        for (int64_t s = 0; s < n; s += p->fixed_block) bstart.push_back((int32_t)s);
        bstart.push_back((int32_t)n);
    } else {
        bstart = partition_ilu1t(A, colptr, rowind, cval, p->tau_analyze, p->max_block, unit_groups(n));
    }
    if (n == 0) bstart.assign(1, 0);

    // (re)build device state
    factor_free(c);
    apply_free(c);
    gmres_free(c);
    sqmr_free(c);
    matrix_free(c);
    c->state = 0;
    c->p = *p;
    c->n = n;
    c->nnz = nnz;
    c->alpha = alpha;
    c->h_bstart = bstart;
    c->nb = (int32_t)bstart.size() - 1;
    c->bmax = 0;
    c->bmin = n > 0 ? BILU_MAX_BLOCK : 0;
    c->h_Dptr.assign(c->nb + 1, 0);
    std::vector<int32_t> blkof(std::max<int64_t>(n, 1));
    for (int32_t K = 0; K < c->nb; ++K) {
        const int32_t b = bstart[K + 1] - bstart[K];
        c->bmax = std::max(c->bmax, b);
        c->bmin = std::min(c->bmin, b);
        c->h_Dptr[K + 1] = c->h_Dptr[K] + (int64_t)b * b;
        for (int32_t i = bstart[K]; i < bstart[K + 1]; ++i) blkof[i] = K;
    }
    std::vector<int32_t> rp32(n + 1);
    for (int64_t i = 0; i <= n; ++i) rp32[i] = (int32_t)A.rowptr[i];

    auto up = [&](auto *&dptr, const auto &vec) -> cudaError_t {
        using T = std::remove_reference_t<decltype(*dptr)>;
        cudaError_t e = dev_alloc(&dptr, (int64_t)vec.size());
        if (e != cudaSuccess) return e;
        if (vec.empty()) return cudaSuccess;
        return cudaMemcpyAsync((void *)dptr, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
    };
    cudaError_t e;
    if ((e = up(c->d_rowptr, rp32)) != cudaSuccess || (e = up(c->d_colind, A.colind)) != cudaSuccess ||
        (e = up(c->d_val, A.val)) != cudaSuccess || (e = up(c->d_colptr, colptr)) != cudaSuccess ||
        (e = up(c->d_rowind, rowind)) != cudaSuccess || (e = up(c->d_cval, cval)) != cudaSuccess ||
        (e = up(c->d_bstart, bstart)) != cudaSuccess || (e = up(c->d_blkof, blkof)) != cudaSuccess ||
        (e = up(c->d_Dptr, c->h_Dptr)) != cudaSuccess) {
        matrix_free(c);
        return e == cudaErrorMemoryAllocation ? set_err(c, BILU_ERR_OOM, "device allocation failed in analyze")
                                              : cuda_err(c, e, "analyze upload");
    }
    if (p->schedule == BILU_SCHED_TREE) {
        bilu_status st = tree_setup(c, A);
        if (st != BILU_OK) {
            matrix_free(c);
            return st;
        }
    }
    BILU_CUDA(c, cudaStreamSynchronize(c->stream));
    c->t_analyze_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    c->state = 1;
    return BILU_OK;
}
