// Random-input stress of the library's host analysis (Sec. 3.1-3.4 helpers), built with the
// address and undefined-behaviour sanitizers by tests/test_host_analysis_sanitizers.py.  Only host
// code runs; the stubs stand for the device-side symbols analyze.cu refers to but never reaches here.
#include <algorithm>
#include <cstdio>
#include <limits>
#include <random>
#include <string>
#include <vector>
#include "bilu_internal.h"

// stubs for symbols analyze.cu references but this driver never calls
void factor_free(bilu_ctx *) {}
void apply_free(bilu_ctx *) {}
void gmres_free(bilu_ctx *) {}
void sqmr_free(bilu_ctx *) {}
bilu_status set_err(bilu_ctx *, bilu_status st, const std::string &) { return st; }
bilu_status cuda_err(bilu_ctx *, cudaError_t, const char *) { return BILU_ERR_CUDA; }

int main() {
    std::mt19937_64 rng(1);
    long checked = 0;
    for (int trial = 0; trial < 3000; ++trial) {
        const int n = (int)(rng() % 40);
        const double dens = std::vector<double>{0.0, 0.05, 0.2, 0.6, 1.0}[rng() % 5];
        std::vector<int64_t> rp(n + 1, 0);
        std::vector<int32_t> ci;
        std::vector<double> va;
        std::uniform_real_distribution<double> U(-2, 2), Pr(0, 1);
        const bool diag = rng() % 2;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j)
                if ((diag && i == j) || Pr(rng) < dens) { ci.push_back(j); va.push_back(i == j ? 4.0 : U(rng)); }
            rp[i + 1] = (int64_t)ci.size();
        }
        std::string err;
        const int mb = 1 + (int)(rng() % 64);
        std::vector<int32_t> perm(n + 1), bs(n + 2), order(n + 1), parent(n + 1), sigma(n + 1);
        std::vector<double> dl(n + 1), dr(n + 1);
        int32_t nb = 0, h = 0;
        cosine_blocking_host(n, rp.data(), ci.data(), Pr(rng), mb, perm.data(), bs.data(), &nb, &err);
        partition_ilu1t_host(n, rp.data(), ci.data(), va.data(), Pr(rng) * 0.3, mb, nb, bs.data(), order.data(), &h,
                             &err);
        partition_ilu1t_host(n, rp.data(), ci.data(), va.data(), 1e-2, mb, -1, nullptr, order.data(), &h, &err);
        std::vector<int64_t> orp(n + 1);
        std::vector<int32_t> oci(ci.size() + 1);
        std::vector<double> ova(va.size() + 1);
        permute_csr_host(n, rp.data(), ci.data(), va.data(), perm.data(), orp.data(), oci.data(), ova.data(), &err);
        // partition for the dissection: blocks of random width
        std::vector<int32_t> part{0};
        while (part.back() < n) part.push_back(std::min(n, part.back() + 1 + (int)(rng() % 4)));
        const int32_t np = (int32_t)part.size() - 1;
        std::vector<int32_t> pbs(np + 1), pord(np + 1);
        nd_order_host(n, rp.data(), ci.data(), np, part.data(), 1 + (int)(rng() % 3), perm.data(), pbs.data(),
                      pord.data(), &err);
        block_etree_host(n, rp.data(), ci.data(), np, part.data(), parent.data(), &h, &err);
        mwm_host(n, rp.data(), ci.data(), va.data(), sigma.data(), dl.data(), dr.data(), &err);
        scale_permute_csr_host(n, rp.data(), ci.data(), va.data(), perm.data(), perm.data(), dl.data(), dr.data(),
                               orp.data(), oci.data(), ova.data(), &err);
        {
            // the symmetrised matching: refused on this (mostly unsymmetric) pattern, then run on
            // its symmetric part (a_ij and a_ji both set to the row-major first of the two)
            std::vector<int32_t> us(n + 2);
            int32_t nu = 0;
            sym_mwm_host(n, rp.data(), ci.data(), va.data(), perm.data(), dl.data(), us.data(), &nu, &err);
            std::vector<std::vector<std::pair<int32_t, double>>> rows(n);
            for (int i = 0; i < n; ++i)
                for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                    const int j = ci[e];
                    if (j >= i) {
                        rows[i].push_back({j, va[e]});
                        if (j != i) rows[j].push_back({i, va[e]});
                    }
                }
            std::vector<int64_t> srp(n + 1, 0);
            std::vector<int32_t> sci;
            std::vector<double> sva;
            for (int i = 0; i < n; ++i) {
                std::sort(rows[i].begin(), rows[i].end());
                for (const auto &rv : rows[i]) { sci.push_back(rv.first); sva.push_back(rv.second); }
                srp[i + 1] = (int64_t)sci.size();
            }
            sym_mwm_host(n, srp.data(), sci.data(), sva.data(), perm.data(), dl.data(), us.data(), &nu, &err);
            // the cosine blocking of the pattern compressed by random units (some invalid)
            std::vector<int32_t> units{0};
            while (units.back() < n) units.push_back(std::min(n, units.back() + 1 + (int)(rng() % 3)));
            if (rng() % 8 == 0 && units.size() > 2) units[1] = units[2];  // an empty unit: refused
            std::vector<int32_t> ub(n + 2);
            int32_t nub = 0;
            cosine_blocking_units_host(n, rp.data(), ci.data(), Pr(rng), mb, (int32_t)units.size() - 1, units.data(),
                                       perm.data(), ub.data(), &nub, &err);
        }
        // analysis: validation, CSC copy and partition run on the host; the device upload that
        // follows fails where there is no GPU (or succeeds where there is one)
        {
            bilu_ctx ctx;
            bilu_params p{};
            p.blocking = (int32_t)(rng() % 2);
            p.max_block = mb;
            p.fixed_block = 1 + (int32_t)(rng() % mb);
            p.tau_analyze = 1e-2;
            p.perturb = 1;
            p.pert_tau = 1e-2;
            p.pert_rho = 1e-1;
            std::vector<int32_t> ci2(ci);
            std::vector<double> va2(va);
            const int corrupt = (int)(rng() % 6);
            if (corrupt == 1 && ci2.size() > 1) std::swap(ci2[0], ci2[1]);
            if (corrupt == 2 && !va2.empty()) va2[0] = std::numeric_limits<double>::quiet_NaN();
            if (corrupt == 3 && !ci2.empty()) ci2.back() = n + 3;
            if (corrupt == 4) {  // a caller's partition, merged or not
                std::vector<int32_t> g{0};
                while (g.back() < n) g.push_back(std::min(n, g.back() + 1 + (int)(rng() % mb)));
                analyze_run(&ctx, n, rp.data(), ci2.data(), va2.data(), 0, &p, g.data(), (int32_t)g.size() - 1);
            } else {
                analyze_run(&ctx, n, rp.data(), ci2.data(), va2.data(), 0, &p);
            }
            matrix_free(&ctx);
        }
        ++checked;
    }
    std::printf("ok %ld trials\n", checked);
    return 0;
}
