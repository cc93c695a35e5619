"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of the oracle, on the CPU: a wrong sign, a
transposed operand, a dropped term, an index off by one, a changed threshold, norm or
tie-break. It then runs the pin tests (the oracle against the paper and the mathematics)
against that copy, and at least one pin must fail. The unmodified copy must pass them all,
which shows that the harness itself works. The product library is not involved: the copy
holds only the oracle, the pin tests and the seeded input generators.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ["test_oracle.py", "test_partition_oracle.py", "test_block_check_oracle.py", "test_skip_oracle.py",
             "test_golden.py", "test_cosine_oracle.py", "test_mwm_oracle.py", "test_nd_oracle.py",
             "test_aggregation_oracle.py", "test_bildl_oracle.py", "test_sqmr_oracle.py", "test_sym_matching_oracle.py"]
ORACLE_FILES = ["__init__.py", "bilu_oracle.c", "bilu_oracle.h", "block_check.py", "skip_oracle.py",
                "cosine_oracle.py", "mwm_oracle.py", "nd_oracle.py"]

C, BCK, SKP, COS, MWM, ND = ("bilu_oracle.c", "block_check.py", "skip_oracle.py", "cosine_oracle.py", "mwm_oracle.py",
                             "nd_oracle.py")

# (name, file, fragment, replacement, which occurrence of the fragment: 1 = first)
MUTANTS = [
    # Crout block factorization (Algorithm 1 with blocks, Sec. 2.2)
    ("L-update sign", C, "TL.buf[(size_t)sl * b + (F->Ucol.a[q] - s0)] -= sum;",
     "TL.buf[(size_t)sl * b + (F->Ucol.a[q] - s0)] += sum;", 1),
    ("U-update sign", C, "TU.buf[(size_t)sl * b + (F->Lrow.a[p] - s0)] -= sum;",
     "TU.buf[(size_t)sl * b + (F->Lrow.a[p] - s0)] += sum;", 1),
    ("pivot rows miss L-side updates", C, "int64_t ps = lower_bound_i32(F->Lrow.a, F->Lptr[J], F->Lptr[J + 1], s0);",
     "int64_t ps = lower_bound_i32(F->Lrow.a, F->Lptr[J], F->Lptr[J + 1], s1);", 1),
    ("block row of A loses its first column", C, "if (j < s1) continue;", "if (j <= s1) continue;", 1),
    ("only the previous block produces updates", C, "if (t != last) { vi_push(&prodU[t], K); last = t; }",
     "if (t != last && t == K + 1) { vi_push(&prodU[t], K); last = t; }", 1),
    ("L scaling by D transposed", C, "s += trow[k] * D[k * b + c];", "s += trow[k] * D[c * b + k];", 1),
    ("U scaling by D transposed", C, "s += D[r * b + k] * tcol[k];", "s += D[k * b + r] * tcol[k];", 1),
    ("L kept at the threshold", C, "if (sqrt(nrm2) > droptol) {", "if (sqrt(nrm2) >= droptol) {", 1),
    ("U kept at the threshold", C, "if (sqrt(nrm2) > droptol) {", "if (sqrt(nrm2) >= droptol) {", 2),
    ("L max-norm", C, "nrm2 += s * s;", "nrm2 = fmax(nrm2, s * s);", 1),
    ("U max-norm", C, "nrm2 += s * s;", "nrm2 = fmax(nrm2, s * s);", 2),
    ("U-side updates skip the first column right of the block", C,
     "int64_t qs = lower_bound_i32(F->Ucol.a, F->Uptr[J], F->Uptr[J + 1], s1);",
     "int64_t qs = lower_bound_i32(F->Ucol.a, F->Uptr[J], F->Uptr[J + 1], s1 + 1);", 1),
    ("pivot tie takes the last row", C, "if (fabs(a[i * b + j]) > amax)", "if (fabs(a[i * b + j]) >= amax)", 1),
    ("row swap not recorded", C, "int32_t t = perm[j]; perm[j] = perm[p]; perm[p] = t;", "", 1),
    ("LU multipliers not divided by the pivot", C, "for (int i = j + 1; i < b; ++i) a[i * b + j] /= a[j * b + j];",
     "for (int i = j + 1; i < b; ++i) a[i * b + j] /= 1.0;", 1),
    ("inverse multiplies by the pivot", C, "y[i] /= lu[i * b + i];", "y[i] *= lu[i * b + i];", 1),
    # progressive aggregation (Sec. 3.5)
    ("merge test 1.3 mu", C, "return (5 * nu <= 6 * mu) || (nu <= mu + 2 * (p + q));",
     "return (10 * nu <= 13 * mu) || (nu <= mu + 2 * (p + q));", 1),
    ("merge test without the two-entry allowance", C, "return (5 * nu <= 6 * mu) || (nu <= mu + 2 * (p + q));",
     "return (5 * nu <= 6 * mu);", 1),
    ("mu misses the U rows of block k-1", C, "const int64_t mu = p * (p + r + s + rp + sp) + q * (q + t + tp);",
     "const int64_t mu = p * (p + r + s) + q * (q + t + tp);", 1),
    ("merged L rows keep L_{i,k-1} unchanged", C, "for (int64_t m = 0; m < q; ++m) acc -= lb[m] * L21[m * p + j];", "",
     1),
    ("merged U columns add L21 U with the wrong sign", C, "for (int64_t m = 0; m < p; ++m) acc += L21[i * p + m] * ua[m];",
     "for (int64_t m = 0; m < p; ++m) acc -= L21[i * p + m] * ua[m];", 1),
    ("merged inverse without the coupling term", C, "for (int64_t m = 0; m < q; ++m) acc += DU[i * q + m] * DL[m * p + j];",
     "", 1),
    ("merged pivot block with L21 and U12 swapped", C, "for (int64_t j = 0; j < q; ++j) Ph[i * w + p + j] = U12[i * q + j];",
     "for (int64_t j = 0; j < q; ++j) Ph[i * w + p + j] = L21[j * p + i];", 1),
    ("producer lists keep the void block", C, "if (tb != last) { fix_producers(&prodU[tb], k); last = tb; }", "", 1),
    ("merged producer read with its unmerged width", C,
     "int bJ = F->bstart[J + 1] - F->bstart[J]; /* a merged producer spans its void predecessor */",
     "int bJ = bstart[J + 1] - bstart[J];", 1),
    # BILDL, the symmetric variant (Sec. 4.2)
    ("bildl: pivot block mirrored from the upper triangle", C,
     "for (int c = r + 1; c < b; ++c) P[r * b + c] = P[c * b + r];",
     "for (int c = r + 1; c < b; ++c) P[c * b + r] = P[r * b + c];", 1),
    ("bildl: D_K symmetrised on one side only", C, "                    D[c * b + r] = v;\n", "", 1),
    ("bildl: U-breve column holds the normalised row", C,
     "memcpy(F->Uval.a + F->Uval.n, trow, (size_t)b * sizeof(double));",
     "memcpy(F->Uval.a + F->Uval.n, ell, (size_t)b * sizeof(double));", 1),
    ("bildl: breakdown perturbed off the diagonal", C, "if (sym) k = bad;", "", 1),
    # simplified QMR (Sec. 4.2)
    ("sqmr: alpha inverted", C, "double alpha = rho / sigma;", "double alpha = sigma / rho;", 1),
    ("sqmr: theta from the previous residual", C, "double theta1 = sqrt(dot(n, r, r)) / tau;",
     "double theta1 = sqrt(dot(n, t, t)) / tau;", 1),
    ("sqmr: d without the c^2 theta^2 term", C, "d[i] = c * c * theta * theta * d[i] + c * c * alpha * q[i];",
     "d[i] = c * c * alpha * q[i];", 1),
    ("sqmr: tau not damped by c", C, "tau = tau * theta1 * c;", "tau = tau * theta1;", 1),
    ("sqmr: beta inverted", C, "double beta = rho1 / rho;", "double beta = rho / rho1;", 1),
    ("sqmr: direction without the preconditioner", C, "for (int64_t i = 0; i < n; ++i) q[i] = u[i] + beta * q[i];",
     "for (int64_t i = 0; i < n; ++i) q[i] = r[i] + beta * q[i];", 1),
    ("sqmr: backward error without ||b||", C, "double den = anorm * xmax + bmax;", "double den = anorm * xmax;", 1),
    # perturbation (Sec. 3.6)
    ("sign(0) = -1", C, "return x >= 0.0 ? 1.0 : -1.0;", "return x > 0.0 ? 1.0 : -1.0;", 1),
    ("rho ignored", C, "return d * (1.0 + prho) + sgn_plus(d) * ptau * alpha;",
     "return d + sgn_plus(d) * ptau * alpha;", 1),
    ("zero rows not perturbed", C, "if (zero) { P[i * b + i] = perturbed(P[i * b + i], ptau, prho, alpha); ++count; }",
     "", 1),
    ("diagonal preference lost", C, "if (2.0 * fabs(P[bad * b + bad]) >= fabs(P[k * b + bad])) k = bad;",
     "if (fabs(P[bad * b + bad]) >= fabs(P[k * b + bad])) k = bad;", 1),
    # preconditioner application (Sec. 2.2)
    ("forward sweep sign", C, "y[F->Lrow.a[p]] -= s;", "y[F->Lrow.a[p]] += s;", 1),
    ("backward sweep sign", C, "t[i] -= ucol[i] * zj;", "t[i] += ucol[i] * zj;", 1),
    ("apply D transposed", C, "s += D[i * b + k] * t[k];", "s += D[k * b + i] * t[k];", 1),
    # GMRES (Sec. 4)
    ("Givens rotation sign", C, "H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c2;",
     "H[(i + 1) * m + j] = sn[i] * a + cs[i] * c2;", 1),
    ("Gram-Schmidt against the newest vector only", C, "for (int i = 0; i <= j; ++i) {",
     "for (int i = j; i <= j; ++i) {", 1),
    ("least squares without the diagonal of H", C, "y[i] = s / H[i * m + i];", "y[i] = s;", 1),
    ("Givens update of g sign", C, "g[j + 1] = -sn[j] * g[j];", "g[j + 1] = sn[j] * g[j];", 1),
    ("correction not preconditioned", C, "for (int64_t e = 0; e < n; ++e) x[e] += zt[e];",
     "for (int64_t e = 0; e < n; ++e) x[e] += w[e];", 1),
    ("stopping test not relative to ||b||", C, "if (fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;",
     "if (fabs(g[j + 1]) <= tol || hn == 0.0) break;", 1),
    # ILU(1,tau) blocking (Sec. 3.4)
    ("growth rule loses its second clause", C,
     "int accept = (3 * f2 <= 4 * scal2) || (f2 <= scal2 + 4 * l2);", "int accept = (3 * f2 <= 4 * scal2);", 1),
    ("scalar count without the diagonal", C, "scal += I->n + J->n + 1;", "scal += I->n + J->n;", 1),
    ("group joins beyond max_block", C, "if (l + gs > max_block) break;", "if (l + gs > max_block + 1) break;", 1),
    ("fill rows ignored", C, "if (fabs(c->val[f] * ajk) >= tau * fabs(ajj * akk) && stamp[i] != stampval) {",
     "if (0 && stamp[i] != stampval) {", 1),
    ("strict threshold on original entries", C,
     "if (i > k && fabs(c->val[e]) >= tau * fabs(akk) && stamp[i] != stampval) {",
     "if (i > k && fabs(c->val[e]) > tau * fabs(akk) && stamp[i] != stampval) {", 1),
    ("new rows all counted", C, "r2 += (inR[GI.a[t]] != blk && GI.a[t] >= end);", "r2 += 1;", 1),
    ("rows inside the block counted", C, "r2 += (R.a[t] >= end);", "r2 += (R.a[t] >= end - 1);", 1),
    ("rows of the candidate group counted", C, "r2 += (inR[GI.a[t]] != blk && GI.a[t] >= end);",
     "r2 += (inR[GI.a[t]] != blk);", 1),
    # single block step checker
    ("checker: L-side update sign", BCK, "t[uc[qs:qe] - s0] -= upd[a]", "t[uc[qs:qe] - s0] += upd[a]", 1),
    ("checker: U-side update sign", BCK, "t[lr[ps2:pe2] - s0] -= upd[:, a]", "t[lr[ps2:pe2] - s0] += upd[:, a]", 1),
    ("checker: pivot rows miss updates", BCK, "ps = np.searchsorted(lr, s0)", "ps = np.searchsorted(lr, s1)", 1),
    ("checker: L scaling by D transposed", BCK, ".reshape(-1, b) @ D if", ".reshape(-1, b) @ D.T if", 1),
    ("checker: U scaling by D transposed", BCK, "uh = (D @ Uc.T).T", "uh = (D.T @ Uc.T).T", 1),
    ("checker: D is the transposed inverse", BCK, "D = sla.lu_solve(sla.lu_factor(P), np.eye(b))",
     "D = np.linalg.inv(P).T", 1),
    ("checker: any flip accepted", BCK, "assert abs(nrm[k] - tau) <= flip_rtol * tau",
     "assert abs(nrm[k] - tau) <= 1e30 * tau", 1),
    # cosine blocking (Sec. 3.2)
    ("cosine: strict test", COS, "float(cnt) ** 2 >= (tau", "float(cnt) ** 2 > (tau", 1),
    ("cosine: excluded partners join", COS, "if placed[j] or skip[j] or bw + w[j] > max_block:",
     "if placed[j] or bw + w[j] > max_block:", 1),
    ("cosine: block one larger than max_block", COS, "if placed[j] or skip[j] or bw + w[j] > max_block:",
     "if placed[j] or skip[j] or bw + w[j] > max_block + 1:", 1),
    ("cosine: exclusion by rows only", COS, "return np.array([a or b for a, b in zip(r, c)], dtype=bool)",
     "return np.array([a for a, b in zip(r, c)], dtype=bool)", 1),
    ("cosine: three sigma", COS, "var4 = 4 * (n * S - nnz * nnz)", "var4 = 9 * (n * S - nnz * nnz)", 1),
    ("cosine: members in decreasing order", COS, "partners = sorted({j for k in rows[i] for j in cols[k] if j > i})",
     "partners = sorted({j for k in rows[i] for j in cols[k] if j > i}, reverse=True)", 1),
    ("cosine: test against the column count", COS, "(tau * len(rows[i])) * len(rows[j])",
     "(tau * len(rows[i])) * len(cols[j])", 1),
    # maximum weight matching with scaling (Sec. 3.1)
    ("matching: cost from the row maximum", MWM, "amax[j] = max(amax[j], abs(float(A.val[e])))",
     "amax[i] = max(amax[i], abs(float(A.val[e])))", 1),
    ("matching: cost sign", MWM, "C[i, j] = math.log(amax[j]) - math.log(a)", "C[i, j] = math.log(a) - math.log(amax[j])", 1),
    ("matching: greedy (no potentials on the path)", MWM, "d = dist[j] + C[i, k] - u[i] - v[k]",
     "d = C[i, k] - u[i] - v[k]", 1),
    ("matching: row potential not raised", MWM, "u[row_of[j]] += D - dist[j]", "u[row_of[j]] += 0.0", 1),
    ("matching: column potential sign", MWM, "v[j] -= D - dist[j]", "v[j] += D - dist[j]", 1),
    ("matching: start row potential", MWM, "u[s] += D", "u[s] += 0.0", 1),
    ("matching: left scaling inverted", MWM, "dl = np.array([math.exp(x) for x in u])",
     "dl = np.array([math.exp(-x) for x in u])", 1),
    ("matching: right scaling not normalised", MWM,
     "dr = np.array([math.exp(v[j]) / (amax[j] if amax[j] > 0 else 1.0) for j in range(A.n)])",
     "dr = np.array([math.exp(v[j]) for j in range(A.n)])", 1),
    # block nested dissection and elimination tree (Sec. 3.3)
    ("symmetric matching: singleton's diagonal ignored", MWM,
     "                score = _log(_abs_entry(A, cyc[s], cyc[s]))", "                score = 0.0", 1),
    ("symmetric matching: one-sided scaling", MWM, "    ds = np.sqrt(dl * dr)", "    ds = dl", 1),
    ("symmetric matching: units in cycle order", MWM, "    units.sort(key=lambda u: u[0])\n", "", 1),
    ("symmetric matching: odd cycle paired past the neighbour", MWM,
     "                units.append(sorted([cyc[t % k], cyc[(t + 1) % k]]))\n    units.sort",
     "                units.append(sorted([cyc[t % k], cyc[(t + 2) % k]]))\n    units.sort", 1),
    ("cosine units: the block's capacity ignored", COS, "if placed[j] or skip[j] or bw + w[j] > max_block:",
     "if placed[j] or skip[j]:", 1),
    ("cosine units: compressed row from the unit's first row only", COS,
     "cols = sorted({unit_of[int(c)] for i in range(ustart[p], ustart[p + 1])",
     "cols = sorted({unit_of[int(c)] for i in range(ustart[p], ustart[p] + 1)", 1),
    ("nd: separator is the first level", ND, "m = len(levels) // 2", "m = 1", 1),
    ("nd: separator ordered first", ND, "order += dissect(adj, first, leaf) + dissect(adj, second, leaf) + sorted(levels[m])",
     "order += sorted(levels[m]) + dissect(adj, first, leaf) + dissect(adj, second, leaf)", 1),
    ("nd: graph not symmetrised", ND, "                adj[L].add(K)\n", "", 1),
    ("nd: root not pseudo-peripheral", ND, "        if len(lv) <= len(levels):", "        if True:", 1),
    ("etree: no fill", ND, "            later[p] |= later[K] - {p}", "            pass", 1),
    ("etree: parent is the last later neighbour", ND, "            p = min(later[K])", "            p = max(later[K])", 1),
    # learned-skip features and classifier
    ("features: sum of products is the last one", SKP, "S += v", "S = v", 1),
    ("features: max is a sum", SKP, "M = max(M, v)", "M = M + v", 1),
    ("features: d from block K", SKP, "d = Dfro[K - 1] if K > 0", "d = Dfro[K] if K > 0", 1),
    ("features: 1-norm of A's part", SKP, "apart[i] += float(cval[e]) ** 2", "apart[i] += abs(float(cval[e]))", 1),
    ("features: position from s_{K-1}", SKP, "max(0, i - s1)", "max(0, i - s0)", 1),
    ("features: producer width not averaged", SKP, "(SB / C / 64.0) if C else 0.0", "(SB / 64.0) if C else 0.0", 1),
    ("features: Y norm is a max", SKP, "yf = float(np.sqrt(sum(Ynorms[k] ** 2 for k in ys_in)))",
     "yf = float(max(Ynorms[k] for k in ys_in))", 1),
    ("features: first row right of the block never a candidate", SKP, "cand.update(i for i in Xset if i >= s1)",
     "cand.update(i for i in Xset if i > s1)", 1),
    ("features: labels inverted", SKP, "ys.append(0.0 if i in kept else 1.0)", "ys.append(1.0 if i in kept else 0.0)", 1),
    ("classifier: no second ReLU", SKP, "h2 = np.maximum(a2, 0.0)", "h2 = a2", 1),
    ("classifier: normalisation multiplies", SKP, "/ p[\"std\"]", "* p[\"std\"]", 1),
    ("classifier: W2 transposed", SKP, "a2 = h1 @ p[\"W2\"].T + p[\"b2\"]", "a2 = h1 @ p[\"W2\"] + p[\"b2\"]", 1),
    ("classifier: b1 dropped", SKP, "a1 = xs @ p[\"W1\"].T + p[\"b1\"]", "a1 = xs @ p[\"W1\"].T", 1),
    ("classifier: gradient sign", SKP, "dz = (1.0 / (1.0 + np.exp(-z)) - y) / n", "dz = (y - 1.0 / (1.0 + np.exp(-z))) / n", 1),
    ("classifier: W2 gradient transposed", SKP, "g[\"W2\"] = da2.T @ h1", "g[\"W2\"] = h1.T @ da2", 1),
]


def _plant(text: str, old: str, new: str, nth: int) -> str:
    pos = -1
    for _ in range(nth):
        pos = text.find(old, pos + 1)
        if pos < 0:
            raise AssertionError(f"fragment not found (occurrence {nth}): {old!r}")
    return text[:pos] + new + text[pos + len(old):]


def _tree(dst: str, mutant) -> None:
    os.makedirs(os.path.join(dst, "oracle"))
    os.makedirs(os.path.join(dst, "tests"))
    os.makedirs(os.path.join(dst, "paper_1908_10169_gb300"))
    for f in ORACLE_FILES:
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    for f in PIN_TESTS + ["conftest.py"]:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    # the seeded input generators only (no arithmetic of the method, no library binding)
    shutil.copy(os.path.join(ROOT, "paper_1908_10169_gb300", "workloads.py"),
                os.path.join(dst, "paper_1908_10169_gb300", "workloads.py"))
    open(os.path.join(dst, "paper_1908_10169_gb300", "__init__.py"), "w").close()
    shutil.copy(os.path.join(ROOT, "pytest.ini"), os.path.join(dst, "pytest.ini"))
    if mutant is not None:
        _, fname, old, new, nth = mutant
        p = os.path.join(dst, "oracle", fname)
        text = open(p).read()
        open(p, "w").write(_plant(text, old, new, nth))


def _run(dst: str):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "tests"], cwd=dst, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def test_fragments_are_present():
    """Every planted mistake still finds the code it changes (the check fails loudly when the
    oracle is edited under it)."""
    for name, fname, old, new, nth in MUTANTS:
        text = open(os.path.join(ROOT, "oracle", fname)).read()
        _plant(text, old, new, nth)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    cases = [("unmodified", None)] + [(m[0], m) for m in MUTANTS]
    dirs = {}
    for i, (name, m) in enumerate(cases):
        d = str(tmp_path / f"m{i:02d}")
        _tree(d, m)
        dirs[name] = d
    workers = max(2, min(8, (os.cpu_count() or 2)))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        res = dict(zip(dirs, ex.map(_run, dirs.values())))
    rc0, out0 = res.pop("unmodified")
    assert rc0 == 0, f"the unmodified oracle copy fails its pins:\n{out0}"
    survived = [n for n, (rc, _) in res.items() if rc == 0]
    crashed = {n: (rc, out) for n, (rc, out) in res.items() if rc not in (0, 1)}
    assert not survived, f"planted mistakes that no pin catches: {survived}"
    assert not crashed, f"mutants that ended without a failing pin: {crashed}"
