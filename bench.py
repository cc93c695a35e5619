#!/usr/bin/env python
"""Benchmark: block ILU factorization + preconditioned GMRES(30) to relative residual 1e-8.

Workload: 3D convection-diffusion, 7-point first-order upwind stencil on a 64^3 interior grid
(n = 262,144, nnz = 1,810,432), diffusion coefficients log-uniform in [1e-3, 1e3] per node
(seed 1), |v| = 100 along (1,1,1), Dirichlet boundaries eliminated, b = A * ones, drop
tolerance 1e-2, diagonal blocks of 64 consecutive unknowns (one grid line), reordered by block
nested dissection (Sec. 3.3, host analysis outside the timed region), FP64, factored by the
tree schedule (CTA groups on independent subtrees of the block elimination tree).

One step = bilu_factor + gmres_solve (x0 = 0) through the C ABI, with the matrix and b
already resident on the GPU (bilu_analyze runs once, outside the timed region).  L2 is
flushed (512 MB write) before every timed step.  The JSON line also reports the end-to-end
time through the same API from pinned host buffers (analyze + factor + solve + copy of x),
the roofline of the dominant kernel, and the FP64 CPU oracle on the host.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Other lines (not the default): --precision fp32|bf16 (mixed-precision updates), --skip
bound|learned (norm-bound or learned candidate skip; learned trains its classifier first, on
200 generated 3D problems, untimed), --workload elasticity|laplace27x4 (the mixed-precision and
learned-skip configurations' matrices), --batch N (N uneven 2D / 3D systems in one launch and
one graph per GMRES cycle, sharded over the ranks under torchrun), --mwm / --blocking
cosine|cosine+ilu1t|ilu1t / --order nd (the host analysis of Sec. 3.1-3.4 before the factorization,
outside the timed region and inside the end-to-end time; --workload cd3d_rows_scrambled is the
benchmark matrix with its equations in random order, which needs --mwm), --aggregate N
(progressive aggregation up to N columns), --compare-fp64 (plain FP64 on the same matrix
beside the line), --droptol T, and the symmetric variant: --symmetric (BILDL + SQMR to the
backward error 1e-6, metric "BILDL factor+SQMR seconds") on --workload elasticity_shifted
(symmetric indefinite) or kkt (a saddle-point system, with --sym-mwm: the symmetrised matching
of Sec. 4.2 and blocks of whole pivot units, optionally their cosine blocking). Under torchrun the
single-matrix line runs one replica per rank; the reference arm runs on rank 0 only (with
--batch it times the oracle on every 16th system and scales by the batch's unknowns).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BILU factor+GMRES seconds to rel. residual 1e-8"
UNIT = "s"
METRIC_SYM = "BILDL factor+SQMR seconds to backward error 1e-6"
SQMR_TOL = 1e-6  # the paper's stop for SQMR (normwise backward error)
REF_BUDGET_S = 150.0  # the reference arm's timed steps: full oracle steps while they fit in this
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12  # nominal: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=["cd3d", "elasticity", "laplace27x4", "cd3d_rows_scrambled",
                                           "elasticity_shifted", "kkt"], default="cd3d",
                    help="cd3d: 3D upwind convection-diffusion (the benchmark); elasticity: Q1 3-dof/node "
                         "(mixed-precision configuration, --side 48 --block 63); laplace27x4: Q1 27-point, "
                         "4 dof/node (learned-skip evaluation, --side 64)")
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--block", type=int, default=64)
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16"], default="fp64")
    ap.add_argument("--skip", choices=["none", "bound", "learned"], default="none")
    ap.add_argument("--train-count", type=int, default=200,
                    help="learned skip: training problems (3D 7-point, sides 32..48, Peclet 1..1000)")
    ap.add_argument("--train-rate", type=float, default=0.05, help="learned skip: share of candidates recorded")
    ap.add_argument("--mwm", action="store_true",
                    help="maximum weight matching + scaling (Sec. 3.1) before the factorization (host)")
    ap.add_argument("--blocking", choices=["fixed", "ilu1t", "cosine", "cosine+ilu1t"], default="fixed",
                    help="fixed blocks of --block (default); the ILU(1,tau) guess (Sec. 3.4); cosine blocks "
                         "(Sec. 3.2), as they are or merged by the ILU(1,tau) rule")
    ap.add_argument("--order", choices=["natural", "nd"], default="nd",
                    help="nd (default): block nested dissection of the blocks (Sec. 3.3) before the factorization "
                         "(host analysis, outside the timed region); natural: the generator's order")
    ap.add_argument("--schedule", choices=["chain", "tree"], default="tree",
                    help="tree (default): CTA groups factor independent subtrees of the block elimination tree "
                         "(pays off with --order nd), the trunk on the whole GPU; chain: one block after another")
    ap.add_argument("--group-ctas", type=int, default=0, help="tree schedule: CTAs per group (0: library default)")
    ap.add_argument("--no-tensor", action="store_true",
                    help="bf16: compute the update tiles on the FP32 units instead of the tensor cores")
    ap.add_argument("--aggregate", type=int, default=0,
                    help="progressive aggregation (Sec. 3.5): merge consecutive blocks up to this size (0: off)")
    ap.add_argument("--batch", type=int, default=0,
                    help="factor + solve this many uneven 2D/3D matrices in one batched launch instead")
    ap.add_argument("--symmetric", action="store_true",
                    help="BILDL (incomplete block L D L^T, Sec. 4.2) solved by SQMR to the backward error "
                         "1e-6 instead of BILU + GMRES(30); needs a symmetric workload (elasticity_shifted)")
    ap.add_argument("--droptol", type=float, default=None, help="drop tolerance (default: the workload's)")
    ap.add_argument("--sym-mwm", action="store_true",
                    help="symmetric variant: the symmetrised matching of Sec. 4.2 (symmetric scaling, 1 x 1 / "
                         "2 x 2 pivot units kept inside the blocks; cosine blocking on the compressed units) "
                         "before the blocking and the ordering")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="also time plain FP64 factor + GMRES (no skip) on the same matrix, order and schedule, "
                         "and report the variant's speedup over it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_systems(sizes, world):
    """Independent systems of a batch over `world` ranks: largest first onto the rank with the
    least work so far (work estimate: the given sizes, e.g. nnz), ties to the lower rank.
    Deterministic; returns one ascending index list per rank."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def max_over_ranks(value, device):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args):
    """The matrix of a run: the 3D upwind convection-diffusion benchmark matrix (default), the Q1
    elasticity matrix of the mixed-precision configuration, or the 27-point 4-dof/node matrix
    the learned skip is evaluated on."""
    from paper_1908_10169_gb300 import workloads as W
    if args.workload == "elasticity":
        w = W.elasticity3d(side=args.side, seed=2, block=args.block)
    elif args.workload == "laplace27x4":
        w = W.laplace27_4dof(side=args.side, seed=3, block=args.block)
    if args.workload == "cd3d_rows_scrambled":
        w = W.rows_scrambled(W.cd3d(side=args.side, seed=1, block=args.block), seed=5)
    elif args.workload == "elasticity_shifted":
        w = W.elasticity3d_shifted(side=args.side, seed=2, block=args.block)
    elif args.workload == "kkt":
        w = W.kkt_elasticity(side=args.side, seed=2, block=args.block)
    else:
        w = W.cd3d(side=args.side, seed=1, block=args.block)
    if getattr(args, "droptol", None) is not None:
        w = dataclasses.replace(w, droptol=args.droptol)
    return w


class Prepared:
    """The system the factorization sees after the host analysis of Sec. 3.1-3.4, and the map
    of its solution back to the original unknowns."""

    def __init__(self, A, b, bstart, steps, maps):
        self.A, self.b, self.bstart, self.steps, self._maps = A, b, bstart, steps, maps

    def to_original(self, y):
        """x of A x = b from the solution y of the prepared system."""
        import numpy as np
        x = np.asarray(y, dtype=np.float64)
        for f in reversed(self._maps):
            x = f(x)
        return x


def preprocess(args, w):
    """Runs the library's host analysis calls the options ask for, in the paper's order:
    matching + scaling (A^ = D_l A D_r Pi, Sec. 3.1), cosine blocking (Q^T A Q, Sec. 3.2), block
    nested dissection (P^T A P, Sec. 3.3).  With no option it returns the workload unchanged
    (bstart None: fixed blocks of --block)."""
    import numpy as np

    import paper_1908_10169_gb300 as B
    from paper_1908_10169_gb300 import workloads as W
    A, b, bstart, steps, maps = w.A, w.b, None, [], []
    if getattr(args, "mwm", False):
        sigma, dl, dr = B.bilu_mwm(A.n, A.rowptr, A.colind, A.val)
        A = W.CSR(A.n, *B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, None, sigma, dl, dr))
        b = dl * b

        def unmatch(y, sigma=sigma, dr=dr):
            x = np.empty_like(y)
            x[sigma] = dr[sigma] * y
            return x
        maps.append(unmatch)
        steps.append("mwm")

    units = None
    if getattr(args, "sym_mwm", False):
        perm, ds, units = B.bilu_sym_mwm(A.n, A.rowptr, A.colind, A.val)
        A = W.CSR(A.n, *B.bilu_scale_permute_csr(A.n, A.rowptr, A.colind, A.val, perm, perm, ds, ds))
        b = (ds * b)[perm]

        def unsym(y, perm=perm, ds=ds):
            x = np.empty_like(y)
            x[perm] = ds[perm] * y
            return x
        maps.append(unsym)
        steps.append("sym_mwm")

    def sym_permute(perm):
        nonlocal A, b
        A = W.CSR(A.n, *B.bilu_permute_csr(A.n, A.rowptr, A.colind, A.val, perm))
        b = b[perm]

        def unpermute(y, perm=perm):
            x = np.empty_like(y)
            x[perm] = y
            return x
        maps.append(unpermute)

    blocking = getattr(args, "blocking", "fixed")
    if units is not None:  # blocks made of whole pivot units
        if blocking.startswith("cosine"):  # Sec. 4.2: cosine blocking of the compressed units
            perm, groups = B.bilu_cosine_blocking_units(A.n, A.rowptr, A.colind, units, 0.8, 64)
            sym_permute(perm)
            bstart = groups
            if blocking == "cosine+ilu1t":
                bstart = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, 1e-2, 64, groups)
            steps.append(blocking)
        elif blocking == "ilu1t":
            bstart = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, 1e-2, 64, units)
            steps.append("ilu1t")
        else:
            out = [0]
            for k in range(1, len(units)):
                if units[k] - out[-1] > args.block:
                    out.append(int(units[k - 1]))
            bstart = np.array(out + ([A.n] if out[-1] != A.n else []), dtype=np.int32)
    elif blocking.startswith("cosine"):
        perm, groups = B.bilu_cosine_blocking(A.n, A.rowptr, A.colind, 0.8, 64)
        sym_permute(perm)
        bstart = groups
        if blocking == "cosine+ilu1t":
            bstart = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, 1e-2, 64, groups)
        steps.append(blocking)
    elif blocking == "ilu1t":
        bstart = B.bilu_partition_ilu1t(A.n, A.rowptr, A.colind, A.val, 1e-2, 64)
        steps.append("ilu1t")
    if getattr(args, "order", "natural") == "nd":
        if bstart is None:
            bstart = np.append(np.arange(0, A.n, args.block), A.n).astype(np.int32)
        perm, bstart, _ = B.bilu_nd_order(A.n, A.rowptr, A.colind, bstart)
        sym_permute(perm)
        steps.append("nd")
    return Prepared(A, b, bstart, steps, maps)


def config(args, w, extra=None):
    blocking = getattr(args, "blocking", "fixed")
    c = {"workload": w.name, "n": w.A.n, "nnz": w.A.nnz, "droptol": w.droptol,
         "blocking": f"fixed {args.block}" if blocking == "fixed" else blocking, "gmres": f"GMRES({w.restart}) rtol {w.gmres_tol}, x0 = 0, b = A*1",
         "updates": getattr(args, "precision", "fp64"), "skip": getattr(args, "skip", "none"),
         "order": getattr(args, "order", "natural"), "schedule": getattr(args, "schedule", "chain"),
         "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{args.gpus}"}
    if getattr(args, "aggregate", 0):
        c["aggregate_max"] = args.aggregate
    if getattr(args, "symmetric", False):
        c["factorization"] = "BILDL (incomplete block L D L^T, symmetric variant)"
        c["gmres"] = f"none: SQMR to the normwise backward error {SQMR_TOL}, x0 = 0, b = A*1"
    if getattr(args, "precision", "fp64") == "bf16":
        c["update_tiles"] = "FP32 units" if getattr(args, "no_tensor", False) else "tensor cores (tcgen05, BF16 x BF16 -> FP32)"

    pre = [k for k, on in (("mwm", getattr(args, "mwm", False)), ("sym_mwm", getattr(args, "sym_mwm", False)),
                           ("nd", getattr(args, "order", "natural") == "nd")) if on]
    if pre or blocking != "fixed":
        c["host_analysis"] = pre + ([blocking] if blocking != "fixed" else [])
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bilu_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def load_traffic():
    """DRAM bytes per stored factor value from the committed ncu summary, per kernel, kept
    only while the kernel sources still hash to what was captured."""
    import hashlib
    out = {}
    try:
        data = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except Exception:
        return out
    for k, v in data.items():
        if not isinstance(v, dict) or "sources" not in v:
            continue
        h = hashlib.sha256()
        try:
            for f in v["sources"]:
                h.update(open(os.path.join(ROOT, f), "rb").read())
        except Exception:
            continue
        if h.hexdigest()[:16] == v.get("source_sha"):
            out[k] = v["bytes_per_factor_value"]
    return out


def fp64_gemm_tflops(dev, n=4096, reps=5):
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul, n^3 float64, 2 n^3 flops),
    the best of `reps` timed with CUDA events after a warm-up; context for the derived FP64 peak
    that the factor's roofline uses."""
    import torch
    try:
        a = torch.randn(n, n, dtype=torch.float64, device=dev)
        b = torch.randn(n, n, dtype=torch.float64, device=dev)
        torch.matmul(a, b)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    except Exception:
        return None


def oracle_step(w, bstart, symmetric=False):
    """One full step of the FP64 CPU oracle (single thread): factor + GMRES(30), or with
    symmetric BILDL + SQMR to the backward error SQMR_TOL."""
    import oracle as O
    t0 = time.perf_counter()
    F = O.bildl_factor(w.A, bstart, w.droptol) if symmetric else O.bilu_factor(w.A, bstart, w.droptol)
    t1 = time.perf_counter()
    if symmetric:
        r = O.sqmr(w.A, F, w.b, tol=SQMR_TOL, maxit=10000)
    else:
        r = O.gmres(w.A, F, w.b, tol=w.gmres_tol, restart=w.restart)
    t2 = time.perf_counter()
    F.free()
    return t2 - t0, t1 - t0, t2 - t1, r.iters


def cpu_desc():
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def batch_sample(count):
    """The batch systems the reference arm times: every 16th system of each kind (even index:
    2D 5-point, odd index: 3D 7-point), so that both kinds are in the sample."""
    evens, odds = list(range(0, count, 2)), list(range(1, count, 2))
    return {"2d": evens[::16], "3d": odds[::16]}


def run_reference_batch(args):
    """Reference arm of the batched line: the oracle (factor + GMRES) on a fixed sample of the
    batch's systems (every 16th system of each kind), each kind's time scaled to all systems of
    that kind by their number of unknowns (the oracle's time per system grows about linearly
    with n on these stencils, at a different rate for 2D and 3D)."""
    import numpy as np
    import oracle as O
    from paper_1908_10169_gb300 import workloads as W
    oracle_cores, model = cpu_desc()
    ws = W.cd_batch(count=args.batch, seed0=100)
    kinds = batch_sample(len(ws))
    sample = sorted(i for v in kinds.values() for i in v)
    small = W.cd3d(side=12, seed=1, block=12)
    for _ in range(args.warmup):
        oracle_step(small, O.partition_fixed(small.A.n, 12))
    n_all = sum(w.A.n for w in ws)
    n_sample = sum(ws[i].A.n for i in sample)
    scale = {}
    for k, idx in kinds.items():
        members = range(0, len(ws), 2) if k == "2d" else range(1, len(ws), 2)
        scale[k] = sum(ws[i].A.n for i in members) / max(1, sum(ws[i].A.n for i in idx))
    times = []
    for _ in range(args.steps):
        t = 0.0
        for k, idx in kinds.items():
            for i in idx:
                w = ws[i]
                if args.order == "nd":  # the same host analysis as the GPU arm (not timed)
                    pw = preprocess(argparse.Namespace(block=w.fixed_block, order="nd", mwm=False, blocking="fixed"), w)
                    t += oracle_step(dataclasses.replace(w, A=pw.A, b=np.ascontiguousarray(pw.b)), pw.bstart)[0] * scale[k]
                else:
                    t += oracle_step(w, O.partition_fixed(w.A.n, w.fixed_block))[0] * scale[k]
        times.append(t)
    v = sum(times) / len(times)
    line = {"impl": "reference", "metric": f"batched BILU factor+GMRES seconds for {len(ws)} systems to rel. residual 1e-8",
            "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"cd_batch_{len(ws)}", "sum_n": int(n_all), "sample_systems": sample,
                       "sample_by_kind": kinds, "order": args.order},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"oracle factor + GMRES on systems {sample} ({n_sample} of {n_all} unknowns; "
                                       f"2D {kinds['2d']}, 3D {kinds['3d']}), each kind scaled by its unknowns to "
                                       f"all systems of that kind; host {model}, {oracle_cores} cores visible, 1 used"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if getattr(args, "batch", 0):
        return run_reference_batch(args)
    import oracle as O
    oracle_cores, model = cpu_desc()
    w = workload(args)
    # the options' host analysis prepares the input (library calls, not timed); the oracle's
    # factor + GMRES on the prepared system is what is timed
    prep = preprocess(args, w)
    bs = prep.bstart if prep.bstart is not None else O.partition_fixed(w.A.n, args.block)
    w = dataclasses.replace(w, A=prep.A, b=prep.b)
    sargs = argparse.Namespace(**{**vars(args), "side": 16, "block": 16})
    small = workload(sargs)
    sprep = preprocess(sargs, small)
    small = dataclasses.replace(small, A=sprep.A, b=sprep.b)
    for _ in range(args.warmup):  # warm-up on a small case of the same kind
        oracle_step(small, sprep.bstart if sprep.bstart is not None else O.partition_fixed(small.A.n, 16),
                    args.symmetric)
    # one full step on the workload itself (the last warm-up step); when K of them would take
    # longer than REF_BUDGET_S, every timed step is a bounded sample instead: the oracle's full
    # step on the same kind of problem with 3/4 of the side, scaled by the ratio of the two
    # measured once here
    t_full, _, _, iters = oracle_step(w, bs, args.symmetric)
    sample_note = ("full step (oracle factor + " + ("SQMR" if args.symmetric else "GMRES") +
                   ", FP64 arithmetic, every candidate computed) on the same matrix")
    times = []
    if t_full * args.steps <= REF_BUDGET_S:
        times.append(t_full)
        for _ in range(args.steps - 1):
            t, tf, tg, iters = oracle_step(w, bs, args.symmetric)
            times.append(t)
        times = times[:args.steps]
    else:
        side_s = max(8, (3 * args.side) // 4)
        sa = argparse.Namespace(**{**vars(args), "side": side_s})
        ws_ = workload(sa)
        sp_ = preprocess(sa, ws_)
        ws_ = dataclasses.replace(ws_, A=sp_.A, b=sp_.b)
        bs_ = sp_.bstart if sp_.bstart is not None else O.partition_fixed(ws_.A.n, args.block)
        t_cal = oracle_step(ws_, bs_, args.symmetric)[0]
        for _ in range(args.steps):
            times.append(oracle_step(ws_, bs_, args.symmetric)[0] * t_full / t_cal)
        sample_note = (f"each timed step: the oracle's full step (factor + GMRES, FP64) on the {side_s}^3 problem of "
                       f"the same kind and host analysis, scaled by t({args.side}^3) / t({side_s}^3) = "
                       f"{t_full:.2f} s / {t_cal:.2f} s, both measured once before the timed steps (a full step on "
                       f"the workload takes {t_full:.1f} s, {args.steps} of them would exceed {REF_BUDGET_S:.0f} s)")
    v = sum(times) / len(times)
    line = {"impl": "reference", "metric": METRIC_SYM if args.symmetric else METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, w, {"gmres_iters": iters}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample_note}; host {model}, {oracle_cores} cores visible, 1 used"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    import paper_1908_10169_gb300 as B

    if args.skip == "learned" and args.schedule == "tree":
        args.schedule = "chain"  # the learned skip reads the previous block's inverse: chain schedule only

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args)
    stream = torch.cuda.Stream(device=dev)
    ctx = B.bilu_create(local, stream)
    if args.no_tensor:
        B.bilu_debug_set(ctx, B.BILU_DEBUG_NO_TENSOR, 1)
    params = B.bilu_params_default(blocking=B.BILU_BLOCKING_FIXED, fixed_block=args.block, max_block=64,
                                   precision={"fp64": B.BILU_PREC_FP64, "fp32": B.BILU_PREC_FP32,
                                              "bf16": B.BILU_PREC_BF16}[args.precision],
                                   skip={"none": B.BILU_SKIP_NONE, "bound": B.BILU_SKIP_BOUND,
                                         "learned": B.BILU_SKIP_LEARNED}[args.skip],
                                   schedule={"chain": B.BILU_SCHED_CHAIN, "tree": B.BILU_SCHED_TREE}[args.schedule],
                                   group_ctas=args.group_ctas, aggregate_max=args.aggregate,
                                   symmetric=1 if args.symmetric else 0)
    learned = None
    if args.skip == "learned":  # train the classifier first (not timed)
        from paper_1908_10169_gb300 import learned_skip as LS
        from paper_1908_10169_gb300 import workloads as W
        t0 = time.time()
        xs, ys = LS.record(W.cd3d_skip_train(count=args.train_count), device=local, rate=args.train_rate)
        t1 = time.time()
        sm = LS.train(xs, ys, device=local, epochs=4, batch=4096, lr=2e-3, seed=1, max_false_drop=2e-3)
        learned = {"train_problems": args.train_count, "samples": sm.samples, "drop_fraction": sm.drop_fraction,
                   "train_loss": sm.train_loss, "logit_hi": sm.logit_hi, "train_skip_rate": sm.skip_rate,
                   "train_false_drop_rate": sm.false_drop_rate, "record_s": t1 - t0, "train_s": time.time() - t1}
        B.bilu_set_skip_model(ctx, sm.model, sm.logit_hi)
    prep = preprocess(args, w)  # host analysis of Sec. 3.1-3.3 when asked for (outside the timed region)
    rp = torch.from_numpy(prep.A.rowptr.astype(np.int64)).to(dev)
    ci = torch.from_numpy(prep.A.colind.astype(np.int32)).to(dev)
    va = torch.from_numpy(prep.A.val).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(prep.b)).to(dev)
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    if prep.bstart is None:
        B.bilu_analyze(ctx, w.A.n, rp, ci, va, params)
    else:
        B.bilu_analyze_partition(ctx, w.A.n, rp, ci, va, prep.bstart, params)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def solve(c_, b_, x_):
        if args.symmetric:
            return B.sqmr_solve(c_, b_, x_, SQMR_TOL, 10000)
        return B.gmres_solve(c_, b_, x_, w.gmres_tol, w.restart, 10000)

    def step():
        B.bilu_factor(ctx, w.droptol)
        with torch.cuda.stream(stream):
            x.zero_()
        return solve(ctx, b, x)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    s0 = B.bilu_stats(ctx)
    launches0 = s0.kernel_launches
    times, tf, ts, infos = [], [], [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            stream.synchronize()
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1))
            st = B.bilu_stats(ctx)
            tf.append(st.t_factor_ms)
            ts.append(info.t_solve_ms)
            infos.append((info.iters, getattr(info, "restarts", 0), info.relres_true))
    st = B.bilu_stats(ctx)
    launches = (st.kernel_launches - launches0) / args.steps
    ms = sum(times) / len(times)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    iters, restarts, relres = infos[-1]

    # live kernel timings for the roofline: the factor kernel (library events) and one apply
    t_factor = statistics.median(tf)
    r = torch.randn(w.A.n, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    for _ in range(3):
        B.bilu_apply(ctx, r, z)
    napply = 20
    with torch.cuda.stream(stream):
        flush.fill_(2)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(napply):
        B.bilu_apply(ctx, r, z)
    a1.record(stream)
    a1.synchronize()
    t_apply = a0.elapsed_time(a1) / napply
    n = w.A.n
    vbytes = {"fp64": 8, "fp32": 4, "bf16": 2}[args.precision]
    apply_bytes = vbytes * (st.nnz_l + st.nnz_u) + 8 * st.nnz_d + 4 * (st.kept_rows + st.kept_cols) + 8 * 3 * n
    factor_tf = st.flops_factor / (t_factor * 1e-3) / 1e12
    apply_gbs = apply_bytes / (t_apply * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    fp64_meas = fp64_gemm_tflops(dev)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # GMRES: one per Arnoldi step, one per cycle for x; SQMR: one per step and one at the start
    applies_per_step = iters + (1 if args.symmetric else restarts)
    share_factor = t_factor / ms
    share_apply = applies_per_step * t_apply / ms
    traffic = load_traffic()
    nvals = st.nnz_l + st.nnz_u + st.nnz_d
    kname = "bilu_factor_tree_kernel" if args.schedule == "tree" else "bilu_factor_kernel"
    roof_factor = {"kernel": kname, "bound": "alu", "achieved": factor_tf,
                   "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": factor_tf / FP64_PEAK_TFLOPS,
                   "peak_source": "derived FP64 DFMA peak (152 SMs x 4 flop/clk x 2070 MHz)",
                   "peak_measured_fp64_gemm": fp64_meas,
                   "frac_of_measured_fp64_gemm": factor_tf / fp64_meas if fp64_meas else None,
                   "traffic": (traffic[kname] * nvals) if kname in traffic else None,
                   "traffic_source": "ncu dram bytes per stored factor value on 48^3 (profiles/), scaled",
                   "flops_per_launch": st.flops_factor, "ms_per_launch": t_factor, "share_of_step": share_factor}
    roof_apply = {"kernel": "apply_forward_kernel+apply_backward_kernel", "bound": "hbm", "achieved": apply_gbs,
                  "peak": hbm_peak, "unit": "GB/s", "frac": apply_gbs / hbm_peak, "peak_source": hbm_src,
                  "traffic": ((traffic["apply_forward_kernel"] + traffic["apply_backward_kernel"]) * nvals
                              if "apply_forward_kernel" in traffic and "apply_backward_kernel" in traffic else None),
                  "traffic_note": "forward + backward sweep",
                  "bytes_per_launch": apply_bytes, "ms_per_launch": t_apply, "share_of_step": share_apply}
    dominant, other = (roof_factor, roof_apply) if share_factor >= share_apply else (roof_apply, roof_factor)
    if args.precision == "bf16" and not args.no_tensor and args.skip == "none":
        # the Schur updates of the candidate tiles run on the tensor cores: their algorithmic
        # flops (the pivot-row tiles, on the FP32 units, are a small part) over the factor time,
        # against the measured dense BF16 rate (a lower bound of the pipe's use while it runs)
        upd = st.flop_upd_l + st.flop_upd_u
        pk = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
        ach = upd / (t_factor * 1e-3) / 1e12
        other = dict(other, tensor_updates={"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                                            "frac": ach / pk, "peak_source": "measured bf16 (sustained)",
                                            "flops_per_launch": upd, "ms_per_launch": t_factor})

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_rp = torch.from_numpy(w.A.rowptr.astype(np.int64)).pin_memory()
        h_ci = torch.from_numpy(w.A.colind.astype(np.int32)).pin_memory()
        h_va = torch.from_numpy(w.A.val).pin_memory()
        h_b = torch.from_numpy(w.b).pin_memory()
        h_x = torch.zeros(n, dtype=torch.float64).pin_memory()
        ctx2 = B.bilu_create(local, stream)
        if learned is not None:
            B.bilu_set_skip_model(ctx2, sm.model, sm.logit_hi)
        et = []
        for k in range(min(args.steps, 3) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if prep.steps:  # the host analysis is part of the end-to-end path
                p2 = preprocess(args, w)
                hb = torch.from_numpy(np.ascontiguousarray(p2.b))
                if p2.bstart is None:
                    B.bilu_analyze(ctx2, n, p2.A.rowptr, p2.A.colind, p2.A.val, params)
                else:
                    B.bilu_analyze_partition(ctx2, n, p2.A.rowptr, p2.A.colind, p2.A.val, p2.bstart, params)
                B.bilu_factor(ctx2, w.droptol)
                h_x.zero_()
                solve(ctx2, hb, h_x)
                p2.to_original(h_x.numpy())
            else:
                B.bilu_analyze(ctx2, n, h_rp, h_ci, h_va, params)
                B.bilu_factor(ctx2, w.droptol)
                h_x.zero_()
                solve(ctx2, h_b, h_x)
            torch.cuda.synchronize()
            if k > 0:
                et.append(time.perf_counter() - t0)
        B.bilu_destroy(ctx2)
        bi = 8 * (n + 1) + 4 * w.A.nnz + 8 * w.A.nnz + 8 * n
        e2e = {"value": sum(et) / len(et), "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": 8 * n}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        cores, model = cpu_desc()
        wp = dataclasses.replace(w, A=prep.A, b=prep.b)
        t, tfo, tgo, it_o = oracle_step(wp, prep.bstart if prep.bstart is not None else O.partition_fixed(n, args.block),
                                        args.symmetric)
        cpu = {"value": t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full step (oracle factor {tfo:.1f} s + {'SQMR' if args.symmetric else 'GMRES'} "
                         f"{tgo:.1f} s, {it_o} iters) on the "
                         f"same matrix; host {model}, {cores} cores visible, 1 used",
               "gmres_iters": it_o}
    plain = None
    if args.compare_fp64:  # plain FP64 (no skip) on the same matrix, order and schedule, same timing
        ctx4 = B.bilu_create(local, stream)
        p4 = B.bilu_params_default(blocking=B.BILU_BLOCKING_FIXED, fixed_block=args.block, max_block=64,
                                   schedule=params.schedule, group_ctas=args.group_ctas)
        if prep.bstart is None:
            B.bilu_analyze(ctx4, w.A.n, rp, ci, va, p4)
        else:
            B.bilu_analyze_partition(ctx4, w.A.n, rp, ci, va, prep.bstart, p4)
        pt = []
        for k in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            torch.cuda.synchronize()
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            B.bilu_factor(ctx4, w.droptol)
            with torch.cuda.stream(stream):
                x.zero_()
            i4 = B.gmres_solve(ctx4, b, x, w.gmres_tol, w.restart, 10000)
            q1.record(stream)
            q1.synchronize()
            if k >= args.warmup:
                pt.append(q0.elapsed_time(q1))
        s4 = B.bilu_stats(ctx4)
        pms = sum(pt) / len(pt)
        plain = {"ms_per_step": pms, "factor_ms": s4.t_factor_ms, "solve_ms": i4.t_solve_ms, "gmres_iters": i4.iters,
                 "schedule": "tree" if p4.schedule == B.BILU_SCHED_TREE else "chain",
                 "method": "BILU + GMRES(30), rel. residual %g" % w.gmres_tol,
                 "speedup_of_this_line": pms / ms, "factor_speedup": s4.t_factor_ms / t_factor,
                 "iters_ratio": iters / max(1, i4.iters)}
        B.bilu_destroy(ctx4)
    if learned is not None:  # the method without the skip on the same matrix, for the gain
        learned.update({"skipped": st.skipped_rows + st.skipped_cols, "candidates": st.cand_rows + st.cand_cols,
                        "kept": st.kept_rows + st.kept_cols, "flops_factor": st.flops_factor})
        ctx3 = B.bilu_create(local, stream)
        params.skip = B.BILU_SKIP_NONE
        if prep.bstart is None:
            B.bilu_analyze(ctx3, w.A.n, rp, ci, va, params)
        else:
            B.bilu_analyze_partition(ctx3, w.A.n, rp, ci, va, prep.bstart, params)
        for _ in range(2):
            B.bilu_factor(ctx3, w.droptol)
        s3 = B.bilu_stats(ctx3)
        with torch.cuda.stream(stream):
            x.zero_()
        i3 = B.gmres_solve(ctx3, b, x, w.gmres_tol, w.restart, 10000)
        learned.update({"exact_factor_ms": s3.t_factor_ms, "exact_flops_factor": s3.flops_factor,
                        "exact_kept": s3.kept_rows + s3.kept_cols, "exact_gmres_iters": i3.iters,
                        "exact_solve_ms": i3.t_solve_ms})
        B.bilu_destroy(ctx3)
        # the exact skip (the norm bound: the same factor as no skip) on the same schedule
        ctx5 = B.bilu_create(local, stream)
        params.skip = B.BILU_SKIP_BOUND
        if prep.bstart is None:
            B.bilu_analyze(ctx5, w.A.n, rp, ci, va, params)
        else:
            B.bilu_analyze_partition(ctx5, w.A.n, rp, ci, va, prep.bstart, params)
        for _ in range(2):
            B.bilu_factor(ctx5, w.droptol)
        s5 = B.bilu_stats(ctx5)
        with torch.cuda.stream(stream):
            x.zero_()
        i5 = B.gmres_solve(ctx5, b, x, w.gmres_tol, w.restart, 10000)
        learned.update({"bound_factor_ms": s5.t_factor_ms, "bound_flops_factor": s5.flops_factor,
                        "bound_kept": s5.kept_rows + s5.kept_cols, "bound_gmres_iters": i5.iters,
                        "bound_solve_ms": i5.t_solve_ms, "bound_skipped": s5.skipped_rows + s5.skipped_cols})
        B.bilu_destroy(ctx5)
        params.skip = B.BILU_SKIP_LEARNED
    B.bilu_destroy(ctx)
    if rank == 0:
        line = {"metric": METRIC_SYM if args.symmetric else METRIC, "value": ms / 1e3 / world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32+f64", "bf16": "bf16+f32+f64"}[args.precision],
                "data": "synthetic",
                "config": config(args, w, {"gmres_iters": iters, "gmres_restarts": restarts,
                                           "relres_true": relres, "factor_ms": t_factor,
                                           "solve_ms": statistics.median(ts), "apply_ms": t_apply,
                                           "fill_nnz(L+U+D)/nnz(A)": (st.nnz_l + st.nnz_u + st.nnz_d) / w.A.nnz,
                                           "nblocks": st.nblocks, "bound_drops": st.bound_drops,
                                           "block_size": {"avg": st.avg_bsize, "max": st.max_bsize},
                                           **({"aggregation": {"merges": st.agg_merges,
                                                               "blocks_after": st.nblocks - st.agg_merges,
                                                               "max_block_after": st.agg_max_bsize,
                                                               "ms": st.t_aggregate_ms}}
                                              if args.aggregate else {}),
                                           **({"tree": {"height": st.tree_height, "trunk_blocks": st.tree_trunk,
                                                        "group_ctas": st.group_ctas,
                                                        "groups": (torch.cuda.get_device_properties(dev).multi_processor_count
                                                                   // max(1, st.group_ctas)),
                                                        "idle_ms_summed": round(st.idle_ms, 3)}}
                                              if args.schedule == "tree" else {}),
                                           "factor_phase_ms": dict(zip(["candidates", "pivot_rows+lu", "inverse",
                                                                        "bound_skip_updates", "scale_drop", "compact",
                                                                        "cta0_lu_work", "cta0_pivot_tile_wait"],
                                                                       [round(v, 3) for v in st.phase_ms])),
                                           **({"learned_skip": learned} if learned is not None else {}),
                                           **({"plain_fp64": plain} if plain is not None else {})}),
                "roofline": dominant, "roofline_other": other,
                "gpu_launches": launches, "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Batched workload: `args.batch` uneven convection-diffusion matrices (2D 5-point and 3D
    7-point, n log-uniform in [1e4, 2e5]) factored in one persistent launch and solved with one
    graph per restart cycle; compared with factoring and solving them one by one."""
    import numpy as np
    import torch

    import paper_1908_10169_gb300 as B
    from paper_1908_10169_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:  # the systems are independent: each rank takes a share, no data-path collective
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    t_start = time.time()

    def progress(msg):
        print(f"[batch {time.time() - t_start:7.1f} s] {msg}", file=sys.stderr, flush=True)

    ws_all = W.cd_batch(count=args.batch, seed0=100)
    mine = shard_systems([w.A.nnz for w in ws_all], world)[rank]
    ws = [ws_all[i] for i in mine]
    prec = {"fp64": B.BILU_PREC_FP64, "fp32": B.BILU_PREC_FP32, "bf16": B.BILU_PREC_BF16}[args.precision]
    stream = torch.cuda.Stream(device=dev)
    skip = {"none": B.BILU_SKIP_NONE, "bound": B.BILU_SKIP_BOUND, "learned": B.BILU_SKIP_LEARNED}[args.skip]
    learned = None
    if args.skip == "learned":  # train the classifier first (not timed)
        from paper_1908_10169_gb300 import learned_skip as LS
        xtr, ytr = LS.record(W.cd3d_skip_train(count=args.train_count), device=local, rate=args.train_rate)
        sm = LS.train(xtr, ytr, device=local, epochs=4, batch=4096, lr=2e-3, seed=1, max_false_drop=2e-3)
        learned = {"train_problems": args.train_count, "samples": sm.samples, "logit_hi": sm.logit_hi,
                   "train_skip_rate": sm.skip_rate}
        progress(f"classifier trained on {sm.samples} samples")
    # each system as the factor sees it: with --order nd its blocks reordered by nested dissection
    # (host analysis, not timed), else as generated
    prepared = []
    for w in ws:
        if args.order == "nd":
            pw = preprocess(argparse.Namespace(block=w.fixed_block, order="nd", mwm=False, blocking="fixed"), w)
            prepared.append((pw.A, np.ascontiguousarray(pw.b), pw.bstart))
        else:
            prepared.append((w.A, w.b, None))

    def analyze(c, A, bst, params):
        t = [torch.from_numpy(v).to(dev) for v in (A.rowptr, A.colind, A.val)]
        if bst is None:
            B.bilu_analyze(c, A.n, *t, params)
        else:
            B.bilu_analyze_partition(c, A.n, *t, bst, params)

    ctxs, bs, xs = [], [], []
    for w, (Aw, bw, bst) in zip(ws, prepared):
        c = B.bilu_create(local, stream if not ctxs else None)
        analyze(c, Aw, bst, B.bilu_params_default(fixed_block=w.fixed_block, max_block=64, precision=prec, skip=skip))
        if learned is not None:
            B.bilu_set_skip_model(c, sm.model, sm.logit_hi)
        ctxs.append(c)
        bs.append(torch.from_numpy(bw).to(dev))
        xs.append(torch.zeros(w.A.n, dtype=torch.float64, device=dev))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    progress(f"{len(ws)} systems analysed")

    def step():
        B.bilu_factor_batch(ctxs, 1e-2)
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        return B.gmres_solve_batch(ctxs, bs, xs, 1e-8, 30, 10000)

    for k in range(max(3, args.warmup)):  # the group size is tuned on the second call
        infos = step()
        progress(f"warm-up step {k} done, GMRES iterations max {max(i.iters for i in infos)}")
    l0 = sum(B.bilu_stats(c).kernel_launches for c in ctxs)
    times = []
    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = step()
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(max_over_ranks(e0.elapsed_time(e1), dev))
            progress(f"timed step: {times[-1]:.1f} ms")
    launches = (sum(B.bilu_stats(c).kernel_launches for c in ctxs) - l0) / args.steps
    batch_factor_ms, batch_gmres_ms = B.bilu_stats(ctxs[0]).t_factor_ms, infos[0].t_solve_ms
    if learned is not None:
        learned.update({"skipped": sum(B.bilu_stats(c).skipped_rows + B.bilu_stats(c).skipped_cols for c in ctxs),
                        "candidates": sum(B.bilu_stats(c).cand_rows + B.bilu_stats(c).cand_cols for c in ctxs)})
    ms = sum(times) / len(times)
    iters_b = [i.iters for i in infos]
    # the same systems one by one, plain FP64
    t_seq, iters_s = 0.0, []
    one = B.bilu_create(local, stream)
    for w, bvec, (Aw, bw, bst) in zip(ws, bs, prepared):
        # one by one: plain FP64 on the same ordering, with the single-matrix schedule of that ordering
        analyze(one, Aw, bst, B.bilu_params_default(fixed_block=w.fixed_block, max_block=64,
                                                    schedule=B.BILU_SCHED_TREE if bst is not None else B.BILU_SCHED_CHAIN))
        x = torch.zeros_like(bvec)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bilu_factor(one, 1e-2)
        iters_s.append(B.gmres_solve(one, bvec, x, 1e-8, 30, 10000).iters)
        e1.record(stream)
        torch.cuda.synchronize()
        t_seq += e0.elapsed_time(e1)
        progress(f"one by one: {w.name} {e0.elapsed_time(e1):.1f} ms")
    B.bilu_destroy(one)
    for c in ctxs:
        B.bilu_destroy(c)
    # job totals: one by one the whole batch runs serially (the ranks' shares add up)
    ratio = max_over_ranks(max(a / max(1, b2) for a, b2 in zip(iters_b, iters_s)), dev)
    t_seq_all = t_seq
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_seq, launches], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        t_seq_all, launches = float(tt[0].item()), float(tt[1].item())
    if rank == 0:
        line = {"metric": f"batched BILU factor+GMRES seconds for {len(ws_all)} systems to rel. residual 1e-8",
                "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32+f64", "bf16": "bf16+f32+f64"}[args.precision],
                "data": "synthetic",
                "config": {"workload": f"cd_batch_{len(ws_all)}", "sum_n": int(sum(w.A.n for w in ws_all)),
                           "n_range": [int(min(w.A.n for w in ws_all)), int(max(w.A.n for w in ws_all))],
                           "parallelism": f"systems sharded over {world} GPU(s) by nnz, no collective",
                           "order": args.order,
                           "systems_on_rank0": len(ws), "updates": args.precision,
                           "gmres_iters_batched_rank0": iters_b, "gmres_iters_plain_fp64_rank0": iters_s,
                           "max_iter_ratio": ratio,
                           "plain_fp64_one_by_one_s": t_seq_all / 1e3,
                           "speedup_vs_plain_one_by_one": t_seq_all / ms,
                           "l2": "flushed (512 MB write) before every timed step", "skip": args.skip,
                           "batch_factor_ms_rank0": batch_factor_ms, "batch_gmres_ms_rank0": batch_gmres_ms,
                           **({"learned_skip": learned} if learned is not None else {})},
                "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.symmetric and args.workload not in ("elasticity_shifted", "kkt"):
        raise SystemExit("--symmetric needs a symmetric workload: --workload elasticity_shifted")
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
