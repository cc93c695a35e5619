"""bench.py's contract on CPU: the reference arm (the timed oracle) prints one JSON line with
the keys the harness reads, and the argument defaults give a short N = 1 run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--side", "10",
                          "--block", "10", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["gmres_iters"] > 0


def test_argument_defaults():
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = old
    assert a.gpus == 1 and a.impl == "gpu" and a.warmup >= 3 and 1 <= a.steps <= 10
    assert a.side == 64 and a.block == 64 and a.workload == "cd3d" and a.precision == "fp64"


def _args(**kw):
    import argparse
    base = dict(side=8, block=8, workload="cd3d", mwm=False, blocking="fixed", order="natural", sym_mwm=False,
                droptol=None)
    base.update(kw)
    return argparse.Namespace(**base)


import pytest  # noqa: E402


@pytest.mark.parametrize("kw", [
    {},
    {"order": "nd"},
    {"blocking": "cosine"},
    {"blocking": "cosine+ilu1t", "workload": "elasticity", "side": 3, "block": 9},
    {"blocking": "ilu1t", "order": "nd"},
    {"workload": "cd3d_rows_scrambled", "mwm": True},
    {"workload": "cd3d_rows_scrambled", "mwm": True, "order": "nd"},
    {"workload": "kkt", "sym_mwm": True, "side": 4, "block": 24},
    {"workload": "kkt", "sym_mwm": True, "order": "nd", "side": 4, "block": 24},
    {"workload": "kkt", "sym_mwm": True, "blocking": "ilu1t", "side": 4, "block": 24},
    {"workload": "kkt", "sym_mwm": True, "blocking": "cosine+ilu1t", "order": "nd", "side": 4, "block": 24},
])
def test_preprocessed_system_maps_back(kw):
    """The prepared system (matching, cosine blocking, ILU(1,tau), nested dissection as
    asked), solved exactly and mapped back, solves the original A x = b; its partition is
    valid and the default leaves the workload untouched."""
    import numpy as np
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    sys.path.insert(0, ROOT)
    import bench
    args = _args(**kw)
    w = bench.workload(args)
    prep = bench.preprocess(args, w)
    if not kw:
        assert prep.A is w.A and prep.bstart is None and not prep.steps
    Ap = sp.csr_matrix((prep.A.val, prep.A.colind, prep.A.rowptr), shape=(w.A.n, w.A.n)).tocsc()
    y = spla.spsolve(Ap, prep.b)
    x = prep.to_original(y)
    A0 = sp.csr_matrix((w.A.val, w.A.colind, w.A.rowptr), shape=(w.A.n, w.A.n))
    assert np.linalg.norm(A0 @ x - w.b) <= 1e-9 * np.linalg.norm(w.b)
    if prep.bstart is not None:
        bs = np.asarray(prep.bstart)
        assert bs[0] == 0 and bs[-1] == w.A.n and np.all(np.diff(bs) >= 1) and np.diff(bs).max() <= 64
    if kw.get("mwm"):
        assert np.allclose(np.abs(Ap.diagonal()), 1.0, atol=1e-12)
    if kw.get("sym_mwm"):  # symmetric bit for bit, |a^| <= 1, no block splits a 2 x 2 unit
        assert (Ap != Ap.T).nnz == 0 and np.abs(Ap.data).max() <= 1 + 1e-12
        assert prep.bstart is not None
        import paper_1908_10169_gb300 as B
        perm, ds, units = B.bilu_sym_mwm(w.A.n, w.A.rowptr, w.A.colind, w.A.val)
        if kw.get("order") != "nd" and not kw.get("blocking", "fixed").startswith("cosine"):
            assert set(np.asarray(prep.bstart).tolist()) <= set(units.tolist())


def test_reference_arm_with_host_analysis():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cd3d_rows_scrambled", "--mwm", "--order", "nd", "--side", "8",
                          "--block", "8", "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["config"]["host_analysis"] == ["mwm", "nd"] and d["config"]["gmres_iters"] > 0


def test_clock_summary_parses_samples_and_reasons(tmp_path):
    """nvidia-smi rows (index, sm MHz, max MHz, power, active mask, hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap): median and maximum clocks, the
    reasons seen Active in any sample; rows that do not parse are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2010, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
    s = c.summary()
    assert s["sm_mhz"] == 1980 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.path = str(tmp_path / "missing.csv")
    assert c.summary()["sm_mhz"] is None


def test_traffic_figures_only_while_sources_match(tmp_path, monkeypatch):
    """The committed ncu traffic per stored value is used only while the kernel sources hash
    to what was captured; after a change the figure is dropped (the bench reports null)."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(
        {"note": "x", "my_kernel": {"bytes_per_factor_value": 8.5, "source_sha": sha, "sources": ["k.cu"]}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic() == {"my_kernel": 8.5}
    (tmp_path / "k.cu").write_text("kernel v2")
    assert bench.load_traffic() == {}


def test_reference_arm_batch_line():
    """--impl reference --batch N: the oracle on a sample of the batch, scaled to all systems,
    with the batched line's metric."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--batch", "3",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and d["metric"].startswith("batched") and d["value"] > 0
    assert d["config"]["workload"] == "cd_batch_3" and d["config"]["sample_systems"] == [0, 1]


def test_batch_sample_covers_both_kinds():
    """The batch alternates 2D (even index) and 3D (odd index) systems; the reference arm's
    sample holds both kinds, every 16th of each."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1908_10169_gb300 import workloads as W
    s = bench.batch_sample(64)
    assert s == {"2d": [0, 32], "3d": [1, 33]}
    ws = W.cd_batch(count=4, seed0=100)
    assert "cd2d" in ws[0].name and "cd3d" in ws[1].name
    assert bench.batch_sample(3) == {"2d": [0], "3d": [1]}


def test_reference_arm_symmetric_line():
    """--symmetric: the oracle's BILDL + SQMR on the shifted elasticity matrix, with its own
    metric; a symmetric line on a nonsymmetric workload is refused."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "elasticity_shifted", "--symmetric", "--droptol", "1e-3", "--side", "4",
                          "--block", "24", "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["metric"].startswith("BILDL") and d["config"]["droptol"] == 1e-3
    assert d["config"]["factorization"].startswith("BILDL") and d["config"]["gmres_iters"] > 0
    bad = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--symmetric",
                          "--side", "4"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert bad.returncode != 0 and "symmetric workload" in bad.stderr
