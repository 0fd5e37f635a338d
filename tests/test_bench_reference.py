"""The reference arm of bench.py (the oracle, timed on the host) prints one
JSON line with the keys the benchmark contract names; CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith("inclusions") and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["host"]["nproc"] >= 1 and d["cpu_baseline"]["sample"].startswith("measured")
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the value is what the timed steps measured: units per step over the step time
    assert abs(d["value"] - d["config"]["rhs"] * 2 * 35937 / (d["ms_per_step"] / 1e3) / 1e6) <= 1e-3 * d["value"]
    assert len(d["iters_sample"]["fp64"]) == 8 and min(d["iters_sample"]["fp64"]) > 0


def test_oracle_jobs_report_parity_and_sample():
    # the bench's spawned oracle processes: a sample step and one full-size
    # parity solve (the 2D layered square), collected with their results
    sys.path.insert(0, ROOT)
    import bench
    jobs = bench.OracleJobs("inclusions_32", ["c1"], with_sample=False)
    res = jobs.collect(300)
    jobs.cleanup()
    assert len(res) == 1 and res[0]["cfg"] == "c1" and "error" not in res[0]
    rows = {r["measure"]: r for r in res[0]["rows"]}
    assert set(rows) == {"material", "classical"}
    assert all(r["status"] == 0 and r["rel_res"] <= 1e-8 and r["iters"] > 0 for r in rows.values())


def test_setup_roofline_bytes_and_fraction():
    """algorithmic bytes of the setup phases from the level sizes: a two-level
    hierarchy by hand"""
    sys.path.insert(0, ROOT)
    import bench
    sizes = [dict(n=1000, nnz=27000, nnz_P=3000, nc=100, nnz_gc=20000),
             dict(n=100, nnz=2700, nnz_P=0, nc=0, nnz_gc=0)]
    r = bench.setup_roofline({"galerkin": 1.0, "strength": 0.5, "dense": 2.0, "cheb_bounds": 1.0}, sizes, 1000.0)
    # Galerkin: A (12 B per entry) in, P and R (12 B per entry each) in, A_c out, coarse row pointers
    g = 12 * 27000 + 24 * 3000 + 12 * 2700 + 8 * 101
    assert r["galerkin"]["algorithmic_GB"] == round(g / 1e9, 3)
    assert abs(r["galerkin"]["GBs"] - g / 1e-3 / 1e9) < 0.1
    assert r["strength"]["frac_of_hbm"] == round((13 * 27000 + 8 * 1001 + 16 * 1000) / 0.5e-3 / 1e9 / 1000.0, 3)
    assert r["cheb_bounds"]["algorithmic_GB"] == round(10 * (12 * 27000 + 24 * 1000) / 1e9, 3)
    assert r["dense"]["flops"] == 100 ** 3 / 3.0


def test_traffic_record_only_for_unchanged_sources(tmp_path, monkeypatch):
    """a recorded ncu DRAM figure enters the line only while the sources of
    its kernel family hash as when it was taken"""
    sys.path.insert(0, ROOT)
    import bench
    hb, h1 = bench.kernel_source_hash("bcheb64"), bench.kernel_source_hash("cheb64")
    assert len(hb) == 16 and hb == bench.kernel_source_hash("bcg_spmv") and hb != h1
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps({"bcheb64_level0@w": {"bytes_per_launch": 123, "source_hash": hb},
                             "cheb64_level0@w": {"bytes_per_launch": 45, "source_hash": hb}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.traffic_for("bcheb64_level0", "w") == 123.0
    assert bench.traffic_for("bcheb64_level0", "other") is None
    assert bench.traffic_for("cheb64_level0", "w") is None      # one-vector family: other sources
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel="": "0" * 16)
    assert bench.traffic_for("bcheb64_level0", "w") is None


def test_fp64_flops_of_level0_kernels():
    """two flops per stored entry and column plus the row updates; level-0
    FP64 kernels only.  The 320^3 inclusions Chebyshev step: the figure the
    bench line reports per launch"""
    sys.path.insert(0, ROOT)
    import bench
    nnz, n = bench.inclusions_nnz(320), 321 ** 3
    assert bench.fp64_flops("bcheb64", 0, nnz, n, 8) == 15480424984.0
    assert bench.fp64_flops("bcheb64", 0, nnz, n, 8) == 8 * bench.fp64_flops("cheb64", 0, nnz, n, 1)
    assert bench.fp64_flops("bresid64", 0, 100, 10, 4) == 4 * (200 + 10)
    assert bench.fp64_flops("bcheb64", 1, nnz, n, 8) is None
    assert bench.fp64_flops("bcheb32", 0, nnz, n, 8) is None
