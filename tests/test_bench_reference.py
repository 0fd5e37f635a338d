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
