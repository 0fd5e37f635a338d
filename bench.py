"""Benchmark of the SA-AMG hot path on one GB300 (or N replicas).

Default step, the largest single-GPU configuration ("inclusions_320"): Q1
hexahedra on 320^3 elements of [0,1]^3 (33,076,161 dofs, 884,836,159 stored
entries), seeded random spheres (radius 4-12 elements, >= 20 % of the
volume) with sigma = 1e6 I inside a matrix of sigma = diag(1, 1, 1e-2),
u = 0 on x = 0, and 8 right-hand sides ~ N(0,1) on the free dofs:

  classical SA setup (theta 0.04)
  + FP64 PCG on the 8 right-hand sides as one block
  + FP32-V-cycle flexible CG on the same 8 right-hand sides as one block,
  each column to a true relative residual <= 1e-8.

`value` is the step's throughput in dof-solves per second (dofs x
right-hand sides brought to 1e-8, 16 per step, divided by the step time;
MDoF-solves/s, higher is better); `ms_per_step` is the step's time to
solution.  Inputs are resident in HBM before the timed region and far larger
than L2 (the matrix alone is 10.6 GB), so no L2 flush is needed.

Besides the timed step the run reports, untimed: the same step once more with
per-launch CUDA events (roofline, kernel table, setup phases), the step
through the C ABI from pinned host buffers (`e2e`), the battery stack and
the Voronoi workload in both forms and both measures, the material measure
on the inclusions, and the CPU oracle: a measured sample step
(`cpu_baseline`) and full-size oracle solves of every configuration it can
finish within the run (iteration counts and the GPU solutions' error against
the oracle's).

--impl reference times the oracle on a bounded sample of the same workload
(the inclusions at 32^3 elements, same step) in the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
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

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 FMA lanes: 2 per SM per cycle (one warp instruction per 16 cycles; the
# nominal 1.25 TFLOP/s at 152 SMs x 2070 MHz x 4 FLOP)
N_SM, FP64_FLOP_PER_SM_CYCLE, SM_MAX_MHZ = 152, 4.0, 2070.0

WORKLOADS = {
    "inclusions_320": 320, "inclusions_160": 160, "inclusions_96": 96, "inclusions_48": 48, "inclusions_32": 32,
}
CLS_THETA, MAT_THETA, TOL, NRHS = 0.04, 0.05, 1e-8, 8
SAMPLE_N_EL = 32         # the oracle's bounded sample of the inclusions workload
METRIC = ("time-to-1e-8 residual as throughput: dofs x right-hand sides solved per second over the step "
          "(classical setup + 8-RHS FP64 PCG + 8-RHS FP32-V-cycle FCG)")
UNIT = "MDoF-solves/s"


# the paper's own figures for its battery model (Sec. 4.3; CPU cluster, FP64
# assumed, different problems and aggregation code): context for the line,
# not a target
PAPER_CONTEXT = {
    "source": "arXiv 2602.05686, Sec. 4.3, thermal battery model (Trilinos/MueLu CG, FP64 assumed)",
    "cg_iterations_16x_radial_refinement": {"classical_sa_theta_0.04": 34, "material_theta_0.08": 17},
    "smoother_complexity_same_runs": {"classical_sa_theta_0.04": 1.32, "material_theta_0.08": 1.70},
    "solve_s_n_3.25e7": {"hardware": "Eclipse: 2x18-core Intel Broadwell E5-2695 per node",
                         "1024_ranks": {"classical_sa_theta_0.04": 0.58, "material_theta_0.08": 0.35},
                         "4096_ranks": {"classical_sa": 0.26, "material": 0.17}},
}


def workload_desc(n_el):
    n = (n_el + 1) ** 3
    return (f"inclusions: Q1 hex {n_el}^3 ({n / 1e6:.2f}M dofs), seeded spheres sigma=1e6 in diag(1,1,1e-2), "
            f"u=0 on x=0, {NRHS} RHS ~ N(0,1)")


def inclusions_nnz(n_el):
    """stored entries of the inclusions matrix: the full trilinear pattern,
    prod over the axes of (3N - 2) with N = n_el + 1 nodes per axis, less the
    off-diagonals of the Dirichlet rows on x = 0 and the entries of their
    neighbours' rows in the eliminated columns"""
    N = n_el + 1
    s = 3 * N - 2
    return s ** 3 - 3 * s ** 2 + N ** 2


def workload_config(n_el, ws):
    """the `config` object of the JSON line (both arms)"""
    return {"workload": workload_desc(n_el), "dofs": (n_el + 1) ** 3, "nnz": inclusions_nnz(n_el), "rhs": NRHS,
            "measure": "classical",
            "theta": CLS_THETA, "tol": TOL, "forms": "FP64 PCG and FP32-V-cycle FCG, 8 RHS per block",
            "cheb_degree": 2, "max_coarse": 5000, "l2": "inputs larger than L2 (no flush)",
            "parallelism": f"replicas x{ws}"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(x, ws, op="max"):
    """max (or sum) of a host scalar over the ranks of the default process
    group (NCCL on the GPUs, gloo on CPU); the only collective of the
    replicas-only multi-GPU run"""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(kernel=""):
    """hash of the sources that define a kernel family (a recorded ncu traffic
    figure is used only while they are unchanged): the K-column kernels
    (names starting with b) live in block.cu with the structures of
    vcycle.cuh, the one-vector V-cycle kernels in vcycle.cu and vkern.cuh"""
    files = ("block.cu", "vcycle.cuh") if kernel.startswith("b") else ("vcycle.cu", "vkern.cuh")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2602_05686_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload):
    """ncu DRAM bytes per launch recorded for this kernel and workload, if the
    kernel sources are unchanged since the capture; else None"""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        e = t.get(f"{kernel}@{workload}")
        if e and e.get("source_hash") == kernel_source_hash(kernel):
            return float(e["bytes_per_launch"])
    except Exception:
        pass
    return None


def host_info():
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "machine": platform.machine()}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region"""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        out = os.environ.get("SA_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for k, name in enumerate(names):
                    if parts[5 + k].lower().startswith("active"):
                        reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the CPU oracle: bounded sample step and full-size parity solves, run in
# processes of their own (spawned before the first CUDA call)
# ---------------------------------------------------------------------------
def make_problem(name):
    import gen
    gen.build()
    if name == "c1":
        return gen.layered_2d(32)
    if name == "c2":
        return gen.battery_3d(128, 128, 256)
    if name == "c3":
        return gen.voronoi_3d(160)
    if name.startswith("inclusions_"):
        return gen.inclusions_3d(int(name.split("_")[1]))
    raise KeyError(name)


# (configuration, measure, theta, max_coarse) of the full-size FP64 parity solves
PARITY = {
    "c1": [("material", 0.08, 64), ("classical", 0.08, 64)],
    "c2": [("material", MAT_THETA, 5000), ("classical", CLS_THETA, 5000)],
    "c3": [("material", MAT_THETA, 5000), ("classical", CLS_THETA, 5000)],
    "c5": [("classical", CLS_THETA, 5000)],
}
PARITY_JOBS = [("c1", "c1", None), ("c2", "c2", None), ("c3", "c3", "material"), ("c3", "c3", "classical"),
               ("c5", None, None)]   # c5: the bench's own workload


def oracle_step(p, nrhs=NRHS):
    """the GPU arm's step run by the serial CPU oracle: classical setup, FP64
    PCG and flexible CG (the oracle's V-cycle is FP64 in both) on nrhs
    right-hand sides; returns seconds and iteration counts"""
    import oracle
    t = time.perf_counter()
    h = oracle.Hierarchy(p, CLS_THETA, "classical")
    it64 = [h.solve(p["B"][c], tol=TOL)[1]["iters"] for c in range(nrhs)]
    itf = [h.solve(p["B"][c], tol=TOL, flexible=True)[1]["iters"] for c in range(nrhs)]
    del h
    return time.perf_counter() - t, it64, itf


def _oracle_job(kind, cfg, problem_name, measure, outdir):
    """one oracle job (a spawned process): 'sample' times the bounded sample
    step twice; 'parity' solves the configuration at full size with the FP64
    form and stores iterations and solutions"""
    import numpy as np

    import oracle
    oracle.build()
    res = {"kind": kind, "cfg": cfg, "measure": measure}
    try:
        p = make_problem(problem_name)
        if kind == "sample":
            ts = []
            for _ in range(2):
                t, it64, itf = oracle_step(p)
                ts.append(t)
            res.update(seconds=ts, n=int(p["n"]), iters_fp64=it64, iters_flexible=itf)
        else:
            b = p["B"][0] if "B" in p else p["b"]
            rows = []
            for (m, theta, mc) in PARITY[cfg]:
                if measure and m != measure:
                    continue
                t = time.perf_counter()
                h = oracle.Hierarchy(p, theta, m, max_coarse=mc)
                ts = time.perf_counter() - t
                x, info = h.solve(b, tol=TOL)
                tt = time.perf_counter() - t - ts
                f = os.path.join(outdir, f"x_{cfg}_{m}.npy")
                np.save(f, x)
                rows.append(dict(measure=m, theta=theta, iters=info["iters"], status=info["status"],
                                 rel_res=info["rel_res"], levels=h.nlev, setup_s=round(ts, 2),
                                 solve_s=round(tt, 2), x=f))
                del h
            res["rows"] = rows
    except Exception as e:  # reported, never fatal to the bench
        res["error"] = repr(e)
    with open(os.path.join(outdir, f"{kind}_{cfg}_{measure or 'all'}.json"), "w") as fh:
        json.dump(res, fh)


class OracleJobs:
    """the oracle jobs of one bench run, as spawned processes (spawn, not
    fork: they start before the first CUDA call and share nothing with it)"""

    def __init__(self, workload, parity_cfgs, with_sample=True):
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="sa_oracle_")
        ctx = mp.get_context("spawn")
        self.procs = []
        jobs = []
        if with_sample:
            jobs.append(("sample", "sample", f"inclusions_{SAMPLE_N_EL}", None))
        jobs += [("parity", c, pn or workload, m) for (c, pn, m) in PARITY_JOBS if c in parity_cfgs]
        for j in jobs:
            pr = ctx.Process(target=_oracle_job, args=(*j, self.dir), daemon=True)
            pr.start()
            self.procs.append((j, pr))
        self.t0 = time.perf_counter()

    def cleanup(self):
        import shutil
        shutil.rmtree(self.dir, ignore_errors=True)

    def collect(self, deadline_s):
        """results of the jobs that finished within deadline_s of their start;
        the rest are stopped and reported as not finished"""
        out = []
        for (j, pr) in self.procs:
            left = deadline_s - (time.perf_counter() - self.t0)
            pr.join(timeout=max(0.0, left))
            if pr.is_alive():
                pr.terminate()
                pr.join(timeout=10)
                out.append({"kind": j[0], "cfg": j[1], "measure": j[3],
                            "error": f"not finished within the run's {deadline_s:.0f} s oracle budget"})
                continue
            f = os.path.join(self.dir, f"{j[0]}_{j[1]}_{j[3] or 'all'}.json")
            try:
                with open(f) as fh:
                    out.append(json.load(fh))
            except OSError:
                out.append({"kind": j[0], "cfg": j[1], "measure": j[3], "error": "no result written"})
        return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def setup_phases(prof):
    """stream time per setup phase, summed over levels"""
    out = {}
    for r in prof:
        if r["kind"].startswith("setup_"):
            out[r["kind"][6:]] = out.get(r["kind"][6:], 0.0) + r["ms"]
    return {k: round(v, 2) for k, v in sorted(out.items(), key=lambda kv: -kv[1])}


def setup_roofline(phases_ms, sizes, peak):
    """algorithmic bytes of each setup phase (what it must move at least once,
    summed over the coarsening levels: CSR values 8 B, columns 4 B, row
    pointers 8 B; see the phase list below) against its measured stream time.
    sizes: per level dicts of n, nnz, nnz_P, nc, nnz_gc (level_sizes)."""
    by = {}

    def add(k, b):
        by[k] = by.get(k, 0.0) + b

    L = len(sizes)
    for l, z in enumerate(sizes):
        n, nnz, nP, nc, ngc = z["n"], z["nnz"], z["nnz_P"], z["nc"], z["nnz_gc"]
        if l < L - 1:
            nnz_c = sizes[l + 1]["nnz"]
            add("strength", 12 * nnz + 1 * nnz + 8 * (n + 1) + 16 * n)            # A in, keep + counts out
            add("graph", 5 * nnz + 8 * n + 4 * ngc + 8 * (n + 1))                 # keep, columns in; G_C out
            add("mis2", 4 * ngc + 8 * (n + 1) + 16 * n)                            # one sweep of G_C and tags
            add("aggregate", 4 * ngc + 8 * (n + 1) + 8 * n)
            add("filter", 13 * nnz + 8 * (n + 1) + 12 * (ngc + n) + 16 * n)        # A, keep in; A_F, D~ out
            add("omega", 10 * (12 * (ngc + n) + 24 * n))                           # ten products with A_F
            add("smooth_p", 12 * (ngc + n) + 4 * n + 12 * nP + 8 * (n + 1))        # A_F, agg in; P out
            add("transpose", 2 * (12 * nP) + 8 * (n + 1) + 8 * (nc + 1))           # P in, R out
            add("galerkin", 12 * nnz + 2 * 12 * nP + 12 * nnz_c + 8 * (nc + 1))   # A, P, R in; A_c out
            add("aux", 0)
        add("cheb_bounds", 10 * (12 * nnz + 24 * n) if l < L - 1 else 0)
        add("sell", 12 * nnz + 10 * nnz)                                            # CSR in, SELL copy out
    out = {}
    for k, ms in phases_ms.items():
        if k in by and by[k] > 0 and ms > 0:
            gbs = by[k] / (ms * 1e-3) / 1e9
            out[k] = {"ms": ms, "algorithmic_GB": round(by[k] / 1e9, 3), "GBs": round(gbs, 1),
                      "frac_of_hbm": round(gbs / peak, 3)}
    if sizes:
        nL = sizes[-1]["n"]
        ms = phases_ms.get("dense")
        if ms:
            fl = nL ** 3 / 3.0
            out["dense"] = {"ms": ms, "flops": fl, "TFLOPs": round(fl / (ms * 1e-3) / 1e12, 4),
                            "note": "coarse Cholesky factor (n_L^3/3), overlapped with other setup work"}
    return out


def fp64_flops(kind, level, nnz0, n0, K):
    """FP64 FLOPs per launch of a level-0 FP64 kernel: one FMA per stored
    entry and column plus the row updates"""
    if level != 0:
        return None
    per_row = {"cheb64": 5, "resid64": 1, "cg_spmv": 2}
    per_row_k = {"bcheb64": 5, "bresid64": 1, "bcg_spmv": 2}
    if kind in per_row:
        return 2.0 * nnz0 + per_row[kind] * n0
    if kind in per_row_k:
        return K * (2.0 * nnz0 + per_row_k[kind] * n0)
    return None


def rel_err(x, ref):
    import numpy as np
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / d) if d > 0 else float(np.linalg.norm(x))


def run_ours(args):
    import numpy as np

    ws, rank, local = dist_env()
    n_el = WORKLOADS[args.workload]
    # the oracle processes start before the first CUDA call (spawned)
    jobs = None
    cfgs = [] if args.no_oracle_parity else [c for c in args.oracle_configs.split(",") if c]
    if args.no_extras:
        cfgs = [c for c in cfgs if c == "c5"]
    if rank == 0 and ws == 1 and (cfgs or not args.no_cpu_baseline):
        jobs = OracleJobs(args.workload, cfgs, with_sample=not args.no_cpu_baseline)

    import torch

    import gen
    import paper_2602_05686_gb300 as sa

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sa.build()
    t_gen = time.perf_counter()
    p = gen.inclusions_3d(n_el, nrhs=NRHS)
    gen_s = time.perf_counter() - t_gen
    n, nnz0 = int(p["n"]), int(p["nnz"])
    keys = ("row_ptr", "col", "val")     # what the classical setup reads
    dprob = dict(p, **{k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda()
                       for k in keys + ("coords", "tensors", "elem_nodes", "elem_measure")})
    B = torch.from_numpy(np.ascontiguousarray(p["B"])).cuda()
    stream = torch.cuda.current_stream()
    units = float(n) * 2 * NRHS    # dof-solves per step: every RHS in both forms

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def one_step(prob, rhs, host=False, outs=None):
        """the step; per-part times (ms, CUDA events), solve infos, solutions"""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        h = sa.Hierarchy(prob, theta=CLS_THETA, measure="classical", precision="fp64", host_inputs=host)
        ev[1].record(stream)
        X64, i64 = h.solve_batch(rhs, out=outs[0] if outs else None)
        ev[2].record(stream)
        h.set_precision("fp32")
        ev[3].record(stream)
        X32, i32 = h.solve_batch(rhs, out=outs[1] if outs else None)
        ev[4].record(stream)
        st = h.stats()
        h.free()
        torch.cuda.synchronize()
        t = [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
        parts = dict(setup_ms=t[0], fp64_solve_ms=t[1], fp32_build_ms=t[2], fp32_solve_ms=t[3])
        return parts, dict(fp64=i64, fp32=i32), st, (X64, X32)

    for _ in range(args.warmup):
        one_step(dprob, B)
    # timed region (device-resident inputs): the production path
    clk = ClockSampler(local)
    clk.start()
    l0 = sa.launch_count()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    parts_all, infos, hst, sols = [], None, None, None
    for _ in range(args.steps):
        parts, infos, hst, sols = one_step(dprob, B)
        parts_all.append(parts)
    t1.record(stream)
    barrier()
    launches = sa.launch_count() - l0
    clocks = clk.stop()
    ms_step = t0.elapsed_time(t1) / args.steps
    ms_step = reduce_over_ranks(ms_step, ws, "max")        # the slowest replica sets the step time
    launches = int(reduce_over_ranks(launches, ws, "sum"))  # kernels of all replicas
    value = units * ws / (ms_step * 1e-3) / 1e6

    # one more step with every launch bracketed by CUDA events on the
    # library's stream: the kernel table, the roofline, the setup phases
    sa.profile_enable(True)
    barrier()
    t2 = torch.cuda.Event(enable_timing=True)
    t3 = torch.cuda.Event(enable_timing=True)
    t2.record(stream)
    one_step(dprob, B)
    t3.record(stream)
    barrier()
    prof = sa.profile_read()
    sa.profile_enable(False)
    ms_step_prof = t2.elapsed_time(t3)
    hh = sa.Hierarchy(dprob, theta=CLS_THETA, measure="classical", precision="fp64")
    lsizes = [hh.level_sizes(l) for l in range(hh.stats()["levels"])]
    hh.free()
    x64_0 = sols[0][0].cpu().numpy()
    x32_0 = sols[1][0].cpu().numpy()
    del sols

    # roofline of the dominant kernel (largest total time in the profiled
    # step): algorithmic bytes per launch / mean CUDA-event duration against
    # the measured copy bandwidth, with the FP64-pipe floor beside it for the
    # FP64 fine-level kernels; the larger floor names the bound
    peak, peak_kind = peaks()
    mhz = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
    fp64_peak = N_SM * FP64_FLOP_PER_SM_CYCLE * mhz * 1e6 / 1e12   # TFLOP/s
    rows = sorted(prof, key=lambda r: -r["ms"])
    krows = [r for r in rows if r["bytes"] > 0]
    roof = None
    if krows:
        dom = krows[0]
        per_launch_ms = dom["ms"] / dom["launches"]
        per_launch_bytes = dom["bytes"] / dom["launches"]
        ach = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
        kname = f"{dom['kind']}_level{dom['level']}"
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": traffic_for(kname, args.workload),
                "kernel": kname, "peak_source": peak_kind, "launches": dom["launches"],
                "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": round(per_launch_ms, 5)}
        fl = fp64_flops(dom["kind"], dom["level"], nnz0, n, NRHS)
        if fl:
            t_hbm = per_launch_bytes / (peak * 1e9)
            t_fp64 = fl / (fp64_peak * 1e12)
            a64 = fl / (per_launch_ms * 1e-3) / 1e12
            roof["fp64_pipe"] = {"achieved": round(a64, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                                 "frac": round(a64 / fp64_peak, 4), "flops_per_launch": fl,
                                 "peak_source": f"derived: {N_SM} SMs x 4 FLOP/cycle x {mhz:.0f} MHz"}
            if t_fp64 > t_hbm:   # the FP64 pipe is the tighter floor
                hb = {k: roof.pop(k) for k in ("achieved", "peak", "unit", "frac", "peak_source")}
                roof.update(bound="alu", achieved=roof["fp64_pipe"]["achieved"], peak=roof["fp64_pipe"]["peak"],
                            unit="TFLOP/s", frac=roof["fp64_pipe"]["frac"],
                            peak_source=roof["fp64_pipe"]["peak_source"], hbm=hb)

    # V-cycle bandwidth per form (all V-cycle kernels of the profiled step)
    def vgb(kinds):
        sel = [r for r in prof if r["kind"] in kinds]
        ms = sum(r["ms"] for r in sel)
        by = sum(r["bytes"] for r in sel)
        return {"GBs": round(by / (ms * 1e-3) / 1e9, 1), "frac_of_hbm": round(by / (ms * 1e-3) / 1e9 / peak, 3),
                "ms": round(ms, 1)} if ms > 0 else None

    vc64 = vgb({"bcheb64", "bresid64", "brestrict64", "bprolong64", "bfirst64"})
    vc32 = vgb({"bcheb32", "bresid32", "brestrict32", "bprolong32", "bfirst32"})
    avg = {k: round(statistics.mean(pp[k] for pp in parts_all), 2) for k in parts_all[0]}

    extras = None if args.no_extras else run_extras(sa, torch, dprob)
    # a short serving pass (c4 workload, 128 requests): latency and throughput
    serving = None
    if not args.no_serving and ws == 1:
        del B
        serving = serving_pass(torch, 128, 6, 32, 256, 48, True)

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 2), "higher_is_better": True,
        "ms_per_step_instrumented": round(ms_step_prof, 2),
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 inside the mixed V-cycle)",
        "data": "synthetic (seeded generator; the paper's meshes are not public)",
        "config": workload_config(n_el, ws),
        "time_to_solution_s": {"step": round(ms_step / 1e3, 4), "setup": round(avg["setup_ms"] / 1e3, 4),
                               "fp64_solve_8rhs": round(avg["fp64_solve_ms"] / 1e3, 4),
                               "fp32_solve_8rhs": round((avg["fp32_build_ms"] + avg["fp32_solve_ms"]) / 1e3, 4)},
        "parts_ms": avg,
        "fp32_speedup_vs_fp64_solve": round(avg["fp64_solve_ms"] / (avg["fp32_build_ms"] + avg["fp32_solve_ms"]), 3),
        "iters": {"fp64": [i["iters"] for i in infos["fp64"]], "fp32": [i["iters"] for i in infos["fp32"]]},
        "rel_res_max": {"fp64": max(i["rel_res"] for i in infos["fp64"]),
                        "fp32": max(i["rel_res"] for i in infos["fp32"])},
        "fp32_vs_fp64_solution_rel_diff_rhs0": rel_err(x32_0, x64_0),
        "hierarchy": {"levels": hst["levels"], "n": hst["n"], "op_complexity": round(hst["op_complexity"], 4)},
        "vcycle_bandwidth": {"fp64": vc64, "fp32": vc32},
        "roofline": roof,
        "clocks": clocks,
        "e2e": None,
        "gpu_launches": int(launches),
        "generation_s": round(gen_s, 1),
        "kernel_profile_top": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in r.items()}
                               for r in krows[:10]],
        "setup_phases_ms": setup_phases(prof),
        "setup_roofline": setup_roofline(setup_phases(prof), lsizes, peak),
        "kernel_profile_all": [[r["kind"], r["level"], r["launches"], round(r["ms"], 3)] for r in krows],
        "extras": extras,
        "serving": serving,
        "paper_context": PAPER_CONTEXT,
    }
    if jobs is not None:
        res = jobs.collect(args.oracle_deadline)
        sample = next((r for r in res if r["kind"] == "sample"), None)
        if sample is not None and "seconds" in sample:
            t = statistics.mean(sample["seconds"])
            result["cpu_baseline"] = {
                "value": round(sample["n"] * 2 * NRHS / t / 1e6, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": (f"measured: the same step (classical setup + 8 FP64 PCG + 8 flexible-CG solves, FP64 "
                           f"V-cycle) on the inclusions workload at {SAMPLE_N_EL}^3 elements ({sample['n']} dofs), "
                           f"{t:.2f} s per step, mean of 2 steps, one thread"),
                "iters_fp64": sample["iters_fp64"], "iters_flexible": sample["iters_flexible"],
                "host": host_info()}
        elif sample is not None:
            result["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                      "sample": sample.get("error", "failed"), "host": host_info()}
        par = [r for r in res if r["kind"] == "parity"]
        if par:
            result["oracle_parity"] = parity_report(par, extras, infos, x64_0, x32_0)
        # the oracle at full size on this workload (its parity solve: setup and
        # one FP64 PCG solve, measured in this run), beside the bounded sample
        full = result.get("oracle_parity", {}).get("c5", {}).get("classical")
        if full and result.get("cpu_baseline") and full.get("oracle_solve_s"):
            n5 = result["config"]["dofs"]
            ts = full["oracle_setup_s"] + full["oracle_solve_s"]
            result["cpu_baseline"]["full_size"] = {
                "measured": "full size, same run: classical setup + one FP64 PCG solve (right-hand side 0), one thread",
                "dofs": n5, "setup_s": full["oracle_setup_s"], "solve_s_one_rhs": full["oracle_solve_s"],
                "iters": full["iters_oracle"], "value_one_rhs": round(n5 / ts / 1e6, 5), "unit": UNIT}
        jobs.cleanup()
    # the end-to-end pass runs after the oracle processes have finished, so
    # that their host-memory traffic does not share the host with its copies
    # end to end through the C ABI from pinned host buffers: the matrix and
    # the right-hand sides are copied to the device, and the solutions back,
    # inside the timed region
    e2e = None
    if not args.no_e2e:
        ph = dict(p, **{k: torch.from_numpy(np.ascontiguousarray(p[k])).pin_memory().numpy() for k in keys})
        Bh = torch.from_numpy(np.ascontiguousarray(p["B"])).pin_memory().numpy()
        outs = (torch.empty(Bh.shape, dtype=torch.float64).pin_memory().numpy(),
                torch.empty(Bh.shape, dtype=torch.float64).pin_memory().numpy())
        one_step(ph, Bh, host=True, outs=outs)    # warm
        barrier()
        reps = max(1, min(args.steps, 2))
        te = time.perf_counter()
        for _ in range(reps):
            one_step(ph, Bh, host=True, outs=outs)
        barrier()
        e_s = (time.perf_counter() - te) / reps
        inb = sum(int(np.asarray(p[k]).nbytes) for k in keys)
        # in: the problem arrays and the right-hand sides of each form (the
        # solves start from zero: sa_solve_batch_zero reads no initial guess);
        # out: the solutions of each form
        e2e = {"value": round(units / e_s / 1e6, 3), "unit": UNIT, "seconds_per_step": round(e_s, 4),
               "h2d_bytes_per_step": inb + 2 * int(Bh.nbytes), "d2h_bytes_per_step": 2 * int(Bh.nbytes)}
        del ph, Bh, outs

    result["e2e"] = e2e
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_extras(sa, torch, c5prob):
    """the other configurations, one solve each (untimed region, CUDA events):
    the 2D layered square (c1), the battery stack (c2) and the Voronoi
    anisotropic cube (c3) with both measures and both forms, and the material
    measure on the inclusions (both dropping criteria, FP64 form, capped)"""
    import numpy as np
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    out = {}
    for cfg in ("c1", "c2", "c3"):
        p = make_problem(cfg)
        dp = dict(p, **{k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda()
                        for k in ("row_ptr", "col", "val", "coords", "tensors", "elem_nodes", "elem_measure")})
        b = torch.from_numpy(p["b"]).cuda()
        res = {"dofs": int(p["n"])}
        for (m, theta, mc) in PARITY[cfg]:
            h, ts = timed(lambda: sa.Hierarchy(dp, theta=theta, measure=m, precision="fp64", max_coarse=mc))
            h.solve(b, tol=TOL, check=False)       # first use of a form captures its CG graph
            (x64, i64), t64 = timed(lambda: h.solve(b, tol=TOL, check=False))
            h.set_precision("fp32")
            h.solve(b, tol=TOL, check=False)
            (x32, i32), t32 = timed(lambda: h.solve(b, tol=TOL, check=False))
            st = h.stats()
            h.free()
            res[m] = {"theta": theta, "setup_ms": round(ts, 2), "fp64_solve_ms": round(t64, 2),
                      "fp32_solve_ms": round(t32, 2), "fp32_speedup_vs_fp64_solve": round(t64 / t32, 3),
                      "iters_fp64": i64["iters"], "iters_fp32": i32["iters"], "rel_res_fp64": i64["rel_res"],
                      "rel_res_fp32": i32["rel_res"], "status_fp64": i64["status"], "status_fp32": i32["status"],
                      "levels": st["levels"], "op_complexity": round(st["op_complexity"], 4),
                      "_x64": x64.cpu().numpy(), "_x32": x32.cpu().numpy()}
        out[cfg] = res
        del dp, p
    # the material measure on the inclusions (the paper's measure, both
    # dropping criteria): FP64 form, capped at 200 iterations
    res = {}
    b = c5prob["B"][0]
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    for name, kw in (("pointwise_0.05", dict(theta=MAT_THETA, drop="pointwise")),
                     ("cut_0.08", dict(theta=0.08, drop="cut"))):
        h, ts = timed(lambda: sa.Hierarchy(c5prob, measure="material", precision="fp64", maxit=200, **kw))
        (_, inf), t64 = timed(lambda: h.solve(bt, tol=TOL, check=False))
        st = h.stats()
        h.free()
        res[name] = {"setup_ms": round(ts, 2), "fp64_solve_ms": round(t64, 2), "iters": inf["iters"],
                     "status": inf["status"], "rel_res": inf["rel_res"], "levels": st["levels"],
                     "op_complexity": round(st["op_complexity"], 4)}
    out["c5_material"] = res
    return out


def parity_report(par, extras, infos, x64_0, x32_0):
    """iteration counts of the full-size oracle solves beside the GPU's, and
    the GPU solutions' relative error against the oracle's (FP64 form and
    FP32-V-cycle form)"""
    import numpy as np
    rep = {}
    for r in par:
        cfg = r["cfg"]
        if "error" in r:
            rep.setdefault(cfg, {})[r.get("measure") or "all"] = {"oracle": r["error"]}
            continue
        for row in r["rows"]:
            m = row["measure"]
            xo = np.load(row["x"])
            e = {"iters_oracle": row["iters"], "oracle_status": row["status"], "oracle_rel_res": row["rel_res"],
                 "oracle_setup_s": row["setup_s"], "oracle_solve_s": row["solve_s"]}
            if cfg == "c5":
                e.update(iters=infos["fp64"][0]["iters"], iters_fp32=infos["fp32"][0]["iters"],
                         err_fp64_vs_oracle=rel_err(x64_0, xo), err_fp32_vs_oracle=rel_err(x32_0, xo))
            elif extras and cfg in extras and m in extras[cfg]:
                g = extras[cfg][m]
                e.update(iters=g["iters_fp64"], iters_fp32=g["iters_fp32"],
                         err_fp64_vs_oracle=rel_err(g["_x64"], xo), err_fp32_vs_oracle=rel_err(g["_x32"], xo))
            e["iters_within_1"] = abs(e.get("iters", -99) - row["iters"]) <= 1 if "iters" in e else None
            rep.setdefault(cfg, {})[m] = e
            try:
                os.remove(row["x"])
            except OSError:
                pass
    if extras:
        for cfg in ("c1", "c2", "c3"):
            for m in list(extras.get(cfg, {})):
                if isinstance(extras[cfg][m], dict):
                    extras[cfg][m].pop("_x64", None)
                    extras[cfg][m].pop("_x32", None)
    return rep


# ---------------------------------------------------------------------------
# reference arm: the oracle on a bounded sample, same metric and unit
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import gen
    import oracle
    oracle.build()
    gen.build()
    n_el = WORKLOADS[args.workload]
    p = gen.inclusions_3d(SAMPLE_N_EL, nrhs=NRHS)
    for _ in range(args.warmup):
        oracle_step(p)
    ts, it64, itf = [], None, None
    for _ in range(args.steps):
        t, it64, itf = oracle_step(p)
        ts.append(t)
    sec = statistics.mean(ts)
    val = p["n"] * 2 * NRHS / sec / 1e6
    sample = (f"measured: the same step (classical setup + 8 FP64 PCG + 8 flexible-CG solves, FP64 V-cycle) on the "
              f"inclusions workload at {SAMPLE_N_EL}^3 elements ({p['n']} dofs) per step, one thread")
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 5), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1000, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator; the paper's meshes are not public)",
           "config": workload_config(n_el, ws),
           "iters_sample": {"fp64": it64, "flexible": itf},
           "cpu_baseline": {"value": round(val, 5), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                            "host": host_info()},
           "e2e": {"value": round(val, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# other modes
# ---------------------------------------------------------------------------
def serving_pass(torch, nreq, slots, hbm_gb, max2d, max3d, group, rank=0, ws=1):
    """the serving workload: seeded Poisson-arrival requests on 2D/3D layered
    operators (contrast 10^U(2,10)), several right-hand sides per operator with
    the hierarchy cached, HBM-admitted, FP32 V-cycle inside FP64 flexible CG;
    the arrival rate is 0.8 x the throughput of a back-to-back warm-up run.
    group: single requests of different operators are solved together in
    shared launches (sa_solve_group).  Under torchrun each rank serves the
    operators placed on it and the latencies are gathered."""
    import numpy as np

    import gen
    from paper_2602_05686_gb300.serving import Request, Server, gather_stats, partition

    ops, reqs = gen.serving_requests(nreq, seed=11, max2d=max2d, max3d=max3d)
    t = time.perf_counter()
    probs = {k: gen.layered_serving(o["dim"], o["n_el"], o["contrast"]) for k, o in enumerate(ops)}
    gen_s = time.perf_counter() - t
    rhs = []
    for r in reqs:
        p = probs[r["op"]]
        b = gen.Stream(1000 + r["rhs_seed"], 9).normal(p["n"])
        b[p["dir_mask"] == 1] = 0.0
        rhs.append(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()

    def options(op):
        return dict(theta=0.05, measure="material", precision="fp32", max_coarse=5000)

    def run(scale, realtime):
        srv = Server(lambda op: probs[op], options, slots=slots, hbm_budget=hbm_gb << 30, group_solves=group)
        rs, tt = [], 0.0
        for k, r in enumerate(reqs):
            tt += r["gap"] * scale
            rs.append(Request(rid=k, op=r["op"], arrival=tt, rhs=rhs[k]))
        mine, _ = partition(rs, srv._estimate, rank, ws) if ws > 1 else (rs, None)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        local_out = srv.serve(mine, realtime=realtime)
        srv.close()
        return gather_stats(local_out, ws) if ws > 1 else local_out, mine

    warm, _ = run(0.0, False)
    rate = 0.8 * warm["throughput_rps"]
    out, rs = run(1.0 / rate, True)
    iters = [r.info.get("iters", 0) for r in rs]
    return {"p50_s": round(out["p50_s"], 4), "p99_s": round(out["p99_s"], 4),
            "req_per_s": round(out["throughput_rps"], 2), "arrival_rate_rps": round(rate, 2),
            "warmup_req_per_s": round(warm["throughput_rps"], 2), "requests": nreq, "operators": len(ops),
            "slots": slots, "group_solves": bool(group), "setups": out.get("setups"), "cache_hits": out.get("hits"),
            "groups": out.get("groups"), "max_group": out.get("max_group"), "evictions": out.get("evictions"),
            "failed": out.get("failed"), "mean_iters": round(float(np.mean(iters)), 1) if iters else None,
            "max_rel_res": max((r.info.get("rel_res", 0.0) for r in rs), default=None),
            "per_gpu_requests": out.get("per_device_requests"), "generation_s": round(gen_s, 1),
            "workload": f"serving: {nreq} requests, 2D 16^2..{max2d}^2 and 3D 16^3..{max3d}^3 layered operators, "
                        "contrast 1e2..1e10, 1-16 RHS per operator, FP32 V-cycle in FP64 flexible CG"}


def run_serving(args):
    """Serving workload (c4) on its own, one JSON line (p99 latency as the
    value)."""
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r = serving_pass(torch, args.requests, args.slots, args.hbm_gb, args.max2d, args.max3d, not args.no_group,
                     rank, ws)
    if rank != 0:
        return
    res = {"metric": "serving latency p50/p99 (continuous batching, cached hierarchies)",
           "value": r["p99_s"], "unit": "s (p99 latency)", "higher_is_better": False, "n_gpus": ws, **r,
           "config": {"workload": r["workload"], "precision": "FP32 V-cycle in FP64 flexible CG", "tol": TOL}}
    print(json.dumps(res), flush=True)


def run_annulus(args):
    """The annulus study of Sec. 4.2 (Table 1 analogue): refinements h ..
    h/2^max, contrast 1 .. 1e4, material measure, theta 0.05 and 0.1, FP64
    PCG to 1e-8; one JSON line per configuration."""
    import torch

    import gen
    import paper_2602_05686_gb300 as sa
    from paper_2602_05686_gb300.sweep import annulus_study

    torch.cuda.set_device(0)
    sa.build()
    cache = {}

    def make(rf, k):
        if (rf, k) not in cache:
            cache.clear()
            cache[(rf, k)] = gen.annulus_3d(rf, kappa=k)
        return cache[(rf, k)]

    annulus_study(make, refines=(0,), kappas=(1.0,))   # warm-up (module loads)
    for row in annulus_study(make, refines=tuple(range(args.annulus_refine + 1))):
        print(json.dumps(dict(row, workload="annulus (Sec. 4.2)")), flush=True)


def run_sweep(args):
    """The two-domain drop-tolerance study of Sec. 4.1: (-1,1)^2 with
    32, 128 and 512 elements per side, kappa in {1, 1e2, 1e4}, every theta of
    the paper's list, the three strength measures and both dropping criteria,
    FP64 PCG to 1e-8; one JSON line per configuration."""
    import torch

    import gen
    import paper_2602_05686_gb300 as sa
    from paper_2602_05686_gb300.sweep import theta_sweep

    torch.cuda.set_device(0)
    sa.build()
    theta_sweep(gen.two_domain(32, 1.0), thetas=(0.08,), measures=("material",))   # warm-up (module loads)
    for n_el in (32, 128, 512):
        for kappa in (1.0, 1e2, 1e4):
            p = gen.two_domain(n_el, kappa)
            for row in theta_sweep(p, drops=("pointwise", "cut")):
                print(json.dumps(dict(row, n_el=n_el, kappa=kappa, workload="two-domain (Sec. 4.1)")), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="inclusions_320", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-parity", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--oracle-configs", default="c1,c2,c3,c5",
                    help="configurations the oracle solves at full size beside the GPU (c5 = the workload)")
    ap.add_argument("--oracle-deadline", type=float, default=1080.0,
                    help="seconds after the start of the run within which the oracle jobs must finish")
    ap.add_argument("--serving", action="store_true", help="run the serving workload instead")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--hbm-gb", type=int, default=64)
    ap.add_argument("--max2d", type=int, default=512)
    ap.add_argument("--max3d", type=int, default=96)
    ap.add_argument("--no-group", action="store_true", help="serving without group solves")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving pass of the default run")
    ap.add_argument("--annulus", action="store_true", help="run the annulus study (Sec. 4.2) instead")
    ap.add_argument("--annulus-refine", type=int, default=4)
    ap.add_argument("--sweep", action="store_true", help="run the two-domain theta sweep (Sec. 4.1) instead")
    args = ap.parse_args()
    if args.serving:
        run_serving(args)
    elif args.sweep:
        run_sweep(args)
    elif args.annulus:
        run_annulus(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
