"""Benchmark of the SA-AMG hot path on one GB300 (or N replicas).

One step = the whole hot path on the battery-stack workload (Q1 hex
128 x 128 x 256 elements, 4,276,737 dofs, z-spacing 0.01 of the x/y
spacing, layer cycle sigma = 1e5 / 1e-5 / 1e2 of 8 elements each, u = 0 at
z = 0 and u = 1 at the top):
  material-aware setup (theta 0.05) + FP64 PCG to 1e-8
  + FP32-V-cycle flexible CG to 1e-8 on the same hierarchy
  + classical setup (theta 0.04) + FP64 PCG to 1e-8 (the paper's comparison).
Inputs are resident in HBM before the timed region and are larger than L2
(A alone is 1.36 GB), so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
instead (bounded sample, extrapolated to the full workload by dof count).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
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
    # name: (generator kwargs, description)
    "battery_128x128x256": (dict(nx=128, ny=128, nz=256), "battery-like stack, Q1 hex 128x128x256 (4.28M dofs)"),
    "battery_96x96x192": (dict(nx=96, ny=96, nz=192), "battery-like stack, Q1 hex 96x96x192 (1.8M dofs)"),
    "battery_64x64x128": (dict(nx=64, ny=64, nz=128), "battery-like stack, Q1 hex 64x64x128 (0.54M dofs)"),
    "battery_32x32x64": (dict(nx=32, ny=32, nz=64), "battery-like stack, Q1 hex 32x32x64 (71k dofs)"),
}
MAT_THETA, CLS_THETA, TOL = 0.05, 0.04, 1e-8
METRIC = "time-to-1e-8 residual per step (material setup + FP64 PCG + FP32-V-cycle FCG + classical setup + FP64 PCG)"


def battery_nnz(nx, ny, nz):
    """stored entries of the battery stack's matrix after the Dirichlet
    elimination at z = 0 and at the top (rows there keep their diagonal)"""
    sxy = (3 * (nx + 1) - 2) * (3 * (ny + 1) - 2)
    total = 0
    for k in range(nz + 1):
        if k == 0 or k == nz:
            total += (nx + 1) * (ny + 1)
        else:
            total += sxy * (3 - (k - 1 == 0) - (k + 1 == nz))
    return total


def workload_config(args, ws):
    """the `config` object of the JSON line (both arms)"""
    kw, desc = WORKLOADS[args.workload]
    return {"workload": desc, "dofs": (kw["nx"] + 1) * (kw["ny"] + 1) * (kw["nz"] + 1),
            "nnz": battery_nnz(kw["nx"], kw["ny"], kw["nz"]), "material_theta": MAT_THETA,
            "classical_theta": CLS_THETA, "tol": TOL, "cheb_degree": 2, "max_coarse": 5000,
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"}


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


def kernel_source_hash():
    """hash of the sources that define the V-cycle kernels (a recorded ncu
    traffic figure is used only while they are unchanged)"""
    h = hashlib.sha256()
    for f in ("vcycle.cu", "vkern.cuh"):
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
        if e and e.get("source_hash") == kernel_source_hash():
            return float(e["bytes_per_launch"])
    except Exception:
        pass
    return None


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
# our arm
# ---------------------------------------------------------------------------
def setup_phases(prof, steps):
    """stream time per setup phase, summed over levels, per step"""
    out = {}
    for r in prof:
        if r["kind"].startswith("setup_"):
            out[r["kind"][6:]] = out.get(r["kind"][6:], 0.0) + r["ms"] / steps
    return {k: round(v, 2) for k, v in sorted(out.items(), key=lambda kv: -kv[1])}


def run_ours(args):
    import numpy as np
    import torch

    import gen
    import paper_2602_05686_gb300 as sa

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sa.build()
    kw, desc = WORKLOADS[args.workload]
    p = gen.battery_3d(**kw)
    n = p["n"]
    dev = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda()
           for k in ("row_ptr", "col", "val", "coords", "tensors", "elem_nodes", "elem_measure")}
    dprob = dict(p, **dev)
    b = torch.from_numpy(p["b"]).cuda()
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def one_step(prob, rhs, host=False):
        """returns per-part times (ms, CUDA events) and solve infos"""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        ev[0].record(stream)
        hm = sa.Hierarchy(prob, theta=MAT_THETA, measure="material", precision="fp64", host_inputs=host)
        ev[1].record(stream)
        x64, i64 = hm.solve(rhs, tol=TOL)
        ev[2].record(stream)
        hm.set_precision("fp32")
        ev[3].record(stream)
        x32, i32 = hm.solve(rhs, tol=TOL)
        ev[4].record(stream)
        hm.free()
        hc = sa.Hierarchy(prob, theta=CLS_THETA, measure="classical", precision="fp64", host_inputs=host)
        ev[5].record(stream)
        xc, ic = hc.solve(rhs, tol=TOL)
        ev[6].record(stream)
        st = hc.stats()
        hc.free()
        torch.cuda.synchronize()
        t = [ev[k].elapsed_time(ev[k + 1]) for k in range(6)]
        parts = dict(material_setup_ms=t[0], material_fp64_solve_ms=t[1], fp32_build_ms=t[2],
                     material_fp32_solve_ms=t[3], classical_setup_ms=t[4], classical_fp64_solve_ms=t[5])
        return parts, dict(fp64=i64, fp32=i32, classical=ic), st

    # warm-up
    for _ in range(args.warmup):
        one_step(dprob, b)
    # timed region (device-resident inputs): the production path -- CG loops
    # in CUDA graphs, no per-launch instrumentation
    clk = ClockSampler(local)
    clk.start()
    l0 = sa.launch_count()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    parts_all, infos = [], None
    for _ in range(args.steps):
        parts, infos, _ = one_step(dprob, b)
        parts_all.append(parts)
    t1.record(stream)
    barrier()
    launches = sa.launch_count() - l0
    clocks = clk.stop()
    ms_total = t0.elapsed_time(t1)
    ms_step = ms_total / args.steps
    # the same steps again with every launch bracketed by CUDA events on the
    # library's stream (host-driven CG iterations, so each launch is seen):
    # the per-kernel rows, the roofline and the setup phases come from here
    sa.profile_enable(True)
    barrier()
    t2 = torch.cuda.Event(enable_timing=True)
    t3 = torch.cuda.Event(enable_timing=True)
    t2.record(stream)
    for _ in range(args.steps):
        one_step(dprob, b)
    t3.record(stream)
    barrier()
    prof = sa.profile_read()
    sa.profile_enable(False)
    ms_step_prof = t2.elapsed_time(t3) / args.steps
    ms_step = reduce_over_ranks(ms_step, ws, "max")        # the slowest replica sets the step time
    launches = int(reduce_over_ranks(launches, ws, "sum"))  # kernels of all replicas

    # material hierarchy statistics (untimed)
    hm = sa.Hierarchy(dprob, theta=MAT_THETA, measure="material")
    mst = hm.stats()

    # several right-hand sides on the cached hierarchy: K one-vector solves
    # against one K-column solve (every launch shared), both forms, CUDA events
    multi = None
    if not args.no_multi_rhs:
        # right-hand sides b_c = A x_c of smooth fields x_c (load cases of one
        # stack: the rough N(0,1) loads do not converge on this operator)
        import scipy.sparse as sps
        K = 8
        A = sps.csr_matrix((p["val"], p["col"], p["row_ptr"]), shape=(n, n))
        X3 = p["coords"].reshape(-1, 3)
        zn = (X3[:, 2] - X3[:, 2].min()) / np.ptp(X3[:, 2])
        Bk = torch.from_numpy(np.stack([A @ (np.sin(np.pi * (c + 1) * zn) * (1.0 + 0.25 * c * X3[:, 0]))
                                        for c in range(K)])).cuda()
        del A
        multi = {"rhs": K}
        for form in ("fp64", "fp32"):
            hm.set_precision(form)
            hm.solve(Bk[0].clone())    # warm (graph capture, buffers)
            hm.solve_batch(Bk[:2])
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            its1 = [hm.solve(Bk[c].clone())[1]["iters"] for c in range(K)]
            e[1].record(stream)
            _, inf = hm.solve_batch(Bk)
            e[2].record(stream)
            torch.cuda.synchronize()
            t1, tk = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
            multi[form] = {"one_by_one_ms": round(t1, 2), "block_ms": round(tk, 2),
                           "speedup": round(t1 / tk, 3), "iters": [i["iters"] for i in inf],
                           "iters_equal": its1 == [i["iters"] for i in inf],
                           "max_rel_res": max(i["rel_res"] for i in inf)}
    hm.free()

    # end-to-end through the C ABI with host buffers (copies inside)
    e2e = None
    if not args.no_e2e:
        # the step's inputs in pinned host memory (numpy views of pinned torch
        # tensors), copied to the device inside the timed region
        hkeys = ("row_ptr", "col", "val", "coords", "tensors", "elem_nodes", "elem_measure")
        ph = dict(p, **{k: torch.from_numpy(np.ascontiguousarray(p[k])).pin_memory().numpy() for k in hkeys})
        bh = torch.from_numpy(p["b"].copy()).pin_memory().numpy()
        inb = sum(int(np.asarray(p[k]).nbytes) for k in hkeys)
        barrier()
        te = time.perf_counter()
        for _ in range(max(1, min(args.steps, 2))):
            one_step(ph, bh, host=True)
        barrier()
        e_ms = (time.perf_counter() - te) * 1000.0 / max(1, min(args.steps, 2))
        e2e = {"value": round(e_ms / 1000.0, 4), "unit": "s",
               "h2d_bytes_per_step": 2 * inb + 3 * 2 * n * 8, "d2h_bytes_per_step": 3 * n * 8}

    # roofline of the dominant kernel (largest total time in the timed region):
    # the HBM floor (algorithmic bytes / measured copy bandwidth) and, for the
    # FP64 fine-level kernels, the FP64-pipe floor (algorithmic FLOPs / the FP64
    # peak at the sampled SM clock); the larger floor names the bound
    peak, peak_kind = peaks()
    mhz = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
    fp64_peak = N_SM * FP64_FLOP_PER_SM_CYCLE * mhz * 1e6 / 1e12   # TFLOP/s
    nnz0 = int(p["nnz"])

    def fp64_flops(kind, level):
        """FP64 FLOPs per launch: one FMA per stored entry plus the row updates"""
        if level != 0:
            return None
        per_row = {"cheb64": 5, "resid64": 1, "cg_spmv": 2}.get(kind)
        return None if per_row is None else 2.0 * nnz0 + per_row * n

    rows = sorted(prof, key=lambda r: -r["ms"])
    krows = [r for r in rows if r["bytes"] > 0]   # kernels with an algorithmic-bytes model
    dom = krows[0] if krows else None
    roof = None
    if dom:
        per_launch_ms = dom["ms"] / dom["launches"]
        per_launch_bytes = dom["bytes"] / dom["launches"]
        ach = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
        kname = f"{dom['kind']}_level{dom['level']}"
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": traffic_for(kname, args.workload),
                "kernel": kname, "peak_source": peak_kind, "launches": dom["launches"],
                "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": round(per_launch_ms, 5)}
        fl = fp64_flops(dom["kind"], dom["level"])
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
    # V-cycle bandwidth per form (all V-cycle kernels; algorithmic bytes / time)
    def vgb(kinds):
        sel = [r for r in prof if r["kind"] in kinds]
        ms = sum(r["ms"] for r in sel)
        by = sum(r["bytes"] for r in sel)
        return round(by / (ms * 1e-3) / 1e9, 1) if ms > 0 else None

    vc64 = vgb({"cheb64", "resid64", "restrict64", "prolong64", "first64", "coarse"})
    vc32 = vgb({"cheb32", "resid32", "restrict32", "prolong32", "first32"})
    avg = {k: round(statistics.mean(pp[k] for pp in parts_all), 2) for k in parts_all[0]}

    result = {
        "metric": METRIC, "value": round(ms_step / 1000.0, 4), "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 2), "higher_is_better": False,
        "ms_per_step_instrumented": round(ms_step_prof, 2),
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 inside the mixed V-cycle)",
        "data": "synthetic (seeded generator; paper's battery meshes are not public)",
        "config": workload_config(args, ws),
        "parts_ms": avg,
        "iters": {"material_fp64": infos["fp64"]["iters"], "material_fp32": infos["fp32"]["iters"],
                  "classical_fp64": infos["classical"]["iters"]},
        "rel_res": {k: infos[k]["rel_res"] for k in infos},
        "hierarchy_material": {"levels": mst["levels"], "n": mst["n"], "op_complexity": round(mst["op_complexity"], 3)},
        "vcycle_GBs": {"fp64": vc64, "fp32": vc32},
        "fp32_speedup_vs_fp64_solve": round(avg["material_fp64_solve_ms"] / avg["material_fp32_solve_ms"], 3),
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "kernel_profile_top": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in r.items()}
                               for r in krows[:8]],
        "setup_phases_ms": setup_phases(prof, args.steps),
        "kernel_profile_all": [[r["kind"], r["level"], r["launches"], round(r["ms"], 3)] for r in krows],
        "multi_rhs": multi,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        result["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the oracle (CPU) on a bounded sample
# ---------------------------------------------------------------------------
SAMPLE = dict(nx=48, ny=48, nz=96)


def oracle_step(p):
    """the same step as the GPU arm, run by the serial CPU oracle; seconds"""
    import oracle
    t = time.perf_counter()
    h = oracle.Hierarchy(p, MAT_THETA, "material")
    _, a = h.solve(p["b"], tol=TOL)
    _, f = h.solve(p["b"], tol=TOL, flexible=True)
    del h
    h = oracle.Hierarchy(p, CLS_THETA, "classical")
    _, c = h.solve(p["b"], tol=TOL)
    del h
    return time.perf_counter() - t, (a["iters"], f["iters"], c["iters"])


def cpu_baseline(args, steps=1):
    import gen
    import oracle
    oracle.build()
    p = gen.battery_3d(**SAMPLE)
    full_n = WORKLOADS[args.workload][0]
    nfull = (full_n["nx"] + 1) * (full_n["ny"] + 1) * (full_n["nz"] + 1)
    ts = [oracle_step(p)[0] for _ in range(steps)]
    t = statistics.mean(ts)
    return {"value": round(t * nfull / p["n"], 3), "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"full step on the battery stack 48x48x96 ({p['n']} dofs, {t:.2f} s), scaled by dofs x"
                       f"{nfull / p['n']:.1f} to the {nfull}-dof workload (assumes O(n) cost)")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import gen
    import oracle
    oracle.build()
    p = gen.battery_3d(**SAMPLE)
    kw = WORKLOADS[args.workload][0]
    nfull = (kw["nx"] + 1) * (kw["ny"] + 1) * (kw["nz"] + 1)
    for _ in range(args.warmup):
        oracle_step(p)
    ts, its = [], None
    for _ in range(args.steps):
        t, its = oracle_step(p)
        ts.append(t)
    sec = statistics.mean(ts) * nfull / p["n"]
    out = {"impl": "reference", "metric": METRIC, "value": round(sec, 3), "unit": "s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1000, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator; paper's battery meshes are not public)",
           "config": workload_config(args, ws),
           "iters_sample": {"material_fp64": its[0], "material_flexible": its[1], "classical_fp64": its[2]},
           "cpu_baseline": {"value": round(sec, 3), "unit": "s", "cores": 1, "kind": "oracle",
                            "sample": f"battery stack 48x48x96 ({p["n"]} dofs) per step, scaled by dofs to "
                                      f"{nfull} dofs"},
           "e2e": {"value": round(sec, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_serving(args):
    """Serving workload: seeded Poisson-arrival requests on 2D/3D layered
    operators (contrast 10^U(2,10)), several right-hand sides per operator with
    the hierarchy cached, HBM-admitted, FP32 V-cycle inside FP64 flexible CG.
    The arrival rate is 0.8 x the throughput of a back-to-back warm-up run."""
    import numpy as np
    import torch

    import gen
    from paper_2602_05686_gb300.serving import Request, Server

    torch.cuda.set_device(0)
    nreq = args.requests
    ops, reqs = gen.serving_requests(nreq, seed=11, max2d=args.max2d, max3d=args.max3d)
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
        srv = Server(lambda op: probs[op], options, slots=args.slots, hbm_budget=args.hbm_gb << 30)
        rs, tt = [], 0.0
        for k, r in enumerate(reqs):
            tt += r["gap"] * scale
            rs.append(Request(rid=k, op=r["op"], arrival=tt, rhs=rhs[k]))
        out = srv.serve(rs, realtime=realtime)
        srv.close()
        return out, rs

    warm, _ = run(0.0, False)
    rate = 0.8 * warm["throughput_rps"]
    out, rs = run(1.0 / rate, True)
    iters = [r.info.get("iters", 0) for r in rs]
    res = {"metric": "serving latency p50/p99 (continuous batching, cached hierarchies)",
           "value": round(out["p99_s"], 4), "unit": "s (p99 latency)", "higher_is_better": False,
           "n_gpus": 1, "p50_s": round(out["p50_s"], 4), "p99_s": round(out["p99_s"], 4),
           "throughput_rps": round(out["throughput_rps"], 2), "arrival_rate_rps": round(rate, 2),
           "warmup_throughput_rps": round(warm["throughput_rps"], 2), "requests": nreq, "operators": len(ops),
           "slots": args.slots, "setups": out["setups"], "cache_hits": out["hits"], "evictions": out["evictions"],
           "failed": out["failed"], "mean_iters": round(float(np.mean(iters)), 1),
           "max_rel_res": max(r.info.get("rel_res", 0.0) for r in rs), "generation_s": round(gen_s, 1),
           "config": {"workload": f"serving: {nreq} requests, 2D 16^2..{args.max2d}^2 and 3D 16^3..{args.max3d}^3 "
                                  "layered operators, contrast 1e2..1e10, 1-16 RHS per operator",
                      "precision": "FP32 V-cycle in FP64 flexible CG", "tol": TOL}}
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
    ap.add_argument("--workload", default="battery_128x128x256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-multi-rhs", action="store_true")
    ap.add_argument("--serving", action="store_true", help="run the serving workload instead")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--hbm-gb", type=int, default=64)
    ap.add_argument("--max2d", type=int, default=512)
    ap.add_argument("--max3d", type=int, default=96)
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
