"""Drop-tolerance sweep of the paper's two-domain study (Sec. 4.1): for each
strength measure (classical S^sa, distance Laplacian S^dlap, material-aware
S^dlap_sigma) and each theta, build the hierarchy, solve with PCG to 1e-8
and record iterations, levels, operator complexity C and the cost C x
iterations.  Configurations that stagnate or fail to converge are reported
with their status (the paper omits them from its plots)."""
from __future__ import annotations

THETAS = (0.0, 0.0025, 0.005, 0.01, 0.02, 0.04, 0.08, 0.16, 0.32, 0.64)
MEASURES = ("classical", "distance", "material")


def theta_sweep(problem, thetas=THETAS, measures=MEASURES, max_coarse=64, precision="fp64", maxit=500,
                drops=("pointwise",)):
    import torch

    from .api import Hierarchy, SAError
    b = torch.from_numpy(problem["b"]).cuda()
    rows = []
    for d in drops:
        for m in measures:
            for th in thetas:
                row = dict(measure=m, theta=th, drop=d)
                try:
                    h = Hierarchy(problem, theta=th, measure=m, max_coarse=max_coarse, precision=precision,
                                  maxit=maxit, drop=d)
                except SAError as e:
                    row.update(status=e.status, iters=None, levels=None, op_complexity=None, cost=None)
                    rows.append(row)
                    continue
                st = h.stats()
                _, info = h.solve(b)
                h.free()
                ok = info["status"] == 0
                row.update(status=info["status"], iters=info["iters"], levels=st["levels"],
                           op_complexity=st["op_complexity"],
                           cost=st["op_complexity"] * info["iters"] if ok else None)
                rows.append(row)
    return rows


# the annulus study of Sec. 4.2 (Table 1): refinements h .. h/16 of the
# 20 x 150 x 1 base mesh, contrast kappa in {1, ..., 1e4}, material measure
# with pointwise dropping at theta in {0.05, 0.1}, coarsening to <= 5000
ANNULUS_KAPPAS = (1.0, 10.0, 100.0, 1e3, 1e4)
ANNULUS_THETAS = (0.05, 0.1)


def annulus_study(make_problem, refines=(0, 1, 2, 3, 4), kappas=ANNULUS_KAPPAS, thetas=ANNULUS_THETAS,
                  precision="fp64", max_coarse=5000, maxit=500, tol=1e-8):
    """make_problem(refine, kappa) -> problem dict (the annulus generator).
    Returns one row per (refine, kappa, theta): iterations, levels, operator
    complexity, setup and solve times (CUDA events on the handle's stream)."""
    import torch

    from .api import Hierarchy, SAError
    rows = []
    for rf in refines:
        for k in kappas:
            p = make_problem(rf, k)
            b = torch.from_numpy(p["b"]).cuda()
            for th in thetas:
                row = dict(refine=rf, n=int(p["n"]), kappa=k, theta=th)
                s = torch.cuda.current_stream()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(s)
                try:
                    h = Hierarchy(p, theta=th, measure="material", max_coarse=max_coarse, precision=precision,
                                  maxit=maxit)
                except SAError as e:
                    row.update(status=e.status)
                    rows.append(row)
                    continue
                e1.record(s)
                _, info = h.solve(b, tol=tol)
                e2.record(s)
                st = h.stats()
                h.free()
                torch.cuda.synchronize()
                row.update(status=info["status"], iters=info["iters"], rel_res=info["rel_res"],
                           levels=st["levels"], op_complexity=round(st["op_complexity"], 3),
                           setup_ms=round(e0.elapsed_time(e1), 2), solve_ms=round(e1.elapsed_time(e2), 2))
                rows.append(row)
    return rows
