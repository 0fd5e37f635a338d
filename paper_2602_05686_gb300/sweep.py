"""Drop-tolerance sweep of the paper's two-domain study (Sec. 4.1): for each
strength measure (classical S^sa, distance Laplacian S^dlap, material-aware
S^dlap_sigma) and each theta, build the hierarchy, solve with PCG to 1e-8
and record iterations, levels, operator complexity C and the cost C x
iterations.  Configurations that stagnate or fail to converge are reported
with their status (the paper omits them from its plots)."""
from __future__ import annotations

THETAS = (0.0, 0.0025, 0.005, 0.01, 0.02, 0.04, 0.08, 0.16, 0.32, 0.64)
MEASURES = ("classical", "distance", "material")


def theta_sweep(problem, thetas=THETAS, measures=MEASURES, max_coarse=64, precision="fp64", maxit=500):
    import torch

    from .api import Hierarchy, SAError
    b = torch.from_numpy(problem["b"]).cuda()
    rows = []
    for m in measures:
        for th in thetas:
            row = dict(measure=m, theta=th)
            try:
                h = Hierarchy(problem, theta=th, measure=m, max_coarse=max_coarse, precision=precision, maxit=maxit)
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
