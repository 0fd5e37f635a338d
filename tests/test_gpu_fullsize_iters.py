"""Iteration parity at full size: the GPU's FP64 PCG iteration counts on the
full-size workloads against the CPU oracle's (tests/golden/fullsize_iters.json,
written by tests/golden/make_fullsize_iters.py from the oracle alone), within
one iteration, and the true residual at 1e-8.  The battery stack with the
material measure is left out of the bar: its count is not a stable quantity
of the method (the oracle alone gives 81 to 158 iterations when the input is
moved by one ulp; the outlier eigenvalues behind it are measured in the design
notes), so the test only checks that the GPU reaches the residual there."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "fullsize_iters.json")))
UNSTABLE = {("battery_128x128x256", "material_0.05")}


@pytest.fixture(scope="module")
def sa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_05686_gb300 as m
    m.build()
    return m


def problem(gen_mod, name):
    return {"layered_2d_32": lambda: gen_mod.layered_2d(32),
            "battery_128x128x256": lambda: gen_mod.battery_3d(128, 128, 256),
            "voronoi_160": lambda: gen_mod.voronoi_3d(160),
            "inclusions_320": lambda: gen_mod.inclusions_3d(320, nrhs=1)}[name]()


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_fullsize_iterations_within_one(sa, gen_mod, name):
    import torch
    p = problem(gen_mod, name)
    b = torch.from_numpy(np.ascontiguousarray(p["B"][0] if "B" in p else p["b"])).cuda()
    dp = dict(p, **{k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda()
                    for k in ("row_ptr", "col", "val", "coords", "tensors", "elem_nodes", "elem_measure")})
    for key, ref in GOLDEN[name].items():
        m, theta = key.rsplit("_", 1)
        h = sa.Hierarchy(dp, theta=float(theta), measure=m, precision="fp64", max_coarse=ref["max_coarse"])
        assert h.stats()["levels"] == ref["levels"], (name, key)
        _, info = h.solve(b, tol=1e-8)
        h.free()
        assert info["status"] == 0 and info["rel_res"] <= 1e-8, (name, key, info)
        if (name, key) in UNSTABLE:
            continue
        assert abs(info["iters"] - ref["iters"]) <= 1, (name, key, info["iters"], ref["iters"])
