"""Writes fullsize_iters.json: the CPU oracle's FP64 PCG iteration counts on
the full-size workloads (layered square 32x32, battery stack 128x128x256,
Voronoi cube 160^3, inclusions 320^3 with its first right-hand side), the
reference for the full-size iteration-parity GPU test.  Calls only oracle/
and gen/ (about ten minutes on one core).  Usage:

    python tests/golden/make_fullsize_iters.py [names...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402

# name: (generator, kwargs, [(measure, theta, max_coarse)])
CASES = {
    "layered_2d_32": ("layered_2d", dict(n_el=32), [("material", 0.08, 64), ("classical", 0.08, 64)]),
    "battery_128x128x256": ("battery_3d", dict(nx=128, ny=128, nz=256), [("classical", 0.04, 5000),
                                                                           ("material", 0.05, 5000)]),
    "voronoi_160": ("voronoi_3d", dict(n_el=160), [("material", 0.05, 5000), ("classical", 0.04, 5000)]),
    "inclusions_320": ("inclusions_3d", dict(n_el=320), [("classical", 0.04, 5000)]),
}


def run(name):
    fn, kw, forms = CASES[name]
    p = getattr(gen, fn)(**kw)
    b = p["B"][0] if "B" in p else p["b"]
    out = {}
    for (m, theta, mc) in forms:
        t = time.time()
        h = oracle.Hierarchy(p, theta, m, max_coarse=mc)
        _, info = h.solve(b, tol=1e-8)
        out[f"{m}_{theta}"] = dict(iters=info["iters"], status=info["status"], rel_res=info["rel_res"],
                                   levels=h.nlev, max_coarse=mc, seconds=round(time.time() - t, 1))
        del h
    return out


def main():
    gen.build()
    oracle.build()
    names = sys.argv[1:] or list(CASES)
    path = os.path.join(HERE, "fullsize_iters.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        data[name] = run(name)
        json.dump(data, open(path, "w"), indent=1, sort_keys=True)
        print(name, data[name], flush=True)


if __name__ == "__main__":
    main()
