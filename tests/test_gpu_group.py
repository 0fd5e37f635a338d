"""Group solves (sa_solve_group): problems with different operators, one
right-hand side each, advanced together -- every operator product, V-cycle
kernel (the coarse solves of all problems together) and CG update is one
launch for all problems still iterating.  Each problem follows the one-vector
solve's arithmetic, so it must end bitwise where sa_solve on its handle ends:
same iterations, same status, identical x -- in both forms, for groups of
different hierarchy depths (one-level problems included), for any subset
(alone = in the mix), with a zero right-hand side and with a problem that hits
maxit while the others converge."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_05686_gb300 as m
    m.build()
    return m


def problems(gen_mod):
    return [
        (gen_mod.layered_2d(48, contrast=1e-4), dict(theta=0.08, measure="material", max_coarse=64)),
        (gen_mod.battery_3d(12, 12, 24), dict(theta=0.05, measure="material", max_coarse=200)),
        (gen_mod.voronoi_3d(12, nseeds=6, seed=4), dict(theta=0.04, measure="classical", max_coarse=120)),
        (gen_mod.inclusions_3d(16, rmin=2.0, rmax=4.0, nrhs=1), dict(theta=0.04, measure="classical",
                                                                      max_coarse=300)),
        # one level: the whole problem is the dense coarse solve
        (gen_mod.layered_2d(10), dict(theta=0.08, measure="material", max_coarse=500)),
        (gen_mod.two_domain(40, 1e4), dict(theta=0.08, measure="material", max_coarse=100, drop="cut")),
    ]


def build(sa, gen_mod, precision):
    import torch
    hs, bs = [], []
    for k, (p, kw) in enumerate(problems(gen_mod)):
        h = sa.Hierarchy(p, precision="fp64", **kw)
        if precision == "fp32":
            h.set_precision("fp32")
        rng = np.random.default_rng(100 + k)
        b = rng.standard_normal(p["n"])
        b[p["dir_mask"] == 1] = 0.0
        hs.append(h)
        bs.append(torch.from_numpy(b).cuda())
    return hs, bs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_group_equals_single_solves(sa, gen_mod, precision):
    import torch
    hs, bs = build(sa, gen_mod, precision)
    levels = [h.stats()["levels"] for h in hs]
    assert 1 in levels and max(levels) >= 3            # depths differ inside the group
    X, infos = sa.solve_group(hs, bs)
    for k, h in enumerate(hs):
        x1, i1 = h.solve(bs[k].clone())
        assert infos[k]["status"] == i1["status"] == 0, (k, infos[k], i1)
        assert infos[k]["iters"] == i1["iters"], (k, infos[k], i1)
        assert infos[k]["rel_res"] == i1["rel_res"] and i1["rel_res"] <= 1e-8
        assert torch.equal(X[k], x1), k
    for h in hs:
        h.free()


def test_alone_equals_in_the_mix_for_every_subset(sa, gen_mod):
    import torch
    hs, bs = build(sa, gen_mod, "fp32")
    full, _ = sa.solve_group(hs, bs)
    for sub in ([0], [3], [4], [1, 5], [5, 2, 0], [4, 1, 3, 2]):
        Xs, infos = sa.solve_group([hs[k] for k in sub], [bs[k] for k in sub])
        for j, k in enumerate(sub):
            assert torch.equal(Xs[j], full[k]), (sub, k)
    for h in hs:
        h.free()


def test_group_zero_rhs_and_maxit(sa, gen_mod):
    import torch
    hs, bs = build(sa, gen_mod, "fp64")
    bs[2] = torch.zeros_like(bs[2])
    X, infos = sa.solve_group(hs, bs)
    assert infos[2]["iters"] == 0 and infos[2]["status"] == 0 and not torch.any(X[2])
    # a hierarchy that stops at 3 iterations next to ones that converge
    p, kw = problems(gen_mod)[1]
    short = sa.Hierarchy(p, precision="fp64", maxit=3, **kw)
    others = [sa.Hierarchy(q, precision="fp64", maxit=3, **k2) for (q, k2) in problems(gen_mod)[:1]]
    X, infos = sa.solve_group([short] + others, [bs[1], bs[0]], check=False)
    x1, i1 = short.solve(bs[1].clone(), check=False)
    assert infos[0]["status"] == i1["status"] and infos[0]["iters"] == i1["iters"] == 3
    assert torch.equal(X[0], x1)
    for h in hs + [short] + others:
        h.free()


def test_group_rejects_duplicates_and_mixed_settings(sa, gen_mod):
    import torch
    hs, bs = build(sa, gen_mod, "fp64")
    L = sa.lib()
    h2 = (ctypes.c_void_p * 2)(hs[0].h.value, hs[0].h.value)
    b2 = (ctypes.c_void_p * 2)(bs[0].data_ptr(), bs[0].data_ptr())
    x = [torch.zeros_like(bs[0]) for _ in range(2)]
    x2 = (ctypes.c_void_p * 2)(x[0].data_ptr(), x[1].data_ptr())
    assert L.sa_solve_group(2, h2, b2, x2, 1e-8, None) == -1
    assert b"twice" in L.sa_last_error()
    hs[1].set_precision("fp32")
    with pytest.raises(Exception):
        sa.solve_group(hs[:2], bs[:2])
    assert L.sa_solve_group(0, None, None, None, 1e-8, None) == 0
    for h in hs:
        h.free()


def test_group_with_host_buffers(sa, gen_mod):
    """right-hand sides and solutions in host memory (copied inside the call)"""
    import torch
    hs, bs = build(sa, gen_mod, "fp64")
    sub = [0, 2, 4]
    B = [bs[k].cpu().numpy().copy() for k in sub]
    X = [np.zeros_like(b) for b in B]
    L = sa.lib()
    m = len(sub)
    hp = (ctypes.c_void_p * m)(*[hs[k].h.value for k in sub])
    bp = (ctypes.c_void_p * m)(*[b.ctypes.data for b in B])
    xp = (ctypes.c_void_p * m)(*[x.ctypes.data for x in X])
    infos = (sa.SolveInfo * m)()
    assert L.sa_solve_group(m, hp, bp, xp, 1e-8, infos) == 0
    Xd, _ = sa.solve_group([hs[k] for k in sub], [bs[k] for k in sub])
    for j in range(m):
        assert np.array_equal(X[j], Xd[j].cpu().numpy()) and infos[j].status == 0
    for h in hs:
        h.free()
