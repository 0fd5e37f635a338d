"""Multi-right-hand-side solves (sa_solve_batch): up to 8 columns share every
launch of the operator products, the V-cycle and the CG updates.  Each column
follows the one-vector solve's arithmetic in the same order, so it must end
bitwise where sa_solve on that right-hand side ends: same iteration count,
same status, identical x -- in both solve forms, for blocks of 2..8 columns,
for more than 8 columns (split into blocks), with a zero right-hand side in the
mix and with host buffers."""
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


def rhs(p, k, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((k, p["n"]))
    B[:, p["dir_mask"] == 1] = 0.0
    return B


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [2, 5, 8, 11])
def test_block_columns_equal_single_solves(sa, gen_mod, precision, k):
    import torch
    p = gen_mod.battery_3d(16, 16, 32)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=200, precision=precision)
    B = rhs(p, k, 7 + k)
    B[1] = 0.0                       # a zero right-hand side: done before the first iteration
    Bd = torch.from_numpy(B).cuda()
    X, infos = h.solve_batch(Bd)
    for c in range(k):
        x1, i1 = h.solve(Bd[c].clone())
        assert infos[c]["status"] == i1["status"] and infos[c]["iters"] == i1["iters"], (c, infos[c], i1)
        assert torch.equal(X[c], x1), c
        assert infos[c]["rel_res"] == i1["rel_res"]
    assert infos[1]["iters"] == 0 and not torch.any(X[1])


def test_block_mixed_operators_and_layers(sa, gen_mod):
    """different convergence speeds in one block (a right-hand side close to
    a smooth mode next to rough ones) and a CSR-vector coarse hierarchy
    (voronoi), FP32 form"""
    import torch
    p = gen_mod.voronoi_3d(14, seed=1)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=150, precision="fp32")
    B = rhs(p, 4, 3)
    B[2] = p["b"]
    Bd = torch.from_numpy(B).cuda()
    X, infos = h.solve_batch(Bd)
    its = [i["iters"] for i in infos]
    for c in range(4):
        x1, i1 = h.solve(Bd[c].clone())
        assert infos[c]["iters"] == i1["iters"] and torch.equal(X[c], x1)
        assert infos[c]["rel_res"] <= 1e-8
    assert len(set(its)) >= 1


def test_block_host_buffers(sa, gen_mod):
    p = gen_mod.battery_3d(12, 12, 24)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=100)
    B = rhs(p, 3, 5)
    X, infos = h.solve_batch(B)
    assert isinstance(X, np.ndarray)
    for c in range(3):
        x1, i1 = h.solve(B[c].copy())
        assert infos[c]["iters"] == i1["iters"] and np.array_equal(X[c], x1)


def test_block_rejects_bad_arguments(sa, gen_mod):
    import ctypes
    p = gen_mod.battery_3d(8, 8, 16)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=50)
    infos = (sa.SolveInfo * 2)()
    assert sa.lib().sa_solve_batch(h.h, 2, None, None, 1e-8, infos) == -1
    assert sa.lib().sa_solve_batch(h.h, -1, None, None, 1e-8, infos) == -1
    del ctypes


@pytest.mark.parametrize("n_el,k", [(96, 3), (96, 8), (200, 8)])
def test_block_fp32_staged_sell_level_equals_single_solves(sa, gen_mod, n_el, k):
    """The FP32 several-column kernels of a one-lane SELL level with slices at
    most 32 entries wide (levels of 2^19 rows and more: here the inclusions'
    fine level, 27-entry rows) stage each slice's values and columns in shared
    memory with bulk copies on an mbarrier; the columns of the block solve
    still end bitwise where the one-vector solves end.  96^3 stores 16-bit
    column offsets (slice spans below 2^16), 200^3 32-bit columns (a plane of
    201^2 rows makes the span 2 x 40401)."""
    import torch
    p = gen_mod.inclusions_3d(n_el)
    h = sa.Hierarchy(p, theta=0.04, measure="classical", precision="fp32")
    f0 = h.level_format(0)
    assert f0["lanes"] == 0 and f0["sell_lanes"] == 1 and p["n"] >= 1 << 19
    B = rhs(p, k, 31 + k)
    Bd = torch.from_numpy(B).cuda()
    X, infos = h.solve_batch(Bd)
    for c in range(k):
        x1, i1 = h.solve(Bd[c].clone())
        assert infos[c]["iters"] == i1["iters"] and infos[c]["status"] == i1["status"] == 0
        assert torch.equal(X[c], x1), c
    h.free()
