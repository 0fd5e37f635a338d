"""Parity at the benchmark's full size (battery stack 128 x 128 x 256,
4,276,737 dofs, 113M stored entries) and on the rotated-anisotropy Voronoi
workload (160^3 elements): the fine-level setup of the CUDA path, in the
configuration bench.py times, against the oracle's step functions run on the
same inputs: strength masks, filtered graph, MIS-2 roots and aggregates
bit-exact; the smoothed prolongator and the first coarse operator within
1e-12 of the row's largest magnitude; and a converged solve (properties at any
size: true relative residual <= 1e-8)."""
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


def _rowrel(rp, a, b):
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    scale = np.zeros(n)
    np.maximum.at(scale, rows, np.abs(b))
    return float((np.abs(a - b) / np.maximum(scale[rows], 1e-300)).max()) if len(a) else 0.0


CASES = [("battery-material", "battery", 0.05, "material"), ("battery-classical", "battery", 0.04, "classical"),
         ("voronoi-material", "voronoi", 0.05, "material")]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fine_level_setup_parity_full_size(sa, orc, gen_mod, case):
    import torch
    _, which, theta, measure = case
    p = gen_mod.battery_3d() if which == "battery" else gen_mod.voronoi_3d(160)
    n, rp, ci, v = p["n"], p["row_ptr"], p["col"], p["val"]
    h = sa.Hierarchy(p, theta=theta, measure=measure, keep_setup_data=True)
    g0 = h.export_level(0)
    s0 = h.export_strength(0, keep=True, root=True, aux=False)
    # oracle steps on the same inputs
    dm = orc.dirichlet(n, rp, ci, v)
    assert np.array_equal(dm, s0["dir"])
    if measure == "classical":
        keep = orc.strength_classical(n, rp, ci, v, dm, theta)
    else:
        sig = orc.nodal_from_elements(3, n, p["elem_nodes"], p["elem_measure"], p["tensors"])
        sinv = orc.invert_tensors(3, sig)
        keep = orc.strength_material(3, n, rp, ci, dm, p["coords"], sinv, theta)[2]
    assert np.array_equal(keep, s0["keep"])
    grp, gci = orc.filtered_graph(n, rp, ci, keep, dm)
    assert g0["nnz_gc"] == len(gci)
    root = orc.mis2(n, grp, gci, dm, 0, 0)
    assert np.array_equal(root, s0["root"])
    nc, agg = orc.aggregate(n, grp, gci, dm, root)
    assert nc == g0["nc"] and np.array_equal(agg, g0["agg"])
    F, Dt = orc.filter_matrix(n, rp, ci, v, keep)
    lam = orc.power_estimate(F, np.where(np.isfinite(Dt), 1.0 / np.sqrt(Dt), 0.0), 10, 1, 0)
    omega = 4.0 / 3.0 / lam if lam > 0 else 0.0
    assert s0["omega"] == pytest.approx(omega, rel=1e-12)
    P = orc.smooth_prolongator(F, Dt, omega, agg, nc)
    assert np.array_equal(P["row_ptr"], g0["P_rp"]) and np.array_equal(P["col"], g0["P_ci"])
    assert _rowrel(P["row_ptr"], g0["P_v"], P["val"]) <= 1e-12
    A1 = orc.galerkin(dict(nrows=n, ncols=n, row_ptr=rp, col=ci, val=v), P)
    g1 = h.export_level(1)
    assert np.array_equal(A1["row_ptr"], g1["A_rp"]) and np.array_equal(A1["col"], g1["A_ci"])
    assert _rowrel(A1["row_ptr"], g1["A_v"], A1["val"]) <= 1e-12
    # the solve converges at this size (FP64 and the FP32 V-cycle form)
    b = torch.from_numpy(p["b"]).cuda()
    _, i64 = h.solve(b)
    h.set_precision("fp32")
    _, i32 = h.solve(b)
    assert i64["status"] == 0 and i64["rel_res"] <= 1e-8
    assert i32["status"] == 0 and i32["rel_res"] <= 1e-8


def test_cut_drop_mask_full_size(sa, orc, gen_mod):
    """cut-drop (Sec. 2.1, the paper's recommended criterion with the material
    measure at theta = 0.08) on the full battery stack: the fine-level kept
    mask equals the oracle's on the same inputs, bit for bit"""
    p = gen_mod.battery_3d()
    n, rp, ci = p["n"], p["row_ptr"], p["col"]
    h = sa.Hierarchy(p, theta=0.08, measure="material", keep_setup_data=True, drop="cut")
    s0 = h.export_strength(0, keep=True, root=False, aux=False)
    dm = orc.dirichlet(n, rp, ci, p["val"])
    sig = orc.nodal_from_elements(3, n, p["elem_nodes"], p["elem_measure"], p["tensors"])
    sinv = orc.invert_tensors(3, sig)
    w, D, _ = orc.strength_material(3, n, rp, ci, dm, p["coords"], sinv, 0.08)
    keep = orc.cut_drop(n, rp, ci, dm, orc.strength2_material(n, rp, ci, w, D), 0.08)
    assert np.array_equal(keep, s0["keep"])


def test_multi_rhs_columns_full_size(sa, gen_mod):
    """two load cases on the full battery stack in one multi-RHS solve, FP32
    V-cycle form: each column equals its one-vector solve bitwise"""
    import torch
    p = gen_mod.battery_3d()
    h = sa.Hierarchy(p, theta=0.05, measure="material", precision="fp32")
    b = torch.from_numpy(p["b"]).cuda()
    B = torch.stack([b, 3.0 * b])
    X, infos = h.solve_batch(B)
    for c in range(2):
        x1, i1 = h.solve(B[c].clone())
        assert infos[c]["iters"] == i1["iters"] and torch.equal(X[c], x1)
        assert infos[c]["status"] == 0 and infos[c]["rel_res"] <= 1e-8
