"""CUDA path vs the CPU oracle, level by level and solve by solve.

Bar: aggregates, roots, strength masks and sparsity patterns bit-exact;
FP64 hierarchy values within 1e-12 of the row's largest magnitude; CG
iteration counts within 1 and true relative residual <= 1e-8 (FP64 form);
the FP32 V-cycle form reaches the same residual within a few extra
iterations."""
import numpy as np
import pytest
from _tol import VAL_TOL, chain_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_05686_gb300 as m
    m.build()
    return m


def row_rel_close(rp, a, b, tol=VAL_TOL):
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    scale = np.zeros(n)
    np.maximum.at(scale, rows, np.abs(b))
    err = np.abs(a - b)
    bad = err > tol * np.maximum(scale[rows], 1e-300)
    return not bad.any(), (float((err / np.maximum(scale[rows], 1e-300)).max()) if len(a) else 0.0)


def stepwise(orc, g, s, l, omega_gpu):
    """This level's steps in the oracle on the CUDA path's own A_l, strength
    mask and aggregates: the filtered matrix and 1-norm diagonal (Sec. 2.3),
    omega from 10 power steps (tag 2l+1), P = P^ - omega D~^-1 A_F P^, then
    the Galerkin product with the CUDA path's own P_l.  Identical inputs, so
    the bar is the plain 1e-12 of the row's largest magnitude."""
    n = g["n"]
    F, Dt = orc.filter_matrix(n, g["A_rp"], g["A_ci"], g["A_v"], s["keep"])
    lam = orc.power_estimate(F, np.where(np.isfinite(Dt), 1.0 / np.sqrt(Dt), 0.0), 10, 2 * l + 1, 0)
    om = 4.0 / 3.0 / lam if lam > 0 else 0.0
    assert omega_gpu == pytest.approx(om, rel=1e-12), l
    P = orc.smooth_prolongator(F, Dt, om, g["agg"], g["nc"])
    assert np.array_equal(P["row_ptr"], g["P_rp"]) and np.array_equal(P["col"], g["P_ci"]), l
    ok, e = row_rel_close(P["row_ptr"], g["P_v"], P["val"])
    assert ok, ("stepwise P", l, e)
    Pg = dict(nrows=n, ncols=g["nc"], row_ptr=g["P_rp"], col=g["P_ci"], val=g["P_v"])
    return orc.galerkin(dict(nrows=n, ncols=n, row_ptr=g["A_rp"], col=g["A_ci"], val=g["A_v"]), Pg)


def compare(h, o, keep=True, orc=None):
    st = h.stats()
    assert st["levels"] == o.nlev, (st["n"], [o.level(l)["n"] for l in range(o.nlev)])
    worst = 0.0
    A_next = None
    for l in range(o.nlev):
        g, r = h.export_level(l), o.level(l)
        assert g["n"] == r["n"] and g["nnz"] == r["nnz"], (l, g["n"], r["n"], g["nnz"], r["nnz"])
        assert np.array_equal(g["A_rp"], r["A_rp"]) and np.array_equal(g["A_ci"], r["A_ci"]), l
        ok, e = row_rel_close(r["A_rp"], g["A_v"], r["A_v"], chain_tol(l))
        worst = max(worst, e)
        assert ok, ("chained A", l, e)
        if A_next is not None:
            assert np.array_equal(A_next["row_ptr"], g["A_rp"]) and np.array_equal(A_next["col"], g["A_ci"]), l
            ok, e = row_rel_close(g["A_rp"], g["A_v"], A_next["val"])
            assert ok, ("stepwise A", l, e)
        if l < o.nlev - 1:
            assert np.array_equal(g["agg"], r["agg"]), l
            assert g["nnz_gc"] == r["nnz_gc"], l
            assert np.array_equal(g["P_rp"], r["P_rp"]) and np.array_equal(g["P_ci"], r["P_ci"]), l
            ok, e = row_rel_close(r["P_rp"], g["P_v"], r["P_v"], chain_tol(l))
            worst = max(worst, e)
            assert ok, ("chained P", l, e)
            if keep:
                s = h.export_strength(l, keep=True, root=True, aux=False)
                assert np.array_equal(s["keep"], r["keep"]), l
                assert np.array_equal(s["root"], r["root"]), l
                assert s["omega"] == pytest.approx(r["omega"], rel=chain_tol(l)), l
                assert s["cheb_lmax"] == pytest.approx(r["cheb_lmax"], rel=chain_tol(l)), l
                if orc is not None:
                    A_next = stepwise(orc, g, s, l, s["omega"])
    return worst


CASES = [
    ("c1-material", lambda g: g.layered_2d(32), 0.08, "material", 64),
    ("c1-classical", lambda g: g.layered_2d(32), 0.08, "classical", 64),
    ("c1-distance", lambda g: g.layered_2d(32), 0.08, "distance", 64),
    ("twodomain-material", lambda g: g.two_domain(32, 1e4), 0.08, "material", 64),
    ("twodomain-classical", lambda g: g.two_domain(32, 1e4), 0.08, "classical", 64),
    ("battery-material", lambda g: g.battery_3d(16, 16, 32), 0.05, "material", 200),
    ("battery-classical", lambda g: g.battery_3d(16, 16, 32), 0.04, "classical", 200),
    ("voronoi-material", lambda g: g.voronoi_3d(14, seed=1), 0.05, "material", 150),
    ("voronoi-classical", lambda g: g.voronoi_3d(14, seed=1), 0.04, "classical", 150),
    ("inclusions-material", lambda g: g.inclusions_3d(20, nrhs=1), 0.05, "material", 200),
    ("inclusions-classical", lambda g: g.inclusions_3d(20, nrhs=1), 0.04, "classical", 200),
    ("annulus-material-0.05", lambda g: g.annulus_3d(0, kappa=1e4), 0.05, "material", 500),
    ("annulus-material-0.1", lambda g: g.annulus_3d(0, kappa=1e4), 0.1, "material", 500),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_hierarchy_parity(sa, orc, gen_mod, case):
    _, mk, theta, measure, mc = case
    p = mk(gen_mod)
    h = sa.Hierarchy(p, theta=theta, measure=measure, max_coarse=mc, keep_setup_data=True)
    o = orc.Hierarchy(p, theta, measure, max_coarse=mc)
    assert o.nlev >= 2
    compare(h, o, orc=orc)
    if measure != "classical":
        for l in range(o.nlev):
            s = h.export_strength(l, keep=False, root=False, aux=True)
            r = o.level(l)
            assert np.array_equal(s["x"], r["x"]) and np.array_equal(s["sinv"], r["sinv"]), l


CUT_CASES = [
    ("c1-material-cut", lambda g: g.layered_2d(32), 0.08, "material", 64),
    ("twodomain-classical-cut", lambda g: g.two_domain(32, 1e4), 0.08, "classical", 64),
    ("twodomain-material-cut", lambda g: g.two_domain(32, 1e4), 0.08, "material", 64),
    ("battery-material-cut", lambda g: g.battery_3d(16, 16, 32), 0.08, "material", 200),
    ("voronoi-classical-cut", lambda g: g.voronoi_3d(14, seed=1), 0.08, "classical", 150),
    ("voronoi-material-cut", lambda g: g.voronoi_3d(14, seed=1), 0.08, "material", 150),
]


@pytest.mark.parametrize("case", CUT_CASES, ids=[c[0] for c in CUT_CASES])
def test_hierarchy_parity_cut_drop(sa, orc, gen_mod, case):
    import torch
    _, mk, theta, measure, mc = case
    p = mk(gen_mod)
    h = sa.Hierarchy(p, theta=theta, measure=measure, max_coarse=mc, keep_setup_data=True, drop="cut")
    o = orc.Hierarchy(p, theta, measure, max_coarse=mc, drop="cut")
    assert o.nlev >= 2
    compare(h, o, orc=orc)
    x, info = h.solve(torch.from_numpy(p["b"]).cuda())
    _, oinfo = o.solve(p["b"])
    assert info["status"] == 0 and abs(info["iters"] - oinfo["iters"]) <= 1


SOLVE_CASES = CASES[:2] + CASES[5:8] + CASES[9:11]


@pytest.mark.parametrize("case", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
def test_solve_parity_fp64(sa, orc, gen_mod, case):
    import torch
    _, mk, theta, measure, mc = case
    p = mk(gen_mod)
    h = sa.Hierarchy(p, theta=theta, measure=measure, max_coarse=mc)
    o = orc.Hierarchy(p, theta, measure, max_coarse=mc)
    x, info = h.solve(torch.from_numpy(p["b"]).cuda(), tol=1e-8)
    xo, oinfo = o.solve(p["b"], tol=1e-8)
    assert info["status"] == 0 and oinfo["status"] == 0
    assert info["rel_res"] <= 1e-8
    assert abs(info["iters"] - oinfo["iters"]) <= 1, (info, oinfo)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


@pytest.mark.parametrize("case", SOLVE_CASES[:5], ids=[c[0] for c in SOLVE_CASES[:5]])
def test_solve_mixed_precision(sa, orc, gen_mod, case):
    import torch
    _, mk, theta, measure, mc = case
    p = mk(gen_mod)
    h = sa.Hierarchy(p, theta=theta, measure=measure, max_coarse=mc, precision="fp32")
    o = orc.Hierarchy(p, theta, measure, max_coarse=mc)
    x, info = h.solve(torch.from_numpy(p["b"]).cuda(), tol=1e-8)
    xo, oinfo = o.solve(p["b"], tol=1e-8, flexible=True)
    assert info["status"] == 0, info
    assert info["rel_res"] <= 1e-8
    assert info["iters"] <= oinfo["iters"] + 3, (info, oinfo)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


def test_vcycle_matches_oracle(sa, orc, gen_mod):
    import torch
    p = gen_mod.battery_3d(16, 16, 32)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=200)
    o = orc.Hierarchy(p, 0.05, "material", max_coarse=200)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(p["n"])
    zg = h.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = o.vcycle(r)
    assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)
    hm = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=200, precision="fp32")
    zm = hm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.linalg.norm(zm - zo) <= 1e-3 * np.linalg.norm(zo)


@pytest.mark.parametrize("sig", [(1e2, 1e-2, 1.0), (1e3, 1e-3, 10.0)])
def test_vcycle_long_row_bin_matches_oracle(sa, orc, gen_mod, sig):
    """On the 48x48x96 battery stack with these layer conductivities, coarse
    levels hold rows far longer than the rest (up to 150 and 490 entries
    against averages near 30-45): they are stored as CSR, the outlier rows
    -- longer than max(64, 4 x the mean row length rounded up) -- in a
    long-row bin (a warp per row), exactly those rows.  The V-cycle over them
    equals the oracle's, and a block solve's columns equal the one-vector
    solves bitwise."""
    import torch
    import scipy.sparse as sp
    p = gen_mod.battery_3d(48, 48, 96, sig=sig)
    h = sa.Hierarchy(p, theta=0.05, measure="material")
    nlev = h.stats()["levels"]
    fm = [h.level_format(l) for l in range(nlev)]
    assert fm[0]["lanes"] == 0 and fm[-1]["lanes"] == -1
    binned = 0
    for l, f in enumerate(fm):
        if f["lanes"] <= 0:
            continue
        assert f["lanes"] == 4
        s = h.level_sizes(l)
        lt = max(64, 4 * -(-s["nnz"] // s["n"]))
        lens = np.diff(h.export_level(l)["A_rp"])
        assert f["nlong"] == int((lens > lt).sum()), (l, f, lt)
        assert f["long_threshold"] == (lt if f["nlong"] > 0 else -1), (l, f, lt)
        binned += f["nlong"]
    if sig[0] >= 1e3:
        assert binned > 0, fm  # the 490-entry rows
    o = orc.Hierarchy(p, 0.05, "material")
    rng = np.random.default_rng(3)
    r = rng.standard_normal(p["n"])
    zg = h.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    zo = o.vcycle(r)
    assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)
    hm = sa.Hierarchy(p, theta=0.05, measure="material", precision="fp32")
    zm = hm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.linalg.norm(zm - zo) <= 1e-3 * np.linalg.norm(zo)
    A = sp.csr_matrix((p["val"], p["col"], p["row_ptr"]), shape=(p["n"], p["n"]))
    b = torch.from_numpy(np.stack([p["b"], A @ rng.standard_normal(p["n"])])).cuda()
    for hh in (h, hm):
        X, infos = hh.solve_batch(b)
        for c in range(2):
            x1, i1 = hh.solve(b[c].contiguous())
            assert infos[c]["iters"] == i1["iters"]
            assert torch.equal(X[c], x1)


def test_standalone_strength_worked_example(sa, orc, gen_mod):
    import torch
    for kappa in (1.0, 100.0, 1e4):
        p = gen_mod.worked_example(kappa=kappa)
        sinv = orc.invert_tensors(2, p["tensors"])
        for theta in (0.0, 0.05, 0.1, 0.2):
            _, _, ko = orc.strength_material(2, p["n"], p["row_ptr"], p["col"], None, p["coords"], sinv, theta)
            t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)  # noqa: E731
            kg = sa.strength("material", 2, t(p["row_ptr"], torch.int64), t(p["col"], torch.int32), None,
                             t(p["coords"], torch.float64), t(sinv, torch.float64), None, theta)
            assert np.array_equal(kg.cpu().numpy(), ko)
            kc = sa.strength("classical", 2, t(p["row_ptr"], torch.int64), t(p["col"], torch.int32),
                             t(p["val"], torch.float64), None, None, None, theta)
            assert np.array_equal(kc.cpu().numpy(),
                                  orc.strength_classical(p["n"], p["row_ptr"], p["col"], p["val"], None, theta))


def test_single_level_is_a_direct_solve(sa, gen_mod):
    import torch
    p = gen_mod.layered_2d(16)
    h = sa.Hierarchy(p, theta=0.08, measure="material", max_coarse=5000)
    assert h.stats()["levels"] == 1
    x, info = h.solve(torch.from_numpy(p["b"]).cuda())
    assert info["status"] == 0 and info["iters"] <= 2 and info["rel_res"] <= 1e-8


@pytest.mark.parametrize("n_el", [31, 48])
def test_coarse_block_substitution_is_a_direct_solve(sa, gen_mod, n_el):
    """A one-level hierarchy is the coarse direct solve alone: 1024 rows (one
    diagonal block, the whole inverse) and 2401 rows (three diagonal blocks,
    the last one ragged).  Its V-cycle equals a sparse direct solve, and a
    block solve's columns equal the one-vector solves bitwise."""
    import torch
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    p = gen_mod.layered_2d(n_el, contrast=1e-2)
    h = sa.Hierarchy(p, theta=0.08, measure="material", max_coarse=5000)
    assert h.stats()["levels"] == 1 and h.level_format(0)["lanes"] == -1
    A = sp.csr_matrix((p["val"], p["col"], p["row_ptr"]), shape=(p["n"], p["n"]))
    rng = np.random.default_rng(5)
    r = rng.standard_normal(p["n"])
    z = h.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    ze = spla.spsolve(A.tocsc(), r)
    assert np.linalg.norm(z - ze) <= 1e-9 * np.linalg.norm(ze)
    b = torch.from_numpy(np.stack([r, A @ rng.standard_normal(p["n"])])).cuda()
    X, infos = h.solve_batch(b)
    for c in range(2):
        x1, i1 = h.solve(b[c].contiguous())
        assert infos[c]["iters"] == i1["iters"] <= 2
        assert torch.equal(X[c], x1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_right_hand_side(sa, gen_mod, precision):
    """b = 0 ends before the first iteration with x = 0 and status OK, alone and
    as one column of a block beside a column that iterates (the columns stay
    independent)."""
    import torch
    p = gen_mod.battery_3d(12, 12, 24)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=100, precision=precision)
    z = torch.zeros(p["n"], dtype=torch.float64, device="cuda")
    x, info = h.solve(z)
    assert info["status"] == 0 and info["iters"] == 0 and torch.count_nonzero(x) == 0
    b = torch.from_numpy(p["b"]).cuda()
    xs, i1 = h.solve(b)
    X, infos = h.solve_batch(torch.stack([z, b]))
    assert infos[0]["iters"] == 0 and infos[0]["status"] == 0 and torch.count_nonzero(X[0]) == 0
    assert infos[1]["iters"] == i1["iters"] and torch.equal(X[1], xs)


def test_host_pointer_path_matches_device_path(sa, gen_mod):
    import torch
    p = gen_mod.battery_3d(12, 12, 24)
    hd = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=100)
    hh = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=100, host_inputs=True)
    assert hd.stats() == {**hh.stats(), "device_bytes": hd.stats()["device_bytes"]}
    xd, a = hd.solve(torch.from_numpy(p["b"]).cuda())
    xh, b = hh.solve(p["b"])  # host buffers in, host buffers out
    assert a["iters"] == b["iters"]
    assert np.array_equal(xd.cpu().numpy(), xh)


def test_error_statuses_without_faults(sa, gen_mod):
    import torch
    p = gen_mod.layered_2d(16)
    # negative definite: the coarse Cholesky reports a non-positive pivot
    q = dict(p)
    q["val"] = -p["val"]
    with pytest.raises(sa.SAError) as e:
        sa.Hierarchy(q, theta=0.08, measure="classical", max_coarse=5000)
    assert e.value.status == -4
    # maxit reached: status NO_CONVERGENCE with the last iterate returned
    h = sa.Hierarchy(p, theta=0.08, measure="material", max_coarse=30, maxit=1)
    x, info = h.solve(torch.from_numpy(p["b"]).cuda(), tol=1e-14)
    assert info["status"] == -6 and info["iters"] == 1 and torch.isfinite(x).all()
    # material measure without coordinates is rejected before any copy
    import ctypes
    L = sa.lib()
    o = sa.default_options()
    t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("row_ptr", "col", "val")}
    pr = sa.Problem()
    pr.dim, pr.n, pr.nnz = 2, p["n"], p["nnz"]
    pr.row_ptr, pr.col, pr.val = t["row_ptr"].data_ptr(), t["col"].data_ptr(), t["val"].data_ptr()
    hh = ctypes.c_void_p()
    assert L.sa_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(hh)) == -1
    assert not hh.value


def test_allocator_failure_reports_oom(sa, gen_mod):
    import ctypes
    import torch
    p = gen_mod.layered_2d(16)
    L = sa.lib()
    o = sa.default_options()
    o.max_coarse = 30
    o.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    calls = {"n": 0}

    @sa.api._ALLOC
    def failing_alloc(nbytes, ctx):
        calls["n"] += 1
        return None

    @sa.api._FREE
    def no_free(ptr, ctx):
        pass

    o.alloc = failing_alloc
    o.dealloc = no_free
    t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("row_ptr", "col", "val", "coords")}
    pr = sa.Problem()
    pr.dim, pr.n, pr.nnz = 2, p["n"], p["nnz"]
    pr.row_ptr, pr.col, pr.val = t["row_ptr"].data_ptr(), t["col"].data_ptr(), t["val"].data_ptr()
    pr.coords = t["coords"].data_ptr()
    o.measure = 0
    hh = ctypes.c_void_p()
    assert L.sa_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(hh)) == -2
    assert calls["n"] >= 1 and not hh.value


def test_batch_solve_columns_independent(sa, gen_mod):
    import torch
    p = gen_mod.battery_3d(12, 12, 24)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=100)
    rng = np.random.default_rng(1)
    B = rng.standard_normal((3, p["n"]))
    B[:, p["dir_mask"] == 1] = 0.0
    import ctypes
    Bd = torch.from_numpy(B).cuda().contiguous()
    Xd = torch.zeros_like(Bd)
    infos = (sa.SolveInfo * 3)()
    st = sa.lib().sa_solve_batch(h.h, 3, Bd.data_ptr(), Xd.data_ptr(), 1e-8, infos)
    assert st == 0
    for c in range(3):
        x1, i1 = h.solve(Bd[c].clone())
        assert infos[c].iters == i1["iters"]
        assert torch.equal(Xd[c], x1)
    del ctypes


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_loop_equals_host_loop(sa, gen_mod, precision):
    """the captured CG loop (conditional WHILE graph) and the host-driven loop
    (used while profiling) launch the same kernels in the same order"""
    import torch
    p = gen_mod.battery_3d(16, 16, 32)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=200, precision=precision)
    b = torch.from_numpy(p["b"]).cuda()
    xg, ig = h.solve(b)
    sa.profile_enable(True)
    try:
        xe, ie = h.solve(b)
        rows = sa.profile_read()
    finally:
        sa.profile_enable(False)
    assert ig["iters"] == ie["iters"] and ig["status"] == ie["status"] == 0
    assert torch.equal(xg, xe)
    kinds = {r["kind"] for r in rows}
    assert ("cheb64" if precision == "fp64" else "cheb32") in kinds and "cg_spmv" in kinds
    assert all(r["ms"] > 0 and r["bytes"] > 0 for r in rows)


def test_theta_sweep_matches_oracle(sa, orc, gen_mod):
    """Sec. 4.1 sweep driver on the two-domain problem (kappa = 1e4): every
    (measure, drop, theta) configuration has the oracle's outcome, level
    count and iteration count (within 1); cost = C x iterations."""
    from paper_2602_05686_gb300.sweep import theta_sweep
    p = gen_mod.two_domain(32, 1e4)
    rows = theta_sweep(p, thetas=(0.02, 0.08, 0.32), measures=("classical", "distance", "material"), max_coarse=64,
                       drops=("pointwise", "cut"))
    assert len(rows) == 18
    for r in rows:
        try:
            o = orc.Hierarchy(p, r["theta"], r["measure"], max_coarse=64, drop=r["drop"])
        except Exception:
            assert r["status"] != 0, r   # the oracle refuses the setup too (stagnation)
            continue
        _, oi = o.solve(p["b"])
        assert r["status"] == oi["status"], (r, oi)
        if r["status"] == 0:
            assert r["levels"] == o.nlev and abs(r["iters"] - oi["iters"]) <= 1, (r, oi)
            assert r["cost"] == pytest.approx(r["op_complexity"] * r["iters"])


def test_annulus_study_matches_oracle(sa, orc, gen_mod):
    """Sec. 4.2 study driver on h and h/2 at the extreme contrasts: every
    configuration converges with the oracle's iteration count (within 1),
    level count and operator complexity."""
    from paper_2602_05686_gb300.sweep import annulus_study
    rows = annulus_study(lambda rf, k: gen_mod.annulus_3d(rf, kappa=k), refines=(0, 1), kappas=(1.0, 1e4))
    assert len(rows) == 8
    for r in rows:
        p = gen_mod.annulus_3d(r["refine"], kappa=r["kappa"])
        o = orc.Hierarchy(p, r["theta"], "material")
        _, oi = o.solve(p["b"])
        assert r["status"] == 0 and r["rel_res"] <= 1e-8, r
        assert abs(r["iters"] - oi["iters"]) <= 1 and r["levels"] == o.nlev, (r, oi)
        assert r["op_complexity"] == pytest.approx(o.operator_complexity(), abs=1e-3)


def _raw_handle(sa, p, t, o):
    import ctypes
    pr = sa.Problem()
    pr.dim, pr.n, pr.nnz = 3, p["n"], p["nnz"]
    pr.row_ptr, pr.col, pr.val = t["row_ptr"].data_ptr(), t["col"].data_ptr(), t["val"].data_ptr()
    pr.coords = t["coords"].data_ptr()
    hh = ctypes.c_void_p()
    st = sa.lib().sa_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(hh))
    return st, hh


@pytest.mark.parametrize("precision", [0, 1])
def test_caller_allocator_alignment(sa, gen_mod, precision):
    """a caller allocator's blocks must start on 256-byte boundaries (the
    block kernels move whole rows with 32-byte accesses): aligned blocks give
    bitwise the default allocator's solve; blocks offset by 64 bytes are
    refused at the first allocation, before any kernel runs on them"""
    import ctypes
    import torch
    p = gen_mod.battery_3d(12, 12, 24)
    t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("row_ptr", "col", "val", "coords")}
    L = sa.lib()
    live = {}

    def make(offset):
        @sa.api._ALLOC
        def alloc(nbytes, ctx):
            buf = torch.empty(int(nbytes) + 512, dtype=torch.uint8, device="cuda")
            base = (buf.data_ptr() + 255) // 256 * 256
            ptr = base + offset
            live[ptr] = buf
            return ptr

        @sa.api._FREE
        def free(ptr, ctx):
            live.pop(ptr, None)

        return alloc, free

    def opts(alloc=None, free=None):
        o = sa.default_options()
        o.max_coarse = 100
        o.measure = 0
        o.precision = precision
        o.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        if alloc is not None:
            o.alloc, o.dealloc = alloc, free
        return o

    rng = np.random.default_rng(3)
    B = rng.standard_normal((8, p["n"]))
    B[:, p["dir_mask"] == 1] = 0.0
    Bd = torch.from_numpy(B).cuda().contiguous()
    res = []
    cbs = make(0)
    for o in (opts(), opts(*cbs)):
        st, hh = _raw_handle(sa, p, t, o)
        assert st == 0 and hh.value
        Xd = torch.zeros_like(Bd)
        infos = (sa.SolveInfo * 8)()
        assert L.sa_solve_batch(hh, 8, Bd.data_ptr(), Xd.data_ptr(), 1e-8, infos) == 0
        torch.cuda.synchronize()
        res.append((Xd.cpu(), [infos[c].iters for c in range(8)]))
        L.sa_free(hh)
    assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]
    assert not live  # every block handed back
    bad = make(64)
    st, hh = _raw_handle(sa, p, t, opts(*bad))
    assert st == -2 and not hh.value
    assert b"256 bytes" in sa.lib().sa_last_error()
    assert not live


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_guess_batch_equals_explicit_zeros(sa, gen_mod, precision):
    """sa_solve_batch_zero (X output only) ends bitwise where sa_solve_batch
    from an X of zeros ends: one column, a partial block and a full block,
    device and host buffers"""
    import ctypes
    import torch
    p = gen_mod.battery_3d(12, 12, 24)
    h = sa.Hierarchy(p, theta=0.05, measure="classical", max_coarse=100, precision=precision)
    rng = np.random.default_rng(5)
    L = sa.lib()
    for k in (1, 3, 8):
        B = rng.standard_normal((k, p["n"]))
        B[:, p["dir_mask"] == 1] = 0.0
        Bd = torch.from_numpy(B).cuda().contiguous()
        ref = torch.zeros_like(Bd)
        i0 = (sa.SolveInfo * k)()
        assert L.sa_solve_batch(h.h, k, Bd.data_ptr(), ref.data_ptr(), 1e-8, i0) == 0
        got = torch.full_like(Bd, float("nan"))  # never read
        i1 = (sa.SolveInfo * k)()
        assert L.sa_solve_batch_zero(h.h, k, Bd.data_ptr(), got.data_ptr(), 1e-8, i1) == 0
        torch.cuda.synchronize()
        assert torch.equal(ref, got), k
        assert [i0[c].iters for c in range(k)] == [i1[c].iters for c in range(k)]
        Xh, infos = h.solve_batch(B)  # host buffers, no initial guess
        assert np.array_equal(Xh, ref.cpu().numpy())
        assert [d["iters"] for d in infos] == [i0[c].iters for c in range(k)]
    h.free()
    del ctypes


@pytest.mark.parametrize("measure", ["material", "classical"])
def test_spgemm_one_pass_equals_two_phase(sa, gen_mod, measure, monkeypatch):
    """the one-pass SpGEMM (rows filled once into product-count slots, then
    packed) and the count-then-fill form build the same hierarchy bit for
    bit: every level's aggregates, P and A"""
    p = gen_mod.battery_3d(24, 24, 48)
    h1 = sa.Hierarchy(p, theta=0.05, measure=measure, max_coarse=100)
    monkeypatch.setenv("SA_SPGEMM_PASSES", "2")
    h2 = sa.Hierarchy(p, theta=0.05, measure=measure, max_coarse=100)
    monkeypatch.delenv("SA_SPGEMM_PASSES")
    n1, n2 = h1.stats()["levels"], h2.stats()["levels"]
    assert n1 == n2 and n1 >= 3
    for l in range(n1):
        a, b = h1.export_level(l), h2.export_level(l)
        for k in ("agg", "P_rp", "P_ci", "P_v", "A_rp", "A_ci", "A_v"):
            assert np.array_equal(a[k], b[k]), (l, k)
    h1.free()
    h2.free()
