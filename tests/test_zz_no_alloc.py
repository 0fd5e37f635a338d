"""The allocation-free material strength entry point, called through the C
ABI, against the allocating one (sa_strength, SA_MEASURE_MATERIAL): the
keep masks must be identical on two calls in a row with different inputs.
This file is collected last so that a failure here does not stop the other
tests of a run that stops at the first failure."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import gen
    import oracle
    import paper_2602_05686_gb300 as sa
    sa.build()
    oracle.build()
    return torch, gen, oracle, sa


def _inputs(torch, gen, orc, p):
    dim = p["dim"]
    sig = orc.nodal_from_elements(dim, p["n"], p["elem_nodes"], p["elem_measure"], p["tensors"])
    sinv = orc.invert_tensors(dim, sig)

    def t(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)

    return dict(dim=dim, rp=t(p["row_ptr"], torch.int64), ci=t(p["col"], torch.int32),
                x=t(p["coords"], torch.float64), sinv=t(sinv, torch.float64),
                dirm=t(p["dir_mask"], torch.uint8))


def test_noalloc_matches_allocating_entry_point_twice(env):
    torch, gen, orc, sa = env
    problems = [gen.voronoi_3d(10, nseeds=6, seed=2), gen.layered_2d(64, contrast=1e-3)]
    for p, theta in zip(problems, (0.05, 0.08)):  # two calls in a row, different sizes
        a = _inputs(torch, gen, orc, p)
        ref = sa.strength("material", a["dim"], a["rp"], a["ci"], None, a["x"], a["sinv"], a["dirm"], theta)
        keep = torch.full((p["nnz"],), 7, dtype=torch.uint8, device="cuda")
        st = sa.api.strength_material_noalloc(a["dim"], a["rp"], a["ci"], a["x"], a["sinv"], a["dirm"], theta, keep)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.equal(keep, ref)
        assert int(keep.sum()) > p["n"]  # more than the diagonals are kept


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, gen, orc, sa = env
    p = gen.layered_2d(8)
    a = _inputs(torch, gen, orc, p)
    keep = torch.zeros(p["nnz"], dtype=torch.uint8, device="cuda")
    L = sa.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # sizes beyond 2,097,152 doubles are refused before anything is launched
    st = L.sa_strength_material_noalloc(2, 3_000_000, 3_000_000, a["rp"].data_ptr(), a["ci"].data_ptr(),
                                        a["x"].data_ptr(), a["sinv"].data_ptr(), None, 0.05, keep.data_ptr(), s)
    assert st == -8
    assert b"static scratch" in L.sa_last_error()
    assert int(keep.sum()) == 0


def test_noalloc_rejects_a_malformed_csr_before_any_weight(env):
    torch, gen, orc, sa = env
    p = gen.layered_2d(8)
    a = _inputs(torch, gen, orc, p)
    keep = torch.zeros(p["nnz"], dtype=torch.uint8, device="cuda")
    L = sa.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, nnz = p["n"], p["nnz"]
    # row_ptr[n] beyond nnz: the check reads only row_ptr and the columns
    # below nnz, so nothing outside the caller's buffers is touched
    rp_long = a["rp"].clone()
    rp_long[n] = nnz + 5
    st = L.sa_strength_material_noalloc(2, n, nnz, rp_long.data_ptr(), a["ci"].data_ptr(), a["x"].data_ptr(),
                                        a["sinv"].data_ptr(), None, 0.05, keep.data_ptr(), s)
    assert st == -1
    assert b"invalid CSR" in L.sa_last_error()
    # a column index outside [0, n)
    ci_bad = a["ci"].clone()
    ci_bad[int(p["row_ptr"][3])] = n + 7
    st = L.sa_strength_material_noalloc(2, n, nnz, a["rp"].data_ptr(), ci_bad.data_ptr(), a["x"].data_ptr(),
                                        a["sinv"].data_ptr(), None, 0.05, keep.data_ptr(), s)
    assert st == -1
    torch.cuda.synchronize()
    assert int(keep.sum()) == 0
    # the entry point still works after the refusals
    st = sa.api.strength_material_noalloc(2, a["rp"], a["ci"], a["x"], a["sinv"], a["dirm"], 0.08, keep)
    ref = sa.strength("material", 2, a["rp"], a["ci"], None, a["x"], a["sinv"], a["dirm"], 0.08)
    torch.cuda.synchronize()
    assert st == 0 and torch.equal(keep, ref)
