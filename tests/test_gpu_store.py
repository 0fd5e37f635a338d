"""Hierarchy store (sa_serialize / sa_deserialize): a stored and reloaded
hierarchy is bit-identical level by level and solves bit-identically (FP64
and FP32 V-cycle forms), also in another process; damaged stores are
rejected on the host with SA_ERR_INVALID_ARG."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_05686_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def built(sa, gen_mod):
    p = gen_mod.battery_3d(16, 16, 32)
    h = sa.Hierarchy(p, theta=0.05, measure="material", max_coarse=200)
    return p, h, h.to_bytes()


def test_store_roundtrip_bit_identical(sa, built):
    import torch
    p, h, buf = built
    g = sa.Hierarchy.from_bytes(buf)
    assert g.stats()["n"] == h.stats()["n"] and g.stats()["nnz"] == h.stats()["nnz"]
    for l in range(h.stats()["levels"]):
        a, b = h.export_level(l), g.export_level(l)
        for k in ("A_rp", "A_ci", "A_v", "agg", "P_rp", "P_ci", "P_v"):
            assert np.array_equal(a[k], b[k]), (l, k)
    rhs = torch.from_numpy(p["b"]).cuda()
    x1, i1 = h.solve(rhs)
    x2, i2 = g.solve(rhs)
    assert i1["iters"] == i2["iters"] and torch.equal(x1, x2)
    h.set_precision("fp32")
    g.set_precision("fp32")
    y1, j1 = h.solve(rhs)
    y2, j2 = g.solve(rhs)
    assert j1["iters"] == j2["iters"] and torch.equal(y1, y2) and j2["rel_res"] <= 1e-8
    h.set_precision("fp64")
    # a re-stored loaded hierarchy is the same byte string
    assert np.array_equal(g.to_bytes(), buf)
    g.free()


def test_store_rejects_damage(sa, built):
    _, _, buf = built
    bad = buf.copy()
    bad[len(bad) // 2] ^= 0x40                       # payload bit flip -> checksum
    for b in (bad, buf[:-8], buf[:50], np.concatenate([buf, np.zeros(8, np.uint8)])):
        with pytest.raises(sa.SAError) as e:
            sa.Hierarchy.from_bytes(b)
        assert e.value.status == -1
    magic = buf.copy()
    magic[0] ^= 1
    with pytest.raises(sa.SAError):
        sa.Hierarchy.from_bytes(magic)


def test_store_reused_in_another_process(sa, built, tmp_path):
    import torch
    p, h, buf = built
    path = tmp_path / "battery.saamg"
    h.save(str(path))
    np.save(tmp_path / "b.npy", p["b"])
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import paper_2602_05686_gb300 as sa\n"
        f"g = sa.Hierarchy.load({str(path)!r})\n"
        f"x, i = g.solve(torch.from_numpy(np.load({str(tmp_path / 'b.npy')!r})).cuda())\n"
        f"np.save({str(tmp_path / 'x.npy')!r}, x.cpu().numpy())\n"
        "print(i['iters'])\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    x1, i1 = h.solve(torch.from_numpy(p["b"]).cuda())
    assert int(out.stdout.split()[-1]) == i1["iters"]
    assert np.array_equal(np.load(tmp_path / "x.npy"), x1.cpu().numpy())
