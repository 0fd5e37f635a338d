"""The C-ABI library builds, loads and exports every entry point declared in
include/sa.h (no compute calls: CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "sa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sa_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    d = declared()
    for name in ("sa_setup", "sa_solve", "sa_free", "sa_solve_batch", "sa_hierarchy_stats", "sa_export_level",
                 "sa_default_options", "sa_status_string"):
        assert name in d


def test_library_exports_every_declared_symbol():
    import paper_2602_05686_gb300 as sa
    sa.build()
    L = sa.lib(build_if_missing=False)
    missing = [s for s in declared() if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(sa.EXPORTED) == declared()


def test_defaults_and_status_strings_without_gpu():
    import paper_2602_05686_gb300 as sa
    o = sa.default_options()
    assert o.theta == pytest.approx(0.08) and o.max_coarse == 5000 and o.max_levels == 10
    assert o.cheb_degree == 2 and o.power_iters == 10 and o.omega_sym == pytest.approx(4 / 3)
    L = sa.lib(build_if_missing=False)
    assert L.sa_status_string(0) == b"ok"
    assert L.sa_status_string(-4) == b"coarse operator not SPD"


def test_setup_rejects_bad_arguments_before_touching_a_gpu():
    import ctypes
    import paper_2602_05686_gb300 as sa
    L = sa.lib(build_if_missing=False)
    o = sa.default_options()
    pr = sa.Problem()
    pr.dim = 5  # invalid
    h = ctypes.c_void_p()
    assert L.sa_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == -1
    assert not h.value
    pr.dim, pr.n, pr.nnz = 2, 0, 0
    assert L.sa_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h)) == -1
    assert L.sa_setup(None, ctypes.byref(o), ctypes.byref(h)) == -1


def test_inspection_calls_reject_bad_arguments_without_gpu():
    import ctypes
    import numpy as np
    import paper_2602_05686_gb300 as sa
    L = sa.lib(build_if_missing=False)
    out = np.zeros(5, np.int64)
    assert L.sa_level_format(None, 0, out.ctypes.data) == -1
    assert L.sa_level_sizes(None, 0, out.ctypes.data) == -1
    assert L.sa_level_format(ctypes.c_void_p(), 0, None) == -1
