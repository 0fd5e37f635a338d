"""CPU oracle for SA-AMG with classical / material-aware strength of connection.

TEST INFRASTRUCTURE ONLY.  A plain serial FP64 C implementation
(``sa_oracle.c``) of every step of the hot path, written from the paper's
definitions (arXiv 2602.05686, Sections 2-4) and checked against closed forms,
brute force and invariants in the CPU test suite.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package; the CUDA library shares no code with it.

Every function is pinned by a CPU test (worked example, closed forms, dense
brute force or invariants); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_sa_oracle.so")
_L = None

OK, ERR_INVALID_ARG, ERR_OOM, ERR_NOT_SPD, ERR_STAGNATION, ERR_NO_CONVERGENCE, ERR_BREAKDOWN = (
    0, -1, -2, -4, -5, -6, -7)
MEASURES = {"classical": 0, "material": 1, "distance": 2}
DROPS = {"pointwise": 0, "cut": 1}


def build(force: bool = False) -> str:
    """Compile sa_oracle.c with gcc -O2 -ffp-contract=off (no FMA contraction)."""
    src = os.path.join(_HERE, "sa_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                               src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Opts(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("measure", ctypes.c_int), ("drop", ctypes.c_int),
                ("max_coarse", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("power_iters", ctypes.c_int),
                ("omega_sym", ctypes.c_double), ("cheb_boost", ctypes.c_double),
                ("cheb_ratio", ctypes.c_double), ("seed", ctypes.c_uint32)]


def lib():
    global _L
    if _L is None:
        build()
        L = ctypes.CDLL(_SO)
        P, I64, I32, D, U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint32
        sig = {
            "or_mis_key": (ctypes.c_uint64, [I64, I32, U32]),
            "or_start_value": (D, [I64, U32, U32]),
            "or_dirichlet": (None, [I64, P, P, P, P]),
            "or_nodal_from_elements": (I32, [I32, I64, I64, I32, P, P, P, P]),
            "or_invert_tensors": (None, [I32, I64, P, P]),
            "or_strength_classical": (None, [I64, P, P, P, P, D, P]),
            "or_strength_material": (None, [I32, I64, P, P, P, P, P, D, P, P, P]),
            "or_cut_drop": (None, [I64, P, P, P, P, D, P]),
            "or_strength2_classical": (None, [I64, P, P, P, P]),
            "or_strength2_material": (None, [I64, P, P, P, P, P]),
            "or_filtered_graph": (I64, [I64, P, P, P, P, P, P]),
            "or_mis2": (None, [I64, P, P, P, I32, U32, P]),
            "or_aggregate": (I64, [I64, P, P, P, P, P]),
            "or_coarse_aux": (None, [I32, I64, I64, P, P, P, P, P]),
            "or_setup": (P, [I32, I64, P, P, P, P, I32, P, I64, I32, P, P, P, P]),
            "or_free": (None, [P]),
            "or_num_levels": (I32, [P]),
            "or_level_sizes": (None, [P, I32, P]),
            "or_level_export": (None, [P, I32] + [P] * 13),
            "or_operator_complexity": (D, [P]),
            "or_set_cheb": (None, [P, I32, D, D]),
            "or_pcg": (I32, [P, P, P, D, I32, I32, P, P]),
            "or_pcg_hist": (I32, [P, P, P, D, I32, I32, P, P, P]),
            "or_pcg_diag_cycle": (I32, [I64, P, P, P, I32, P, P, P, D, I32, I32, P, P, P]),
            "or_vcycle": (None, [P, P, P]),
            "or_coarsest_solve": (None, [P, P, P]),
            "or_csr_info": (None, [P, P]),
            "or_csr_copy": (None, [P, P, P, P]),
            "or_csr_free": (None, [P]),
            "or_step_spgemm": (P, [I64, I64, I64, P, P, P, P, P, P]),
            "or_step_transpose": (P, [I64, I64, P, P, P]),
            "or_step_filter": (P, [I64, P, P, P, P, P]),
            "or_step_tentative": (P, [I64, I64, P]),
            "or_step_smooth_prolongator": (P, [I64, I64, P, P, P, P, D, P]),
            "or_step_galerkin": (P, [I64, I64, P, P, P, P, P, P, P]),
            "or_step_power": (D, [I64, P, P, P, P, I32, U32, U32]),
            "or_step_chebyshev": (None, [I64, P, P, P, P, D, D, I32, P, P, I32]),
            "or_dense_cholesky_factor": (I32, [I64, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _unbox(b):
    L = lib()
    info = np.zeros(3, np.int64)
    L.or_csr_info(b, _p(info))
    nr, nc, nnz = (int(x) for x in info)
    rp = np.zeros(nr + 1, np.int64)
    ci = np.zeros(max(nnz, 1), np.int32)
    v = np.zeros(max(nnz, 1), np.float64)
    L.or_csr_copy(b, _p(rp), _p(ci), _p(v))
    L.or_csr_free(b)
    return dict(nrows=nr, ncols=nc, row_ptr=rp, col=ci[:nnz], val=v[:nnz])


# ---------------------------------------------------------------------------
# single steps
# ---------------------------------------------------------------------------
def mis_key(i, level, seed=0):
    return int(lib().or_mis_key(int(i), int(level), int(seed)))


def start_value(i, tag, seed=0):
    return float(lib().or_start_value(int(i), int(tag), int(seed)))


def dirichlet(n, rp, ci, v):
    out = np.zeros(n, np.uint8)
    lib().or_dirichlet(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(v, np.float64)), _p(out))
    return out


def nodal_from_elements(dim, n, elem_nodes, elem_measure, elem_tensors):
    kp = 6 if dim == 3 else 3
    en = _c(elem_nodes, np.int32)
    em = _c(elem_measure, np.float64)
    et = _c(elem_tensors, np.float64)
    ne = em.size
    out = np.zeros(n * kp)
    st = lib().or_nodal_from_elements(dim, n, ne, en.size // ne, _p(en), _p(em), _p(et), _p(out))
    if st:
        raise ValueError(f"oracle nodal tensors status {st}")
    return out


def invert_tensors(dim, sigma):
    kp = 6 if dim == 3 else 3
    s = _c(sigma, np.float64)
    out = np.zeros_like(s)
    lib().or_invert_tensors(dim, s.size // kp, _p(s), _p(out))
    return out


def strength_classical(n, rp, ci, v, dirm, theta):
    keep = np.zeros(len(ci), np.uint8)
    lib().or_strength_classical(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(v, np.float64)),
                                _p(None if dirm is None else _c(dirm, np.uint8)), float(theta), _p(keep))
    return keep


def strength_material(dim, n, rp, ci, dirm, coords, sinv, theta):
    nnz = len(ci)
    w = np.zeros(nnz)
    D = np.zeros(n)
    keep = np.zeros(nnz, np.uint8)
    lib().or_strength_material(dim, n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)),
                               _p(None if dirm is None else _c(dirm, np.uint8)),
                               _p(_c(coords, np.float64)), _p(_c(sinv, np.float64)), float(theta),
                               _p(w), _p(D), _p(keep))
    return w, D, keep


def strength2_classical(n, rp, ci, v):
    s2 = np.zeros(len(ci))
    lib().or_strength2_classical(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(v, np.float64)), _p(s2))
    return s2


def strength2_material(n, rp, ci, w, D):
    s2 = np.zeros(len(ci))
    lib().or_strength2_material(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(w, np.float64)),
                                _p(_c(D, np.float64)), _p(s2))
    return s2


def cut_drop(n, rp, ci, dirm, s2, theta):
    keep = np.zeros(len(ci), np.uint8)
    lib().or_cut_drop(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(None if dirm is None else _c(dirm, np.uint8)),
                      _p(_c(s2, np.float64)), float(theta), _p(keep))
    return keep


def filtered_graph(n, rp, ci, keep, dirm):
    grp = np.zeros(n + 1, np.int64)
    gci = np.zeros(max(len(ci), 1), np.int32)
    m = lib().or_filtered_graph(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(keep, np.uint8)),
                                _p(None if dirm is None else _c(dirm, np.uint8)), _p(grp), _p(gci))
    return grp, gci[:m].copy()


def mis2(n, grp, gci, dirm, level=0, seed=0):
    root = np.zeros(n, np.uint8)
    lib().or_mis2(n, _p(_c(grp, np.int64)), _p(_c(gci, np.int32)),
                  _p(None if dirm is None else _c(dirm, np.uint8)), level, seed, _p(root))
    return root


def aggregate(n, grp, gci, dirm, root):
    agg = np.zeros(n, np.int32)
    nc = lib().or_aggregate(n, _p(_c(grp, np.int64)), _p(_c(gci, np.int32)),
                            _p(None if dirm is None else _c(dirm, np.uint8)), _p(_c(root, np.uint8)),
                            _p(agg))
    return int(nc), agg


def coarse_aux(dim, n, nc, agg, x, sigma):
    kp = 6 if dim == 3 else 3
    xc = np.zeros(nc * dim)
    sc = np.zeros(nc * kp)
    lib().or_coarse_aux(dim, n, nc, _p(_c(agg, np.int32)), _p(_c(x, np.float64)),
                        _p(_c(sigma, np.float64)), _p(xc), _p(sc))
    return xc, sc


def pcg_diag_cycle(n, rp, ci, v, dinvs, b, tol=1e-10, maxit=200, flexible=False):
    """CG whose k-th preconditioner application is diag(dinvs[k mod len(dinvs)]);
    returns x, status, iterations, true relative residual and the recursive
    residual history ||r_k|| / ||r_0||"""
    D = _c(np.stack([np.asarray(d, np.float64) for d in dinvs]), np.float64)
    x = np.zeros(n)
    hist = np.full(maxit + 1, np.nan)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib().or_pcg_diag_cycle(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(v, np.float64)), D.shape[0],
                                 _p(D), _p(_c(b, np.float64)), _p(x), float(tol), int(maxit), int(flexible),
                                 ctypes.byref(it), ctypes.byref(rel), _p(hist))
    return x, dict(status=int(st), iters=int(it.value), rel_res=float(rel.value), hist=hist[:it.value + 1])


def tentative(n, nc, agg):
    return _unbox(lib().or_step_tentative(n, nc, _p(_c(agg, np.int32))))


def filter_matrix(n, rp, ci, v, keep):
    Dt = np.zeros(n)
    F = _unbox(lib().or_step_filter(n, _p(_c(rp, np.int64)), _p(_c(ci, np.int32)), _p(_c(v, np.float64)),
                                    _p(_c(keep, np.uint8)), _p(Dt)))
    return F, Dt


def spgemm(A, B):
    return _unbox(lib().or_step_spgemm(A["nrows"], A["ncols"], B["ncols"], _p(_c(A["row_ptr"], np.int64)),
                                       _p(_c(A["col"], np.int32)), _p(_c(A["val"], np.float64)),
                                       _p(_c(B["row_ptr"], np.int64)), _p(_c(B["col"], np.int32)),
                                       _p(_c(B["val"], np.float64))))


def transpose(A):
    return _unbox(lib().or_step_transpose(A["nrows"], A["ncols"], _p(_c(A["row_ptr"], np.int64)),
                                          _p(_c(A["col"], np.int32)), _p(_c(A["val"], np.float64))))


def smooth_prolongator(F, Dt, omega, agg, nc):
    n = F["nrows"]
    return _unbox(lib().or_step_smooth_prolongator(n, nc, _p(_c(F["row_ptr"], np.int64)),
                                                   _p(_c(F["col"], np.int32)), _p(_c(F["val"], np.float64)),
                                                   _p(_c(Dt, np.float64)), float(omega), _p(_c(agg, np.int32))))


def galerkin(A, P):
    st = ctypes.c_int(0)
    C = _unbox(lib().or_step_galerkin(A["nrows"], P["ncols"], _p(_c(A["row_ptr"], np.int64)),
                                      _p(_c(A["col"], np.int32)), _p(_c(A["val"], np.float64)),
                                      _p(_c(P["row_ptr"], np.int64)), _p(_c(P["col"], np.int32)),
                                      _p(_c(P["val"], np.float64)), ctypes.byref(st)))
    if st.value:
        raise ValueError(f"oracle galerkin status {st.value}")
    return C


def power_estimate(A, s, steps=10, tag=1, seed=0):
    return float(lib().or_step_power(A["nrows"], _p(_c(A["row_ptr"], np.int64)), _p(_c(A["col"], np.int32)),
                                     _p(_c(A["val"], np.float64)), _p(_c(s, np.float64)), steps, tag, seed))


def chebyshev(A, dinv, lmax, lmin, deg, b, x=None):
    n = A["nrows"]
    xz = x is None
    xx = np.zeros(n) if xz else _c(x, np.float64).copy()
    lib().or_step_chebyshev(n, _p(_c(A["row_ptr"], np.int64)), _p(_c(A["col"], np.int32)),
                            _p(_c(A["val"], np.float64)), _p(_c(dinv, np.float64)), float(lmax), float(lmin),
                            int(deg), _p(_c(b, np.float64)), _p(xx), int(xz))
    return xx


def dense_cholesky(A):
    n = A["nrows"]
    L = np.zeros(n * n)
    st = lib().or_dense_cholesky_factor(n, _p(_c(A["row_ptr"], np.int64)), _p(_c(A["col"], np.int32)),
                                        _p(_c(A["val"], np.float64)), _p(L))
    return st, L.reshape(n, n)


# ---------------------------------------------------------------------------
# full hierarchy
# ---------------------------------------------------------------------------
class Hierarchy:
    """Oracle hierarchy built by or_setup; levels exported as numpy dicts."""

    def __init__(self, problem, theta, measure="material", max_coarse=5000, max_levels=10, seed=0,
                 power_iters=10, omega_sym=4.0 / 3.0, cheb_boost=1.1, cheb_ratio=30.0, drop="pointwise"):
        L = lib()
        self.dim = int(problem["dim"])
        self.n = int(problem["n"])
        o = _Opts(theta=float(theta), measure=MEASURES[measure], drop=DROPS[drop], max_coarse=int(max_coarse),
                  max_levels=int(max_levels), power_iters=int(power_iters), omega_sym=float(omega_sym),
                  cheb_boost=float(cheb_boost), cheb_ratio=float(cheb_ratio), seed=int(seed))
        self._keep = [_c(problem["row_ptr"], np.int64), _c(problem["col"], np.int32),
                      _c(problem["val"], np.float64), _c(problem["coords"], np.float64),
                      _c(problem["tensors"], np.float64)]
        tloc = 0 if problem.get("tloc", "element") == "node" else 1
        en = _c(problem.get("elem_nodes", np.zeros(1, np.int32)), np.int32)
        em = _c(problem.get("elem_measure", np.zeros(1)), np.float64)
        self._keep += [en, em]
        ne = em.size if tloc == 1 else 0
        npe = (en.size // max(ne, 1)) if tloc == 1 else 0
        st = ctypes.c_int(0)
        self.h = L.or_setup(self.dim, self.n, _p(self._keep[0]), _p(self._keep[1]), _p(self._keep[2]),
                            _p(self._keep[3]), tloc, _p(self._keep[4]), ne, npe, _p(en), _p(em),
                            ctypes.byref(o), ctypes.byref(st))
        self.status = st.value
        if not self.h:
            raise RuntimeError(f"oracle setup failed with status {st.value}")
        self.nlev = L.or_num_levels(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_free(self.h)
            self.h = None

    def level(self, l):
        L = lib()
        sz = np.zeros(5, np.int64)
        L.or_level_sizes(self.h, l, _p(sz))
        n, nnz, pnnz, nc, ngc = (int(x) for x in sz)
        kp = 6 if self.dim == 3 else 3
        d = dict(n=n, nnz=nnz, nnz_P=pnnz, nc=nc, nnz_gc=ngc,
                 A_rp=np.zeros(n + 1, np.int64), A_ci=np.zeros(max(nnz, 1), np.int32),
                 A_v=np.zeros(max(nnz, 1)), agg=np.full(n, -2, np.int32), root=np.zeros(n, np.uint8),
                 keep=np.zeros(max(nnz, 1), np.uint8), dir=np.zeros(n, np.uint8),
                 P_rp=np.zeros(n + 1, np.int64), P_ci=np.zeros(max(pnnz, 1), np.int32),
                 P_v=np.zeros(max(pnnz, 1)), x=np.zeros(n * self.dim), sinv=np.zeros(n * kp),
                 scalars=np.zeros(4))
        L.or_level_export(self.h, l, *(_p(d[k]) for k in ("A_rp", "A_ci", "A_v", "agg", "root", "keep", "dir",
                                                          "P_rp", "P_ci", "P_v", "x", "sinv", "scalars")))
        for k in ("A_ci", "A_v", "keep"):
            d[k] = d[k][:nnz]
        for k in ("P_ci", "P_v"):
            d[k] = d[k][:pnnz]
        d["omega"], d["lam_omega"], d["cheb_lmax"], d["cheb_lmin"] = (float(x) for x in d["scalars"])
        return d

    def set_cheb(self, l, lmax, lmin):
        """override the Chebyshev interval of level l (experiments only)"""
        lib().or_set_cheb(self.h, int(l), float(lmax), float(lmin))

    def operator_complexity(self):
        return float(lib().or_operator_complexity(self.h))

    def vcycle(self, b):
        z = np.zeros(self.n)
        lib().or_vcycle(self.h, _p(_c(b, np.float64)), _p(z))
        return z

    def solve(self, b, x0=None, tol=1e-8, maxit=500, flexible=False):
        x = np.zeros(self.n) if x0 is None else _c(x0, np.float64).copy()
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = lib().or_pcg(self.h, _p(_c(b, np.float64)), _p(x), float(tol), int(maxit), int(flexible),
                          ctypes.byref(it), ctypes.byref(rel))
        return x, dict(status=int(st), iters=int(it.value), rel_res=float(rel.value))

    def solve_hist(self, b, x0=None, tol=1e-8, maxit=500, flexible=False):
        """solve() plus the recursive residual history ||r_k|| / ||r_0||"""
        x = np.zeros(self.n) if x0 is None else _c(x0, np.float64).copy()
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        hist = np.full(maxit + 1, np.nan)
        st = lib().or_pcg_hist(self.h, _p(_c(b, np.float64)), _p(x), float(tol), int(maxit), int(flexible),
                               ctypes.byref(it), ctypes.byref(rel), _p(hist))
        return x, dict(status=int(st), iters=int(it.value), rel_res=float(rel.value), hist=hist[:it.value + 1])
