"""Thin ctypes binding of the C ABI declared in include/sa.h.

Argument marshalling only: device memory and the stream come from PyTorch,
every numerical step runs in the CUDA library.  There is no CPU fallback:
loading fails loudly when the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_SPD, ERR_STAGNATION, ERR_NO_CONVERGENCE, ERR_BREAKDOWN, \
    ERR_CAPACITY = 0, -1, -2, -3, -4, -5, -6, -7, -8
MEASURE = {"classical": 0, "material": 1, "distance": 2}
PRECISION = {"fp64": 0, "fp32": 1}
DROP = {"pointwise": 0, "cut": 1}

EXPORTED = ["sa_default_options", "sa_setup", "sa_solve", "sa_solve_batch", "sa_solve_batch_zero", "sa_solve_group", "sa_vcycle", "sa_hierarchy_stats",
            "sa_level_sizes", "sa_level_format", "sa_export_level", "sa_export_strength", "sa_free",
            "sa_status_string", "sa_last_error", "sa_strength", "sa_set_precision", "sa_profile_enable", "sa_profile_read",
            "sa_launch_count", "sa_strength_material_noalloc", "sa_serialized_size", "sa_serialize",
            "sa_deserialize"]


class SAError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: status {status}")


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("host", ctypes.c_int), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("coords", ctypes.c_void_p), ("tloc", ctypes.c_int), ("tensors", ctypes.c_void_p),
                ("n_elem", ctypes.c_int64), ("nodes_per_elem", ctypes.c_int), ("elem_nodes", ctypes.c_void_p),
                ("elem_measure", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("measure", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_coarse", ctypes.c_int), ("max_levels", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("cheb_ratio", ctypes.c_double), ("cheb_boost", ctypes.c_double), ("power_iters", ctypes.c_int),
                ("omega_sym", ctypes.c_double), ("seed", ctypes.c_uint32), ("maxit", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("alloc", _ALLOC), ("dealloc", _FREE),
                ("alloc_ctx", ctypes.c_void_p), ("keep_setup_data", ctypes.c_int), ("drop", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res_true", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("status", ctypes.c_int)]


_L = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libsa_gb300.so (building it when stale); raises if it cannot be loaded."""
    global _L
    if _L is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library missing: {_build.LIB} (run build())")
        L = ctypes.CDLL(_build.LIB)
        P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.sa_default_options.argtypes = [ctypes.POINTER(Options)]
        L.sa_setup.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]
        L.sa_solve.argtypes = [P, P, P, D, ctypes.POINTER(SolveInfo)]
        L.sa_solve_batch.argtypes = [P, I, P, P, D, ctypes.POINTER(SolveInfo)]
        L.sa_solve_batch_zero.argtypes = [P, I, P, P, D, ctypes.POINTER(SolveInfo)]
        L.sa_vcycle.argtypes = [P, P, P]
        L.sa_hierarchy_stats.argtypes = [P, P, P, P, P, P]
        L.sa_level_sizes.argtypes = [P, I, P]
        L.sa_level_format.argtypes = [P, I, P]
        L.sa_export_level.argtypes = [P, I] + [P] * 7
        L.sa_export_strength.argtypes = [P, I] + [P] * 6
        L.sa_free.argtypes = [P]
        L.sa_status_string.argtypes = [I]
        L.sa_status_string.restype = ctypes.c_char_p
        L.sa_last_error.argtypes = []
        L.sa_last_error.restype = ctypes.c_char_p
        L.sa_strength.argtypes = [I, I, I64, I64, P, P, P, P, P, P, D, P, P]
        L.sa_set_precision.argtypes = [P, I]
        L.sa_profile_enable.argtypes = [I]
        L.sa_profile_read.argtypes = [I, P, P, P, P, P, P]
        L.sa_strength_material_noalloc.argtypes = [I, I64, I64, P, P, P, P, P, D, P, P]
        L.sa_strength_material_noalloc.restype = I
        L.sa_launch_count.argtypes = []
        L.sa_launch_count.restype = ctypes.c_int64
        L.sa_serialized_size.argtypes = [P, P]
        L.sa_serialize.argtypes = [P, P, ctypes.c_uint64]
        L.sa_deserialize.argtypes = [P, ctypes.c_uint64, P, P]
        L.sa_solve_group.argtypes = [I, P, P, P, D, P]
        for f in ("sa_default_options", "sa_setup", "sa_solve", "sa_solve_batch", "sa_solve_batch_zero",
                  "sa_solve_group", "sa_vcycle",
                  "sa_hierarchy_stats", "sa_level_sizes", "sa_level_format", "sa_export_level",
                  "sa_export_strength", "sa_free",
                  "sa_strength", "sa_set_precision", "sa_profile_enable", "sa_profile_read",
                  "sa_serialized_size", "sa_serialize", "sa_deserialize"):
            getattr(L, f).restype = I
        _L = L
    return _L


def _check(st, what):
    if st != OK:
        L = lib(False)
        msg = L.sa_status_string(st).decode()
        err = L.sa_last_error().decode()
        raise SAError(st, f"{what} failed: {msg} {err}".strip())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the SA-AMG library has no CPU path")
    return torch


def _dev(a, dtype, torch):
    """numpy array or torch tensor -> contiguous CUDA tensor of dtype"""
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=dtype).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def default_options() -> Options:
    o = Options()
    _check(lib().sa_default_options(ctypes.byref(o)), "sa_default_options")
    return o


class Hierarchy:
    """A device-resident SA-AMG hierarchy (sa_setup) with solve / export calls."""

    def __init__(self, problem, theta=0.08, measure="material", precision="fp64", max_coarse=5000,
                 max_levels=10, seed=0, maxit=500, keep_setup_data=False, host_inputs=False, stream=None,
                 cheb_degree=2, power_iters=10, drop="pointwise"):
        torch = _torch()
        L = lib()
        self.torch = torch
        self.n = int(problem["n"])
        self.dim = int(problem["dim"])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = default_options()
        o.theta = float(theta)
        o.measure = MEASURE[measure]
        o.precision = PRECISION[precision]
        o.max_coarse = int(max_coarse)
        o.max_levels = int(max_levels)
        o.seed = int(seed)
        o.maxit = int(maxit)
        o.keep_setup_data = int(keep_setup_data)
        o.cheb_degree = int(cheb_degree)
        o.power_iters = int(power_iters)
        o.drop = DROP[drop]
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.opts = o
        pr = Problem()
        pr.dim = self.dim
        pr.n = self.n
        pr.nnz = int(problem["nnz"])
        node_t = problem.get("tloc", "element") == "node"
        pr.tloc = 0 if node_t else 1
        if host_inputs:
            keep = [np.ascontiguousarray(problem["row_ptr"], np.int64), np.ascontiguousarray(problem["col"], np.int32),
                    np.ascontiguousarray(problem["val"], np.float64),
                    np.ascontiguousarray(problem["coords"], np.float64),
                    np.ascontiguousarray(problem["tensors"], np.float64),
                    np.ascontiguousarray(problem.get("elem_nodes", np.zeros(1, np.int32)), np.int32),
                    np.ascontiguousarray(problem.get("elem_measure", np.zeros(1)), np.float64)]
            ptr = [k.ctypes.data for k in keep]
            pr.host = 1
        else:
            keep = [_dev(problem["row_ptr"], torch.int64, torch), _dev(problem["col"], torch.int32, torch),
                    _dev(problem["val"], torch.float64, torch), _dev(problem["coords"], torch.float64, torch),
                    _dev(problem["tensors"], torch.float64, torch),
                    _dev(problem.get("elem_nodes", np.zeros(1, np.int32)), torch.int32, torch),
                    _dev(problem.get("elem_measure", np.zeros(1)), torch.float64, torch)]
            ptr = [k.data_ptr() for k in keep]
        pr.row_ptr, pr.col, pr.val, pr.coords, pr.tensors, pr.elem_nodes, pr.elem_measure = ptr
        if not node_t:
            pr.n_elem = int(len(problem["elem_measure"]))
            pr.nodes_per_elem = int(len(problem["elem_nodes"]) // max(pr.n_elem, 1))
        h = ctypes.c_void_p()
        st = L.sa_setup(ctypes.byref(pr), ctypes.byref(o), ctypes.byref(h))
        del keep
        _check(st, "sa_setup")
        self.h = h

    # -- store ---------------------------------------------------------------
    def to_bytes(self):
        """The stored FP64 hierarchy (sa_serialize) as a numpy uint8 array."""
        nb = ctypes.c_uint64()
        _check(lib().sa_serialized_size(self.h, ctypes.byref(nb)), "sa_serialized_size")
        buf = np.empty(nb.value, np.uint8)
        _check(lib().sa_serialize(self.h, buf.ctypes.data, nb.value), "sa_serialize")
        return buf

    def save(self, path):
        self.to_bytes().tofile(path)

    @classmethod
    def from_bytes(cls, buf, precision="fp64", maxit=500, stream=None):
        """A handle rebuilt from a store (sa_deserialize) without re-running the
        setup; the setup options come from the store."""
        torch = _torch()
        buf = np.ascontiguousarray(np.frombuffer(buf, np.uint8) if isinstance(buf, (bytes, bytearray)) else buf,
                                   np.uint8)
        self = cls.__new__(cls)
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = default_options()
        o.precision = PRECISION[precision]
        o.maxit = int(maxit)
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        h = ctypes.c_void_p()
        _check(lib().sa_deserialize(buf.ctypes.data, buf.size, ctypes.byref(o), ctypes.byref(h)), "sa_deserialize")
        self.h = h
        self.opts = o
        st = self.stats()
        self.n = int(st["n"][0])
        self.dim = int(np.frombuffer(buf[16:20].tobytes(), np.int32)[0])  # header field after magic, version, order
        return self

    @classmethod
    def load(cls, path, **kw):
        return cls.from_bytes(np.fromfile(path, np.uint8), **kw)

    # -- lifetime ------------------------------------------------------------
    def free(self):
        if getattr(self, "h", None):
            lib(False).sa_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # -- solve ---------------------------------------------------------------
    def solve(self, b, x0=None, tol=1e-8, check=True):
        """b, x0: CUDA tensors (float64) or numpy arrays (host path). Returns (x, info dict)."""
        torch = self.torch
        info = SolveInfo()
        if isinstance(b, torch.Tensor):
            with torch.cuda.stream(self.stream):  # x is written on the handle's stream
                x = torch.zeros(self.n, dtype=torch.float64, device="cuda") if x0 is None else x0.clone()
            st = lib().sa_solve(self.h, b.data_ptr(), x.data_ptr(), float(tol), ctypes.byref(info))
        else:
            bb = np.ascontiguousarray(b, np.float64)
            x = np.zeros(self.n) if x0 is None else np.array(x0, np.float64)
            st = lib().sa_solve(self.h, bb.ctypes.data, x.ctypes.data, float(tol), ctypes.byref(info))
        if check and st not in (OK, ERR_NO_CONVERGENCE):
            _check(st, "sa_solve")
        return x, dict(status=int(st), iters=info.iters, rel_res=info.rel_res_true, setup_ms=info.setup_ms,
                       solve_ms=info.solve_ms)

    def solve_batch(self, B, X0=None, tol=1e-8, check=True, out=None):
        """k right-hand sides at once (sa_solve_batch: up to 8 columns share every
        launch; each column ends bitwise where solve() on it ends).  B: (k, n)
        CUDA tensor (float64) or numpy array; returns (X of the same kind,
        list of per-column info dicts).  Host path: `out` (a C-contiguous
        float64 (k, n) numpy array, e.g. a view of pinned memory) receives X.
        Without X0 the solve starts from zero through sa_solve_batch_zero (X
        is output only: no buffer of zeros is filled or copied)."""
        torch = self.torch
        if isinstance(B, torch.Tensor):
            B = B.to(device="cuda", dtype=torch.float64).contiguous()
            k = int(B.shape[0])
            with torch.cuda.stream(self.stream):
                X = torch.empty_like(B) if X0 is None else X0.to(device="cuda", dtype=torch.float64).clone()
            bp, xp = B.data_ptr(), X.data_ptr()
        else:
            B = np.ascontiguousarray(B, np.float64)
            k = int(B.shape[0])
            if out is not None:
                if out.shape != B.shape or out.dtype != np.float64 or not out.flags.c_contiguous:
                    raise ValueError("solve_batch: out must be a C-contiguous float64 array shaped like B")
                X = out
                if X0 is not None:
                    X[...] = X0
            else:
                X = np.empty_like(B) if X0 is None else np.array(X0, np.float64)
            bp, xp = B.ctypes.data, X.ctypes.data
        infos = (SolveInfo * max(k, 1))()
        entry = lib().sa_solve_batch_zero if X0 is None else lib().sa_solve_batch
        st = entry(self.h, k, bp, xp, float(tol), infos)
        if check and st not in (OK, ERR_NO_CONVERGENCE):
            _check(st, "sa_solve_batch")
        return X, [dict(status=int(infos[c].status), iters=infos[c].iters, rel_res=infos[c].rel_res_true,
                        setup_ms=infos[c].setup_ms, solve_ms=infos[c].solve_ms) for c in range(k)]

    def set_precision(self, precision):
        _check(lib().sa_set_precision(self.h, PRECISION[precision]), "sa_set_precision")

    def vcycle(self, r):
        with self.torch.cuda.stream(self.stream):
            z = self.torch.empty_like(r)
        _check(lib().sa_vcycle(self.h, r.data_ptr(), z.data_ptr()), "sa_vcycle")
        return z

    # -- inspection ----------------------------------------------------------
    def stats(self):
        lv = ctypes.c_int()
        nl = np.zeros(32, np.int64)
        nz = np.zeros(32, np.int64)
        oc = ctypes.c_double()
        db = ctypes.c_int64()
        _check(lib().sa_hierarchy_stats(self.h, ctypes.byref(lv), nl.ctypes.data, nz.ctypes.data, ctypes.byref(oc),
                                        ctypes.byref(db)), "sa_hierarchy_stats")
        k = lv.value
        return dict(levels=k, n=nl[:k].tolist(), nnz=nz[:k].tolist(), op_complexity=oc.value,
                    device_bytes=db.value)

    def level_sizes(self, l):
        out = np.zeros(5, np.int64)
        _check(lib().sa_level_sizes(self.h, int(l), out.ctypes.data), "sa_level_sizes")
        return dict(n=int(out[0]), nnz=int(out[1]), nnz_P=int(out[2]), nc=int(out[3]), nnz_gc=int(out[4]))

    def level_format(self, l):
        """storage of the FP64 V-cycle operator of level l: CSR lanes (0 = SELL-32,
        -1 = dense coarsest level), rows in the long-row bin, its threshold
        (-1: none), stored entries, SELL-32 lanes per row"""
        out = np.zeros(5, np.int64)
        _check(lib().sa_level_format(self.h, int(l), out.ctypes.data), "sa_level_format")
        return dict(lanes=int(out[0]), nlong=int(out[1]), long_threshold=int(out[2]), stored=int(out[3]),
                    sell_lanes=int(out[4]))

    def export_level(self, l):
        s = self.level_sizes(l)
        n, nnz, pn = s["n"], s["nnz"], s["nnz_P"]
        d = dict(s, A_rp=np.zeros(n + 1, np.int64), A_ci=np.zeros(max(nnz, 1), np.int32), A_v=np.zeros(max(nnz, 1)),
                 agg=np.full(n, -2, np.int32), P_rp=np.zeros(n + 1, np.int64), P_ci=np.zeros(max(pn, 1), np.int32),
                 P_v=np.zeros(max(pn, 1)))
        _check(lib().sa_export_level(self.h, int(l), d["agg"].ctypes.data, d["P_rp"].ctypes.data,
                                     d["P_ci"].ctypes.data, d["P_v"].ctypes.data, d["A_rp"].ctypes.data,
                                     d["A_ci"].ctypes.data, d["A_v"].ctypes.data), "sa_export_level")
        d["A_ci"], d["A_v"] = d["A_ci"][:nnz], d["A_v"][:nnz]
        d["P_ci"], d["P_v"] = d["P_ci"][:pn], d["P_v"][:pn]
        return d

    def export_strength(self, l, keep=True, root=True, aux=True):
        s = self.level_sizes(l)
        n, nnz = s["n"], s["nnz"]
        kp = 6 if self.dim == 3 else 3
        out = dict(keep=np.zeros(max(nnz, 1), np.uint8) if keep else None,
                   root=np.zeros(n, np.uint8) if root else None, dir=np.zeros(n, np.uint8),
                   x=np.zeros(n * self.dim) if aux else None, sinv=np.zeros(n * kp) if aux else None,
                   scalars=np.zeros(4))
        ptr = [None if out[k] is None else out[k].ctypes.data for k in ("keep", "root", "dir", "x", "sinv", "scalars")]
        _check(lib().sa_export_strength(self.h, int(l), *ptr), "sa_export_strength")
        if keep:
            out["keep"] = out["keep"][:nnz]
        out["omega"], out["lam_omega"], out["cheb_lmax"], out["cheb_lmin"] = (float(v) for v in out["scalars"])
        return out


def solve_group(hierarchies, rhs, tol=1e-8, x0=None, check=True):
    """sa_solve_group: one right-hand side per hierarchy (distinct handles with
    the same precision setting), all problems advanced together in shared
    launches on the first hierarchy's stream.  rhs: list of CUDA tensors
    (float64, n_i each); returns (list of solutions, list of info dicts)."""
    torch = _torch()
    m = len(hierarchies)
    if m != len(rhs):
        raise ValueError("solve_group: one right-hand side per hierarchy")
    st0 = hierarchies[0].stream
    B = [b.to(device="cuda", dtype=torch.float64).contiguous() for b in rhs]
    with torch.cuda.stream(st0):
        X = [torch.zeros_like(b) if x0 is None else x0[k].to(device="cuda", dtype=torch.float64).clone()
             for k, b in enumerate(B)]
    hs = (ctypes.c_void_p * m)(*[h.h.value for h in hierarchies])
    bp = (ctypes.c_void_p * m)(*[b.data_ptr() for b in B])
    xp = (ctypes.c_void_p * m)(*[x.data_ptr() for x in X])
    infos = (SolveInfo * max(m, 1))()
    st = lib().sa_solve_group(m, hs, bp, xp, float(tol), infos)
    if check and st not in (OK, ERR_NO_CONVERGENCE):
        _check(st, "sa_solve_group")
    return X, [dict(status=int(infos[c].status), iters=infos[c].iters, rel_res=infos[c].rel_res_true,
                    setup_ms=infos[c].setup_ms, solve_ms=infos[c].solve_ms) for c in range(m)]


def strength(measure, dim, row_ptr, col, val, coords, sigma_inv, dirichlet, theta, stream=None):
    """sa_strength on CUDA tensors; returns the keep mask (uint8 CUDA tensor)."""
    torch = _torch()
    n = row_ptr.numel() - 1
    nnz = col.numel()
    keep = torch.empty(max(nnz, 1), dtype=torch.uint8, device="cuda")
    s = (stream or torch.cuda.current_stream()).cuda_stream

    def P(t):
        return None if t is None else t.data_ptr()

    _check(lib().sa_strength(MEASURE[measure], int(dim), n, nnz, P(row_ptr), P(col), P(val), P(coords),
                             P(sigma_inv), P(dirichlet), float(theta), P(keep), ctypes.c_void_p(s)), "sa_strength")
    return keep[:nnz]


PROFILE_KINDS = ["cheb64", "resid64", "restrict64", "prolong64", "first64", "cg_spmv", "cg_vec", "coarse",
                 "cheb32", "resid32", "restrict32", "prolong32", "first32",
                 "setup_nodal", "setup_strength", "setup_graph", "setup_mis2", "setup_aggregate", "setup_filter",
                 "setup_omega", "setup_smooth_p", "setup_transpose", "setup_galerkin", "setup_aux",
                 "setup_cheb_bounds", "setup_dense", "setup_sell", "setup_galerkin_ap", "setup_galerkin_rap",
                 "bcheb64", "bresid64", "brestrict64", "bprolong64", "bfirst64", "bcoarse",
                 "bcheb32", "bresid32", "brestrict32", "bprolong32", "bfirst32", "bcg_spmv", "bcg_vec"]


def profile_enable(on=True):
    _check(lib().sa_profile_enable(1 if on else 0), "sa_profile_enable")


def profile_read():
    """rows of (kind, level, launches, total_ms, bytes) aggregated since profile_enable(True)"""
    n = ctypes.c_int()
    _check(lib().sa_profile_read(0, None, None, None, None, None, ctypes.byref(n)), "sa_profile_read")
    k = max(n.value, 1)
    kind = np.zeros(k, np.int32)
    lev = np.zeros(k, np.int32)
    cnt = np.zeros(k, np.int64)
    ms = np.zeros(k)
    by = np.zeros(k)
    _check(lib().sa_profile_read(k, kind.ctypes.data, lev.ctypes.data, cnt.ctypes.data, ms.ctypes.data,
                                 by.ctypes.data, ctypes.byref(n)), "sa_profile_read")
    return [dict(kind=PROFILE_KINDS[kind[j]], level=int(lev[j]), launches=int(cnt[j]), ms=float(ms[j]),
                 bytes=float(by[j])) for j in range(n.value)]


def launch_count():
    """kernel launches issued by the library in this process"""
    return int(lib().sa_launch_count())


def strength_material_noalloc(dim, row_ptr, col, coords, sigma_inv, dirichlet, theta, keep, stream=None):
    """sa_strength_material_noalloc on CUDA tensors; writes the keep mask into
    the caller's `keep` (uint8, nnz) and returns the status (no allocation
    inside the call)"""
    torch = _torch()
    n = row_ptr.numel() - 1
    nnz = col.numel()
    for t, dt, size, name in ((row_ptr, torch.int64, n + 1, "row_ptr"), (col, torch.int32, nnz, "col"),
                              (coords, torch.float64, n * dim, "coords"),
                              (sigma_inv, torch.float64, n * (6 if dim == 3 else 3), "sigma_inv"),
                              (dirichlet, torch.uint8, n, "dirichlet"), (keep, torch.uint8, nnz, "keep")):
        if t is None and name == "dirichlet":
            continue
        if t is None or t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() < size:
            raise ValueError(f"strength_material_noalloc: {name} must be a contiguous CUDA {dt} tensor "
                             f"of at least {size} elements")
    s = (stream or torch.cuda.current_stream()).cuda_stream

    def P(t):
        return None if t is None else t.data_ptr()

    return int(lib().sa_strength_material_noalloc(int(dim), n, nnz, P(row_ptr), P(col), P(coords), P(sigma_inv),
                                                  P(dirichlet), float(theta), P(keep), ctypes.c_void_p(s)))
