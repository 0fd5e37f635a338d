"""Seeded synthetic problems shaped like the paper's workloads.

Input generation only: Q1 finite-element assembly of -div(sigma grad u) = f
(the paper's Section 1) on tensor-product box meshes, material fields and
right-hand sides drawn from SplitMix64 (Steele, Lea & Flood 2014) with
Box-Muller normals.  Nothing in this module computes any part of the AMG
method; the CUDA library and the CPU oracle both consume its arrays.

Every problem is a dict with
  dim, n, nnz, row_ptr int64[n+1], col int32[nnz], val f64[nnz], b f64[n],
  coords f64[n*dim], tloc ('element'|'node'), tensors f64[(n_e|n)*(3|6)],
  elem_nodes int32[n_e*2^dim], elem_measure f64[n_e], dir_mask u8[n], meta.
Packed symmetric tensors: 2D (xx, yy, xy), 3D (xx, yy, zz, xy, xz, yz).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_q1gen.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the generator's C source into gen/_q1gen.so."""
    src = os.path.join(_HERE, "q1gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        L.q1_pattern_nnz.restype = ctypes.c_int64
        L.q1_pattern_nnz.argtypes = [ctypes.c_int] * 4
        L.q1_assemble.restype = ctypes.c_int64
        L.q1_assemble.argtypes = [ctypes.c_int] * 4 + [P] * 13
        L.q1_uniform.restype = None
        L.q1_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, P]
        L.q1_voronoi_regions.restype = None
        L.q1_voronoi_regions.argtypes = [ctypes.c_int] * 4 + [P, P]
        L.q1_mark_sphere.restype = ctypes.c_int64
        L.q1_mark_sphere.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [P]
        L.q1_annulus_nnz.restype = ctypes.c_int64
        L.q1_annulus_nnz.argtypes = [ctypes.c_int] * 3
        L.q1_assemble_annulus.restype = ctypes.c_int64
        L.q1_assemble_annulus.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [P, P] +
                                          [ctypes.c_double] * 2 + [P] * 8)
        _lib_handle = L
    return _lib_handle


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# seeded random numbers (SplitMix64 counter streams)
# ----------------------------------------------------------------------------
class Stream:
    """Counter-based uniform stream: draw k consumes k consecutive counters."""

    def __init__(self, seed: int, stream: int = 0):
        self.seed = (int(seed) * 0x100000001B3 + int(stream) * 0xC2B2AE3D27D4EB4F) % (1 << 64)
        self.k = 0

    def uniform(self, count: int) -> np.ndarray:
        out = np.empty(int(count), dtype=np.float64)
        if count:
            _lib().q1_uniform(ctypes.c_uint64(self.seed), ctypes.c_uint64(self.k), int(count), _p(out))
        self.k += int(count)
        return out

    def normal(self, count: int) -> np.ndarray:
        """Box-Muller: two uniforms per normal pair."""
        m = (int(count) + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0,1]
        z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
        return z[:count].copy()


# ----------------------------------------------------------------------------
# assembly wrapper
# ----------------------------------------------------------------------------
def assemble(dim, nx, ny, nz, xc, yc, zc, elem_K, elem_f, dir_mask, dir_val=None):
    L = _lib()
    nz_eff = nz if dim == 3 else 0
    Nx, Ny, Nz = nx + 1, ny + 1, (nz + 1 if dim == 3 else 1)
    n = Nx * Ny * Nz
    ne = nx * ny * (nz if dim == 3 else 1)
    nnz_max = L.q1_pattern_nnz(dim, nx, ny, nz_eff)
    row_ptr = np.empty(n + 1, np.int64)
    col = np.empty(nnz_max, np.int32)
    val = np.empty(nnz_max, np.float64)
    b = np.empty(n, np.float64)
    coords = np.empty(n * dim, np.float64)
    elem_nodes = np.empty(ne * (1 << dim), np.int32)
    elem_measure = np.empty(ne, np.float64)
    xc = np.ascontiguousarray(xc, np.float64)
    yc = np.ascontiguousarray(yc, np.float64)
    zc = np.ascontiguousarray(zc if zc is not None else np.zeros(1), np.float64)
    elem_K = np.ascontiguousarray(elem_K, np.float64)
    elem_f = None if elem_f is None else np.ascontiguousarray(elem_f, np.float64)
    dir_mask = np.ascontiguousarray(dir_mask, np.uint8)
    dir_val = None if dir_val is None else np.ascontiguousarray(dir_val, np.float64)
    nnz = L.q1_assemble(dim, nx, ny, nz_eff, _p(xc), _p(yc), _p(zc), _p(elem_K), _p(elem_f),
                        _p(dir_mask), _p(dir_val), _p(row_ptr), _p(col), _p(val), _p(b),
                        _p(coords), _p(elem_nodes), _p(elem_measure))
    if nnz < 0:
        raise ValueError("q1_assemble failed")
    return dict(dim=dim, n=n, nnz=int(nnz), row_ptr=row_ptr, col=col[:nnz].copy(),
                val=val[:nnz].copy(), b=b, coords=coords, elem_nodes=elem_nodes,
                elem_measure=elem_measure, dir_mask=dir_mask, n_elem=ne,
                grid=(nx, ny, nz if dim == 3 else 0))


def _node_ijk(dim, nx, ny, nz):
    Nx, Ny = nx + 1, ny + 1
    Nz = nz + 1 if dim == 3 else 1
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def _elem_ijk(dim, nx, ny, nz):
    ez_n = nz if dim == 3 else 1
    k, j, i = np.meshgrid(np.arange(ez_n), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def _iso(sig, dim):
    sig = np.asarray(sig, np.float64)
    out = np.zeros((sig.size, 3 if dim == 2 else 6))
    out[:, 0] = sig
    out[:, 1] = sig
    if dim == 3:
        out[:, 2] = sig
    return out


def _finish(p, tensors, name, **meta):
    p["tloc"] = "element"
    p["tensors"] = np.ascontiguousarray(tensors, np.float64).ravel()
    p["meta"] = dict(name=name, **meta)
    return p


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------
def layered_2d(n_el=32, contrast=1e-4, layer=4, seed=0):
    """Unit square, n_el^2 Q1 elements, isotropic sigma in horizontal layers of
    `layer` elements alternating 1 and `contrast` (bottom layer = 1),
    Dirichlet u=0 on x=0, Neumann elsewhere, f=1."""
    xc = np.linspace(0.0, 1.0, n_el + 1)
    ei, ej, _ = _elem_ijk(2, n_el, n_el, 0)
    sig = np.where((ej // layer) % 2 == 0, 1.0, contrast)
    K = _iso(sig, 2)
    ni, nj, _ = _node_ijk(2, n_el, n_el, 0)
    dmask = (ni == 0).astype(np.uint8)
    p = assemble(2, n_el, n_el, 0, xc, xc, None, K, np.ones(ei.size), dmask, None)
    return _finish(p, K, "layered_2d", n_el=n_el, contrast=contrast, layer=layer)


def battery_3d(nx=128, ny=128, nz=256, zratio=0.01, layer=8, sig=(1e5, 1e-5, 1e2), seed=0):
    """Battery-like stack: dx=dy=1/nx, dz=zratio*dx; repeating layer cycle of
    `layer` elements each with isotropic sigma values `sig`; u=0 at z=0,
    u=1 at the top, f=0."""
    dx = 1.0 / nx
    xc = np.arange(nx + 1) * dx
    yc = np.arange(ny + 1) * (1.0 / ny)
    zc = np.arange(nz + 1) * (zratio * dx)
    ei, ej, ek = _elem_ijk(3, nx, ny, nz)
    s = np.asarray(sig)[(ek // layer) % len(sig)]
    K = _iso(s, 3)
    ni, nj, nk = _node_ijk(3, nx, ny, nz)
    dmask = ((nk == 0) | (nk == nz)).astype(np.uint8)
    dval = np.where(nk == nz, 1.0, 0.0)
    p = assemble(3, nx, ny, nz, xc, yc, zc, K, None, dmask, dval)
    return _finish(p, K, "battery_3d", nx=nx, ny=ny, nz=nz, zratio=zratio, layer=layer, sig=list(sig))


def _quat_rot(u1, u2, u3):
    """Uniform random rotation from three uniforms (Shoemake 1992)."""
    a = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
    b = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
    c = math.sqrt(u1) * math.sin(2 * math.pi * u3)
    d = math.sqrt(u1) * math.cos(2 * math.pi * u3)
    w, x, y, z = d, a, b, c
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def voronoi_3d(n_el=160, nseeds=64, aniso=(1.0, 1e-3, 1e-3), seed=0):
    """[0,1]^3 with n_el^3 elements split into `nseeds` Voronoi regions of
    seeded points; per region K = R diag(aniso) R^T with a seeded uniform
    rotation R; f ~ U(0,1) per element; Dirichlet u=0 on x=0."""
    L = _lib()
    st = Stream(seed, 3)
    seeds = st.uniform(3 * nseeds)
    region = np.empty(n_el ** 3, np.int32)
    L.q1_voronoi_regions(n_el, n_el, n_el, nseeds, _p(seeds), _p(region))
    Ks = np.zeros((nseeds, 6))
    for s in range(nseeds):
        u = st.uniform(3)
        R = _quat_rot(u[0], u[1], u[2])
        M = R @ np.diag(aniso) @ R.T
        M = 0.5 * (M + M.T)
        Ks[s] = [M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]]
    K = Ks[region]
    f = st.uniform(n_el ** 3)
    xc = np.linspace(0.0, 1.0, n_el + 1)
    ni, _, _ = _node_ijk(3, n_el, n_el, n_el)
    dmask = (ni == 0).astype(np.uint8)
    p = assemble(3, n_el, n_el, n_el, xc, xc, xc, K, f, dmask, None)
    return _finish(p, K, "voronoi_3d", n_el=n_el, nseeds=nseeds, aniso=list(aniso))


def inclusions_3d(n_el=320, frac=0.2, rmin=4.0, rmax=12.0, sig_in=1e6,
                  matrix=(1.0, 1.0, 1e-2), nrhs=8, seed=0):
    """[0,1]^3 with n_el^3 elements; seeded random spheres (radius U(rmin,rmax)
    elements) added until >= frac of element centroids are inside; inside
    sigma = sig_in*I, matrix sigma = diag(matrix); Dirichlet u=0 on x=0;
    `nrhs` right-hand sides ~ N(0,1) on the free dofs (meta 'B')."""
    L = _lib()
    st = Stream(seed, 5)
    ne = n_el ** 3
    inside = np.zeros(ne, np.uint8)
    count = 0
    target = frac * ne
    while count < target:
        u = st.uniform(4)
        r = rmin + (rmax - rmin) * u[3]
        count += L.q1_mark_sphere(n_el, n_el, n_el, u[0] * n_el, u[1] * n_el, u[2] * n_el, r, _p(inside))
    K = np.zeros((ne, 6))
    K[:, 0] = np.where(inside == 1, sig_in, matrix[0])
    K[:, 1] = np.where(inside == 1, sig_in, matrix[1])
    K[:, 2] = np.where(inside == 1, sig_in, matrix[2])
    xc = np.linspace(0.0, 1.0, n_el + 1)
    ni, _, _ = _node_ijk(3, n_el, n_el, n_el)
    dmask = (ni == 0).astype(np.uint8)
    p = assemble(3, n_el, n_el, n_el, xc, xc, xc, K, None, dmask, None)
    B = st.normal(p["n"] * nrhs).reshape(nrhs, p["n"])
    B[:, dmask == 1] = 0.0
    p["B"] = B
    p["b"] = B[0].copy()
    return _finish(p, K, "inclusions_3d", n_el=n_el, frac=float(count / ne), nrhs=nrhs)


def two_domain(n_el=32, kappa=100.0, seed=0):
    """(-1,1)^2, sigma = I for x<0 and diag(kappa,1) for x>=0 (by element
    centroid), homogeneous Dirichlet on the whole boundary, f=1."""
    xc = np.linspace(-1.0, 1.0, n_el + 1)
    ei, ej, _ = _elem_ijk(2, n_el, n_el, 0)
    cx = 0.5 * (xc[ei] + xc[ei + 1])
    K = np.zeros((ei.size, 3))
    K[:, 0] = np.where(cx >= 0, kappa, 1.0)
    K[:, 1] = 1.0
    ni, nj, _ = _node_ijk(2, n_el, n_el, 0)
    dmask = ((ni == 0) | (ni == n_el) | (nj == 0) | (nj == n_el)).astype(np.uint8)
    p = assemble(2, n_el, n_el, 0, xc, xc, None, K, np.ones(ei.size), dmask, None)
    return _finish(p, K, "two_domain", n_el=n_el, kappa=kappa)


def worked_example(sig_low=1.0, kappa=100.0):
    """5x5-node / 4x4-element mesh of the paper's strength-of-connection
    illustration (nodes numbered 1..25 row by row, node 12=(1,2), 13=(2,2),
    14=(3,2)); pointwise nodal scalar sigma: sig_low for x<=1, kappa*sig_low
    for x>=2.  No boundary condition is eliminated."""
    n_el = 4
    xc = np.arange(n_el + 1, dtype=np.float64)
    ni, nj, _ = _node_ijk(2, n_el, n_el, 0)
    sig_node = np.where(ni <= 1, sig_low, kappa * sig_low)
    ei, ej, _ = _elem_ijk(2, n_el, n_el, 0)
    sig_el = np.where(ei + 0.5 < 1.5, sig_low, kappa * sig_low)
    Kel = _iso(sig_el, 2)
    p = assemble(2, n_el, n_el, 0, xc, xc, None, Kel, None, np.zeros(ni.size, np.uint8), None)
    p["tloc"] = "node"
    p["tensors"] = _iso(sig_node, 2).ravel()
    p["meta"] = dict(name="worked_example", sig_low=sig_low, kappa=kappa)
    return p


def layered_serving(dim, n_el, contrast, layer=4, seed=0):
    """Serving operator: 2D square or 3D cube, isotropic layered sigma
    alternating 1 and `contrast` in `layer`-element layers along the last
    axis, Dirichlet u=0 on x=0, f=1."""
    if dim == 2:
        return layered_2d(n_el, contrast, layer, seed)
    xc = np.linspace(0.0, 1.0, n_el + 1)
    ei, ej, ek = _elem_ijk(3, n_el, n_el, n_el)
    sig = np.where((ek // layer) % 2 == 0, 1.0, contrast)
    K = _iso(sig, 3)
    ni, _, _ = _node_ijk(3, n_el, n_el, n_el)
    dmask = (ni == 0).astype(np.uint8)
    p = assemble(3, n_el, n_el, n_el, xc, xc, xc, K, np.ones(ei.size), dmask, None)
    return _finish(p, K, "layered_3d", n_el=n_el, contrast=contrast, layer=layer)


def serving_requests(n_requests=512, seed=0, max2d=512, max3d=96, min_el=16):
    """Request list for the serving workload: operators with dim in {2,3}
    (p=1/2), elements per side log-uniform in [min_el, max2d] (2D) or
    [min_el, max3d] (3D), contrast 10^U(2,10); each operator gets U{1..16}
    consecutive right-hand-side requests; inter-arrival gaps ~ Exp(1) in
    units of the caller's mean gap.  Returns (operators, requests)."""
    st = Stream(seed, 4)
    ops, reqs = [], []
    while len(reqs) < n_requests:
        u = st.uniform(4)
        dim = 2 if u[0] < 0.5 else 3
        hi = max2d if dim == 2 else max3d
        n_el = int(round(math.exp(math.log(min_el) + u[1] * (math.log(hi) - math.log(min_el)))))
        contrast = 10.0 ** (2.0 + 8.0 * u[2])
        k = 1 + min(15, int(u[3] * 16))
        oid = len(ops)
        ops.append(dict(dim=dim, n_el=n_el, contrast=contrast, seed=oid))
        for r in range(k):
            if len(reqs) >= n_requests:
                break
            gap = -math.log1p(-st.uniform(1)[0])
            reqs.append(dict(op=oid, rhs_seed=len(reqs), gap=gap))
    return ops, reqs


def annulus_tensors(coords, elem_nodes, kappa):
    """Per element K = Q^T diag(kappa, 1, 1) Q at the element centroid, with
    Q's rows the circumferential unit vector (-y, x, 0)/r, the radial unit
    vector (x, y, 0)/r and e_z: conductivity kappa along the circle, 1 across
    it.  Packed (xx, yy, zz, xy, xz, yz)."""
    X = coords.reshape(-1, 3)[elem_nodes.reshape(-1, 8)].mean(axis=1)
    r = np.hypot(X[:, 0], X[:, 1])
    tx, ty = -X[:, 1] / r, X[:, 0] / r
    rx, ry = X[:, 0] / r, X[:, 1] / r
    K = np.zeros((X.shape[0], 6))
    K[:, 0] = kappa * tx * tx + rx * rx
    K[:, 1] = kappa * ty * ty + ry * ry
    K[:, 2] = 1.0
    K[:, 3] = kappa * tx * ty + rx * ry
    return K


def annulus_3d(refine=0, kappa=100.0, ri=0.5, ro=1.0, t=0.1, base=(20, 150, 1), g_in=0.0, g_out=1.0,
               load=True, seed=0):
    """Thick annulus r_i <= r <= r_o, 0 <= z <= t, meshed with
    base * 2^refine trilinear hexahedra (radial, circumferential, thickness),
    conductivity kappa along the circumference and 1 radially and through
    the thickness; Dirichlet u = g_in on the inner and u = g_out on the outer
    cylinder, natural conditions on the two flat faces.  With `load`, a
    seeded element load f ~ U(0,1) (so that the right-hand side is not
    rotation invariant); without it f = 0 and the exact solution of the
    continuous problem is ln(r/r_i)/ln(r_o/r_i) scaled to g_in..g_out."""
    L = _lib()
    m = 1 << int(refine)
    nr, nt, nz = base[0] * m, base[1] * m, base[2] * m
    n = (nr + 1) * nt * (nz + 1)
    ne = nr * nt * nz
    nnz_max = L.q1_annulus_nnz(nr, nt, nz)
    row_ptr = np.empty(n + 1, np.int64)
    col = np.empty(nnz_max, np.int32)
    val = np.empty(nnz_max, np.float64)
    b = np.empty(n, np.float64)
    coords = np.empty(3 * n, np.float64)
    elem_nodes = np.empty(8 * ne, np.int32)
    elem_measure = np.empty(ne, np.float64)
    dmask = np.empty(n, np.uint8)
    # the element tensors depend only on the (closed-form) node coordinates
    a = np.arange(nr + 1)
    bq = np.arange(nt)
    c = np.arange(nz + 1)
    C, B, A = np.meshgrid(c, bq, a, indexing="ij")
    rad = ri + (ro - ri) * A.ravel() / nr
    phi = 2.0 * math.pi * B.ravel() / nt
    xyz = np.stack([rad * np.cos(phi), rad * np.sin(phi), t * C.ravel() / nz], axis=1).ravel()
    ec, eb, ea = np.meshgrid(np.arange(nz), np.arange(nt), np.arange(nr), indexing="ij")
    ea, eb, ec = ea.ravel(), eb.ravel(), ec.ravel()
    en = np.stack([(ea + (l & 1)) + (nr + 1) * (((eb + ((l >> 1) & 1)) % nt) + nt * (ec + ((l >> 2) & 1)))
                   for l in range(8)], axis=1)
    K = np.ascontiguousarray(annulus_tensors(xyz, en, kappa))
    f = Stream(seed, 6).uniform(ne) if load else None
    nnz = L.q1_assemble_annulus(nr, nt, nz, ri, ro, t, _p(K), _p(f), g_in, g_out, _p(row_ptr), _p(col), _p(val),
                                _p(b), _p(coords), _p(elem_nodes), _p(elem_measure), _p(dmask))
    if nnz < 0:
        raise ValueError("q1_assemble_annulus failed")
    p = dict(dim=3, n=n, nnz=int(nnz), row_ptr=row_ptr, col=col[:nnz].copy(), val=val[:nnz].copy(), b=b,
             coords=coords, elem_nodes=elem_nodes, elem_measure=elem_measure, dir_mask=dmask, n_elem=ne,
             grid=(nr, nt, nz))
    return _finish(p, K, "annulus_3d", refine=refine, kappa=kappa, nr=nr, nt=nt, nz=nz, load=load)


CONFIGS = {
    "c1": lambda **kw: layered_2d(**kw),
    "c2": lambda **kw: battery_3d(**kw),
    "c3": lambda **kw: voronoi_3d(**kw),
    "c5": lambda **kw: inclusions_3d(**kw),
    "annulus": lambda **kw: annulus_3d(**kw),
}


def make_problem(name: str, **kw):
    """Named workloads: c1 layered 2D (32^2), c2 battery stack (128x128x256),
    c3 rotated-anisotropy Voronoi (160^3), c5 inclusions (320^3); keyword
    overrides shrink them for tests."""
    return CONFIGS[name](**kw)
