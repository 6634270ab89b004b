"""Python access to the plain FP64 CPU oracle (oracle/nl_oracle.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package.  The product library never
does, and the oracle shares no code with it.

Every function restates one definition of the paper (arXiv 2101.08825); the C file
cites the section, equation or algorithm of each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nl_oracle.c")
_LIB = os.path.join(_HERE, "libnloracle.so")
_lib = None

KERNEL_CONST = 0
KERNEL_GAUSS = 1


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2 -ffp-contract=off: no fused multiply-adds, so the
    decisions of Algorithm 1 round exactly as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nl_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_vert", ctypes.c_int64), ("n_elem", ctypes.c_int64),
                ("coords", ctypes.c_void_p), ("conn", ctypes.c_void_p),
                ("elem_in_omega", ctypes.c_void_p), ("node_free", ctypes.c_void_p),
                ("order", ctypes.c_int), ("cell", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("eps", ctypes.c_double), ("C", ctypes.c_double),
                ("kernel", ctypes.c_int), ("L_min", ctypes.c_int), ("L_max", ctypes.c_int),
                ("flags", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("n_point_pairs", ctypes.c_int64), ("n_band_pairs", ctypes.c_int64),
                ("n_integrations", ctypes.c_int64)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.or_xi.restype = d
        L.or_xi.argtypes = [d]
        L.or_mu.restype = d
        L.or_mu.argtypes = [d, d, d]
        L.or_eta.restype = d
        L.or_eta.argtypes = [i, d, d]
        L.or_kernel_constant.restype = d
        L.or_kernel_constant.argtypes = [i, i, d, d]
        L.or_kernel_moment.restype = d
        L.or_kernel_moment.argtypes = [i, i, d, d, d, i]
        L.or_gauss_legendre.argtypes = [i, p, p]
        L.or_quad_rule.argtypes = [i, p, p]
        L.or_aprx_max_dist.restype = d
        L.or_aprx_max_dist.argtypes = [i, p, p, p, p]
        L.or_aprx_min_dist.restype = d
        L.or_aprx_min_dist.argtypes = [i, p, p, p, p]
        L.or_aprx_min_dist_l2.restype = d
        L.or_aprx_min_dist_l2.argtypes = [i, p, p, p, p]
        L.or_pairs.restype = i64
        L.or_pairs.argtypes = [ctypes.POINTER(_Mesh), d, d, p, p, i64, p]
        L.or_csr.restype = i64
        L.or_csr.argtypes = [ctypes.POINTER(_Mesh), p, p, p, p, i64]
        L.or_assemble.argtypes = [ctypes.POINTER(_Mesh), p, p, ctypes.POINTER(_Params), p, p, p,
                                  p, ctypes.POINTER(_Stats)]
        L.or_ms_u.restype = d
        L.or_ms_u.argtypes = [i, i, p]
        L.or_ms_f.restype = d
        L.or_ms_f.argtypes = [i, i, p, i, d, d, d]
        L.or_rhs.argtypes = [ctypes.POINTER(_Mesh), p, p, p, i, i, d, d, d, p]
        L.or_solve_dense.argtypes = [ctypes.POINTER(_Mesh), p, p, p, p, i, p]
        L.or_l2_error.restype = d
        L.or_l2_error.argtypes = [ctypes.POINTER(_Mesh), p, i, i]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OMesh:
    """Keeps the contiguous arrays alive next to the C view of a mesh."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.dim = mesh.dim
        self.coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
        self.conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
        self.elem_in_omega = np.ascontiguousarray(mesh.elem_in_omega, dtype=np.uint8)
        self.node_free = np.ascontiguousarray(mesh.node_free, dtype=np.uint8)
        # nodes per element -> element kind: 2D 3 P1 / 6 P2 triangles, 4 Q1 / 9 Q2 / 8
        # serendipity quadrilaterals (order 3); 3D 4 P1 / 10 P2 tetrahedra, 8 Q1 / 27 Q2 / 20
        # serendipity hexahedra (cell 2)
        npe = self.conn.shape[1]
        self.cell = 1 if (self.dim == 2 and npe in (4, 8, 9)) else (2 if (self.dim == 3 and npe in (8, 20, 27)) else 0)
        self.order = 2 if (npe in (6, 9, 27) or (self.dim == 3 and npe == 10)) else \
            (3 if ((self.cell == 1 and npe == 8) or (self.cell == 2 and npe == 20)) else 1)
        self.c = _Mesh(self.dim, self.coords.shape[1], self.conn.shape[0], _ptr(self.coords).value,
                       _ptr(self.conn).value, _ptr(self.elem_in_omega).value,
                       _ptr(self.node_free).value, self.order, self.cell)


def _om(mesh) -> OMesh:
    return mesh if isinstance(mesh, OMesh) else OMesh(mesh)


# ---- scalar definitions -------------------------------------------------------------

def xi(s: float) -> float:
    return lib().or_xi(float(s))


def mu(r: float, delta: float, eps: float) -> float:
    return lib().or_mu(float(r), float(delta), float(eps))


def eta(kernel: int, r: float, delta: float) -> float:
    return lib().or_eta(int(kernel), float(r), float(delta))


def kernel_constant(dim: int, kernel: int, delta: float, eps: float) -> float:
    return lib().or_kernel_constant(dim, kernel, delta, eps)


def kernel_moment(dim: int, kernel: int, delta: float, eps: float, C: float, p: int) -> float:
    return lib().or_kernel_moment(dim, kernel, delta, eps, C, p)


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def quad_rule(dim: int):
    """(bary (nq, dim+1), weights (nq,) summing to 1) of the degree-5 simplex rule."""
    b = np.zeros(64)
    w = np.zeros(16)
    n = lib().or_quad_rule(dim, _ptr(b), _ptr(w))
    if n <= 0:
        raise RuntimeError("oracle quadrature rule did not converge")
    return b[: n * (dim + 1)].reshape(n, dim + 1).copy(), w[:n].copy()


def aprx_max_dist(lo1, hi1, lo2, hi2) -> float:
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (lo1, hi1, lo2, hi2)]
    return lib().or_aprx_max_dist(len(a[0]), *[_ptr(v) for v in a])


def aprx_min_dist(lo1, hi1, lo2, hi2) -> float:
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (lo1, hi1, lo2, hi2)]
    return lib().or_aprx_min_dist(len(a[0]), *[_ptr(v) for v in a])


def aprx_min_dist_l2(lo1, hi1, lo2, hi2) -> float:
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (lo1, hi1, lo2, hi2)]
    return lib().or_aprx_min_dist_l2(len(a[0]), *[_ptr(v) for v in a])


# ---- pairs, pattern, assembly --------------------------------------------------------

def pairs(mesh, delta: float, eps: float, m_mask=None):
    """m-major element pairs: (pair_off (n_elem+1,), pair_l) with l ascending; with m_mask
    only the lists of the selected inner elements m are filled."""
    om = _om(mesh)
    n = om.conn.shape[0]
    off = np.zeros(n + 1, dtype=np.int64)
    mm = None if m_mask is None else np.ascontiguousarray(m_mask, dtype=np.uint8)
    cap = max(1024, (64 * n) if mm is None else 1024 * (int(mm.sum()) + 1))
    while True:
        pl = np.zeros(cap, dtype=np.int32)
        cnt = lib().or_pairs(ctypes.byref(om.c), delta, eps, _ptr(off), _ptr(pl), cap,
                             None if mm is None else _ptr(mm))
        if cnt < 0:
            raise RuntimeError("or_pairs failed")
        if cnt <= cap:
            return off, pl[:cnt].copy()
        cap = int(cnt)


def csr(mesh, pair_off, pair_l):
    om = _om(mesh)
    nv = om.coords.shape[1]
    row_ptr = np.zeros(nv + 1, dtype=np.int64)
    nnz = lib().or_csr(ctypes.byref(om.c), _ptr(pair_off), _ptr(pair_l), _ptr(row_ptr), None, 0)
    if nnz < 0:
        raise RuntimeError("or_csr failed")
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    lib().or_csr(ctypes.byref(om.c), _ptr(pair_off), _ptr(pair_l), _ptr(row_ptr), _ptr(col), nnz)
    return row_ptr, col[:nnz]


@dataclass
class Stats:
    n_point_pairs: int
    n_band_pairs: int
    n_integrations: int


MINDIST_L2 = 1


def assemble(mesh, pair_off, pair_l, row_ptr, col, delta, eps, L_max, L_min=1,
             kernel=KERNEL_CONST, C=None, m_mask=None, mindist_l2=False):
    """Values of A on the CSR pattern (row_ptr, col) and the work counters.  mindist_l2:
    Algorithm 1's refinement test uses the Euclidean approximate minimum distance."""
    om = _om(mesh)
    if C is None:
        C = kernel_constant(om.dim, kernel, delta, eps)
    P = _Params(delta, eps, C, kernel, L_min, L_max, MINDIST_L2 if mindist_l2 else 0)
    vals = np.zeros(max(int(row_ptr[-1]), 1), dtype=np.float64)
    st = _Stats()
    mm = None
    if m_mask is not None:
        mm = np.ascontiguousarray(m_mask, dtype=np.uint8)
    rc = lib().or_assemble(ctypes.byref(om.c), _ptr(pair_off), _ptr(pair_l), ctypes.byref(P),
                           _ptr(row_ptr), _ptr(col), _ptr(vals), None if mm is None else _ptr(mm),
                           ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"or_assemble failed ({rc})")
    return vals[: int(row_ptr[-1])], Stats(st.n_point_pairs, st.n_band_pairs, st.n_integrations)


def ms_u(ms: int, x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().or_ms_u(ms, len(x), _ptr(x))


def ms_f(ms: int, x, kernel, delta, eps, C) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().or_ms_f(ms, len(x), _ptr(x), kernel, delta, eps, C)


def rhs(mesh, row_ptr, col, vals, ms, kernel, delta, eps, C):
    om = _om(mesh)
    F = np.zeros(om.coords.shape[1])
    rc = lib().or_rhs(ctypes.byref(om.c), _ptr(row_ptr), _ptr(col), _ptr(vals), ms, kernel, delta,
                      eps, C, _ptr(F))
    if rc != 0:
        raise RuntimeError("or_rhs failed")
    return F


def solve_dense(mesh, row_ptr, col, vals, F, ms):
    om = _om(mesh)
    u = np.zeros(om.coords.shape[1])
    rc = lib().or_solve_dense(ctypes.byref(om.c), _ptr(row_ptr), _ptr(col), _ptr(vals), _ptr(F), ms,
                              _ptr(u))
    if rc != 0:
        raise RuntimeError("or_solve_dense failed")
    return u


def l2_error(mesh, u_h, ms, omega_only=False) -> float:
    om = _om(mesh)
    u_h = np.ascontiguousarray(u_h, dtype=np.float64)
    return lib().or_l2_error(ctypes.byref(om.c), _ptr(u_h), ms, 1 if omega_only else 0)


def solve_problem(mesh, delta, eps, L_max, ms, kernel=KERNEL_CONST, L_min=1):
    """Pairs, pattern, A, right-hand side with lifting, dense solve and errors, end to end."""
    om = _om(mesh)
    C = kernel_constant(om.dim, kernel, delta, eps)
    off, pl = pairs(om, delta, eps)
    rp, col = csr(om, off, pl)
    vals, st = assemble(om, off, pl, rp, col, delta, eps, L_max, L_min, kernel, C)
    F = rhs(om, rp, col, vals, ms, kernel, delta, eps, C)
    u = solve_dense(om, rp, col, vals, F, ms)
    return dict(C=C, pair_off=off, pair_l=pl, row_ptr=rp, col=col, values=vals, stats=st, F=F,
                u_h=u, err_all=l2_error(om, u, ms, False), err_omega=l2_error(om, u, ms, True))
