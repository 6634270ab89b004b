"""ctypes binding of libnl.so (include/nl.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all computation runs in
the library's CUDA kernels.  There is no fallback: if libnl.so is missing or fails to load,
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnl.so")
HEADER = os.path.join(HERE, "..", "include", "nl.h")

NL_OK, NL_EINVAL, NL_ENOMEM, NL_ECUDA, NL_ENOTCONV, NL_ETIMEOUT, NL_EBUSY, NL_EINTERNAL = range(8)
STATUS_NAMES = ["NL_OK", "NL_EINVAL", "NL_ENOMEM", "NL_ECUDA", "NL_ENOTCONV", "NL_ETIMEOUT",
                "NL_EBUSY", "NL_EINTERNAL"]
NL_KERNEL_CONST, NL_KERNEL_TRUNC_GAUSS = 0, 1
NL_PREC_FP64, NL_PREC_MIXED_TF32, NL_PREC_MIXED_BF16, NL_PREC_FP32 = 0, 1, 2, 3


class NLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class KernelParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("eps", ctypes.c_double), ("kappa", ctypes.c_double),
                ("kernel", ctypes.c_int), ("C_override", ctypes.c_double)]


class QuadParams(ctypes.Structure):
    _fields_ = [("L_min", ctypes.c_int), ("L_max", ctypes.c_int), ("rule", ctypes.c_int)]


class AssembleStats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_point_pairs", ctypes.c_int64),
                ("n_items", ctypes.c_int64), ("n_exact_checks", ctypes.c_int64),
                ("ms_assemble", ctypes.c_double), ("n_eval_point_pairs", ctypes.c_int64),
                ("n_closed_items", ctypes.c_int64), ("n_band_point_pairs", ctypes.c_int64),
                ("precision_run", ctypes.c_int32), ("n_quad_launches", ctypes.c_int32),
                ("ms_quad", ctypes.c_double), ("ms_scatter", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("cells", ctypes.c_int32 * 3), ("h", ctypes.c_double),
                ("lo", ctypes.c_double * 3), ("layer", ctypes.c_int32), ("jitter", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("kernel", KernelParams), ("quad", QuadParams),
                ("precision", ctypes.c_int), ("ms", ctypes.c_int), ("solver", ctypes.c_int),
                ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("u_out", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("l2_err_omega", ctypes.c_double), ("n_pairs", ctypes.c_int64),
                ("n_point_pairs", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_vert", ctypes.c_int64), ("t_submit_ms", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("message", ctypes.c_char * 160), ("group", ctypes.c_int32)]


_lib = None


def lib():
    """Loads libnl.so (built by __graft_entry__.build() / paper_2101_08825_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    p, i, i64, d, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "nl_set_allocator": (st, [p, p, p]),
        "nl_last_error": (ctypes.c_char_p, []),
        "nl_version": (ctypes.c_char_p, []),
        "nl_launch_count": (i64, []),
        "nl_mesh_create": (st, [i, i64, p, i64, p, p, p, p, pp]),
        "nl_mesh_create_p2": (st, [i, i64, p, i64, p, p, p, p, pp]),
        "nl_mesh_create_quad": (st, [i, i64, p, i64, p, p, p, p, pp]),
        "nl_mesh_create_hex": (st, [i, i64, p, i64, p, p, p, p, pp]),
        "nl_mesh_create_box": (st, [i, p, d, p, ctypes.c_int32, d, ctypes.c_uint64, p, pp]),
        "nl_mesh_info": (st, [p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int64)]),
        "nl_mesh_order": (st, [p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "nl_mesh_export": (st, [p, p, p, p, p]),
        "nl_mesh_destroy": (None, [p]),
        "nl_pairs_build": (st, [p, d, d, pp]),
        "nl_pairs_info": (st, [p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "nl_pairs_export": (st, [p, p, p, p, p]),
        "nl_pairs_destroy": (None, [p]),
        "nl_assemble": (st, [p, p, ctypes.POINTER(KernelParams), ctypes.POINTER(QuadParams), i, pp,
                             ctypes.POINTER(AssembleStats)]),
        "nl_assemble_noalloc": (st, [p, p, ctypes.POINTER(KernelParams), ctypes.POINTER(QuadParams),
                                     i, p, ctypes.POINTER(AssembleStats)]),
        "nl_matrix_export": (st, [p, p]),
        "nl_matrix_apply": (st, [p, p, p]),
        "nl_matrix_device_values": (st, [p, pp]),
        "nl_matrix_destroy": (None, [p]),
        "nl_rhs": (st, [p, p, p, d, p, pp]),
        "nl_vector_export": (st, [p, p]),
        "nl_vector_destroy": (None, [p]),
        "nl_solve": (st, [p, p, p, i, d, i, i, p, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)]),
        "nl_serve_create": (st, [ctypes.c_size_t, i, pp]),
        "nl_serve_submit": (st, [p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "nl_serve_poll": (st, [p, ctypes.c_uint64, ctypes.POINTER(Result)]),
        "nl_serve_wait": (st, [p, ctypes.c_uint64, d, ctypes.POINTER(Result)]),
        "nl_serve_stats": (st, [p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]),
        "nl_serve_destroy": (None, [p]),
        "nl_plan_create": (st, [i, p, p, p, p, i, i, p, pp]),
        "nl_plan_execute": (st, [p]),
        "nl_plan_sync": (st, [p, p]),
        "nl_plan_values": (st, [p, i, pp, ctypes.POINTER(ctypes.c_int64)]),
        "nl_plan_export": (st, [p, i, p]),
        "nl_plan_matrix": (st, [p, i, pp]),
        "nl_plan_shape": (st, [p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_int)]),
        "nl_plan_destroy": (None, [p]),
        "nl_quad_rule": (i, [i, p, p]),
        "nl_kernel_constant": (d, [i, i, d, d]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_functions(header: str = HEADER):
    """Names of the functions declared in include/nl.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(nl_[a-z0-9_]+)\s*\(", text)
    typedef_fns = set(re.findall(r"\(\*\s*(nl_[a-z0-9_]+)\)", text))
    return sorted(set(n for n in names if n not in typedef_fns))


def _check(status: int, what: str = ""):
    if status != NL_OK:
        raise NLError(status, (what + ": " if what else "") + lib().nl_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def current_stream():
    """The torch current CUDA stream handle (0 = legacy default stream when unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


# ---- handles -----------------------------------------------------------------------------

class _Handle:
    _destroy = ""

    def __init__(self, h):
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            getattr(lib(), self._destroy)(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mesh(_Handle):
    _destroy = "nl_mesh_destroy"

    def info(self):
        dim, nv, ne = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nl_mesh_info(self.h, ctypes.byref(dim), ctypes.byref(nv), ctypes.byref(ne)))
        return dim.value, nv.value, ne.value

    def order(self):
        """(polynomial order, nodes per element)."""
        o, nb = ctypes.c_int(), ctypes.c_int()
        _check(lib().nl_mesh_order(self.h, ctypes.byref(o), ctypes.byref(nb)))
        return o.value, nb.value

    def export(self):
        dim, nv, ne = self.info()
        nb = self.order()[1]
        coords = np.zeros(dim * nv)
        conn = np.zeros(ne * nb, dtype=np.int32)
        eio = np.zeros(ne, dtype=np.uint8)
        nf = np.zeros(nv, dtype=np.uint8)
        _check(lib().nl_mesh_export(self.h, _ptr(coords), _ptr(conn), _ptr(eio), _ptr(nf)))
        return coords.reshape(dim, nv), conn.reshape(ne, nb), eio, nf


class Pairs(_Handle):
    _destroy = "nl_pairs_destroy"

    def info(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nl_pairs_info(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def export(self, n_elem: int, n_vert: int):
        n_pairs, nnz = self.info()
        off = np.zeros(n_elem + 1, dtype=np.int64)
        pl = np.zeros(max(n_pairs, 1), dtype=np.int32)
        rp = np.zeros(n_vert + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        _check(lib().nl_pairs_export(self.h, _ptr(off), _ptr(pl), _ptr(rp), _ptr(col)))
        return off, pl[:n_pairs], rp, col[:nnz]


class Matrix(_Handle):
    _destroy = "nl_matrix_destroy"

    def __init__(self, h, nnz):
        super().__init__(h)
        self.nnz = nnz

    def export(self):
        v = np.zeros(max(self.nnz, 1))
        _check(lib().nl_matrix_export(self.h, _ptr(v)))
        return v[: self.nnz]

    def device_values(self) -> int:
        p = ctypes.c_void_p()
        _check(lib().nl_matrix_device_values(self.h, ctypes.byref(p)))
        return p.value

    def apply(self, x_ptr: int, y_ptr: int):
        """nl_matrix_apply: y = A x on the device (x, y: device pointers of n_vert doubles)."""
        _check(lib().nl_matrix_apply(self.h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr)),
               "nl_matrix_apply")


class Vector(_Handle):
    _destroy = "nl_vector_destroy"

    def __init__(self, h, n):
        super().__init__(h)
        self.n = n

    def export(self):
        v = np.zeros(self.n)
        _check(lib().nl_vector_export(self.h, _ptr(v)))
        return v


# ---- entry points ---------------------------------------------------------------------------

def nl_mesh_create(dim, coords, conn, elem_in_omega, node_free, stream=None) -> Mesh:
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(dim, -1)
    conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, dim + 1)
    eio = np.ascontiguousarray(elem_in_omega, dtype=np.uint8)
    nf = np.ascontiguousarray(node_free, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib().nl_mesh_create(dim, coords.shape[1], _ptr(coords), conn.shape[0], _ptr(conn),
                                _ptr(eio), _ptr(nf), stream if stream is not None else current_stream(),
                                ctypes.byref(h)), "nl_mesh_create")
    return Mesh(h)


def nl_mesh_create_p2(dim, coords, conn, elem_in_omega, node_free, stream=None) -> Mesh:
    """Mesh of P2 simplices: conn rows (v0, v1, v2, m01, m12, m02) for triangles, (v0, v1, v2,
    v3, m01, m12, m02, m03, m13, m23) for tetrahedra."""
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(dim, -1)
    conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, 6 if dim == 2 else 10)
    eio = np.ascontiguousarray(elem_in_omega, dtype=np.uint8)
    nf = np.ascontiguousarray(node_free, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib().nl_mesh_create_p2(dim, coords.shape[1], _ptr(coords), conn.shape[0], _ptr(conn),
                                   _ptr(eio), _ptr(nf), stream if stream is not None else current_stream(),
                                   ctypes.byref(h)), "nl_mesh_create_p2")
    return Mesh(h)


def nl_mesh_create_quad(order, coords, conn, elem_in_omega, node_free, stream=None) -> Mesh:
    """Mesh of quadrilaterals: conn rows of 4 (Q1, order 1), 9 (Q2, order 2) or 8
    (serendipity, order 3) nodes."""
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(2, -1)
    conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, {1: 4, 2: 9, 3: 8}[int(order)])
    eio = np.ascontiguousarray(elem_in_omega, dtype=np.uint8)
    nf = np.ascontiguousarray(node_free, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib().nl_mesh_create_quad(int(order), coords.shape[1], _ptr(coords), conn.shape[0], _ptr(conn),
                                     _ptr(eio), _ptr(nf), stream if stream is not None else current_stream(),
                                     ctypes.byref(h)), "nl_mesh_create_quad")
    return Mesh(h)


def nl_mesh_create_hex(order, coords, conn, elem_in_omega, node_free, stream=None) -> Mesh:
    """Mesh of hexahedra: conn rows of 8 vertices (Q1, order 1), 27 nodes (Q2, order 2) or
    20 nodes (serendipity, order 3)."""
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(3, -1)
    conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, {1: 8, 3: 20}.get(int(order), 27))
    eio = np.ascontiguousarray(elem_in_omega, dtype=np.uint8)
    nf = np.ascontiguousarray(node_free, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(lib().nl_mesh_create_hex(int(order), coords.shape[1], _ptr(coords), conn.shape[0], _ptr(conn), _ptr(eio),
                                    _ptr(nf), stream if stream is not None else current_stream(),
                                    ctypes.byref(h)), "nl_mesh_create_hex")
    return Mesh(h)


def mesh_from(mesh, stream=None) -> Mesh:
    """Uploads an nl_inputs.Mesh: P1 simplices, P2 simplices (six or ten nodes per element),
    quadrilaterals (2D, four, eight or nine nodes per element) or hexahedra (3D, eight or
    twenty-seven or twenty)."""
    if mesh.dim == 3 and mesh.conn.shape[1] in (8, 20, 27):
        return nl_mesh_create_hex({8: 1, 27: 2, 20: 3}[mesh.conn.shape[1]], mesh.coords, mesh.conn, mesh.elem_in_omega, mesh.node_free, stream)
    if mesh.dim == 2 and mesh.conn.shape[1] in (4, 8, 9):
        return nl_mesh_create_quad({4: 1, 9: 2, 8: 3}[mesh.conn.shape[1]], mesh.coords, mesh.conn,
                                   mesh.elem_in_omega, mesh.node_free, stream)
    if mesh.conn.shape[1] == (6 if mesh.dim == 2 else 10):
        return nl_mesh_create_p2(mesh.dim, mesh.coords, mesh.conn, mesh.elem_in_omega, mesh.node_free, stream)
    return nl_mesh_create(mesh.dim, mesh.coords, mesh.conn, mesh.elem_in_omega, mesh.node_free, stream)


def nl_mesh_create_box(dim, cells, h, lo, layer, jitter=0.0, seed=0, stream=None) -> Mesh:
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib().nl_mesh_create_box(dim, _ptr(cells), float(h), _ptr(lo), int(layer), float(jitter),
                                    int(seed), stream if stream is not None else current_stream(),
                                    ctypes.byref(out)), "nl_mesh_create_box")
    return Mesh(out)


def nl_pairs_build(mesh: Mesh, delta: float, eps: float) -> Pairs:
    out = ctypes.c_void_p()
    _check(lib().nl_pairs_build(mesh.h, float(delta), float(eps), ctypes.byref(out)), "nl_pairs_build")
    return Pairs(out)


NL_QUAD_COUNT_BAND = 0x100
NL_QUAD_MINDIST_L2 = 0x200


def quad_rule_flags(count_band=False, mindist_l2=False) -> int:
    return (NL_QUAD_COUNT_BAND if count_band else 0) | (NL_QUAD_MINDIST_L2 if mindist_l2 else 0)


def nl_assemble(mesh: Mesh, pairs: Pairs, delta, eps, L_max, L_min=1, kernel=NL_KERNEL_CONST,
                precision=NL_PREC_FP64, C_override=0.0, kappa=0.0, into: Matrix | None = None,
                count_band=False, mindist_l2=False):
    kp = KernelParams(float(delta), float(eps), float(kappa), int(kernel), float(C_override))
    qp = QuadParams(int(L_min), int(L_max), quad_rule_flags(count_band, mindist_l2))
    st = AssembleStats()
    h = ctypes.c_void_p(into.h.value if into is not None else None)
    _check(lib().nl_assemble(mesh.h, pairs.h, ctypes.byref(kp), ctypes.byref(qp), int(precision),
                             ctypes.byref(h), ctypes.byref(st)), "nl_assemble")
    if into is not None:
        return into, st
    return Matrix(h, pairs.info()[1]), st


def nl_assemble_noalloc(mesh: Mesh, pairs: Pairs, delta, eps, L_max, values_ptr: int, L_min=1,
                        kernel=NL_KERNEL_CONST, precision=NL_PREC_FP64, C_override=0.0,
                        kappa=0.0, mindist_l2=False):
    """Assembles into the caller's device array (nnz doubles at values_ptr) without any
    device allocation by the library."""
    kp = KernelParams(float(delta), float(eps), float(kappa), int(kernel), float(C_override))
    qp = QuadParams(int(L_min), int(L_max), quad_rule_flags(False, mindist_l2))
    st = AssembleStats()
    _check(lib().nl_assemble_noalloc(mesh.h, pairs.h, ctypes.byref(kp), ctypes.byref(qp),
                                     int(precision), ctypes.c_void_p(int(values_ptr)),
                                     ctypes.byref(st)), "nl_assemble_noalloc")
    return st


def nl_rhs(mesh: Mesh, A: Matrix, g_nodes, f_const=0.0, f_nodes=None) -> Vector:
    g = np.ascontiguousarray(g_nodes, dtype=np.float64)
    fn = None if f_nodes is None else np.ascontiguousarray(f_nodes, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib().nl_rhs(mesh.h, A.h, None if fn is None else _ptr(fn), float(f_const), _ptr(g),
                        ctypes.byref(out)), "nl_rhs")
    return Vector(out, len(g))


def nl_solve(A: Matrix, rhs: Vector, g_nodes, solver=1, rtol=1e-12, max_iter=10000,
             precision=NL_PREC_FP64, check=True):
    g = np.ascontiguousarray(g_nodes, dtype=np.float64)
    u = np.zeros(len(g))
    it = ctypes.c_int()
    rr = ctypes.c_double()
    s = lib().nl_solve(A.h, rhs.h, _ptr(g), int(solver), float(rtol), int(max_iter), int(precision),
                       _ptr(u), ctypes.byref(it), ctypes.byref(rr))
    if check:
        _check(s, "nl_solve")
    return u, it.value, rr.value, s


def nl_quad_rule(dim: int):
    b = np.zeros(64)
    w = np.zeros(16)
    n = lib().nl_quad_rule(dim, _ptr(b), _ptr(w))
    if n <= 0:
        raise NLError(NL_EINTERNAL, "nl_quad_rule failed")
    return b[: n * (dim + 1)].reshape(n, dim + 1).copy(), w[:n].copy()


def nl_kernel_constant(dim, kernel, delta, eps) -> float:
    return lib().nl_kernel_constant(dim, kernel, delta, eps)


@dataclass
class Problem:
    """Mesh, pairs and matrix of one assembled problem, kept on the device."""
    mesh: Mesh
    pairs: Pairs
    A: Matrix
    stats: AssembleStats


def assemble_problem(mesh_in, delta, eps, L_max, L_min=1, kernel=NL_KERNEL_CONST,
                     precision=NL_PREC_FP64) -> Problem:
    m = mesh_from(mesh_in)
    p = nl_pairs_build(m, delta, eps)
    A, st = nl_assemble(m, p, delta, eps, L_max, L_min, kernel, precision)
    return Problem(m, p, A, st)


# ---- serving ------------------------------------------------------------------------------

def make_request(dim, cells, h, lo, layer, delta, eps, L_max, kernel=NL_KERNEL_CONST,
                 precision=NL_PREC_FP32, ms=1, solver=1, rtol=1e-10, max_iter=20000, jitter=0.0,
                 seed=0, L_min=1, u_out=None, mindist_l2=False) -> Request:
    r = Request()
    r.dim = dim
    for k in range(3):
        r.cells[k] = int(cells[k]) if k < dim else 1
        r.lo[k] = float(lo[k]) if k < dim else 0.0
    r.h, r.layer, r.jitter, r.seed = float(h), int(layer), float(jitter), int(seed)
    r.kernel = KernelParams(float(delta), float(eps), 0.0, int(kernel), 0.0)
    r.quad = QuadParams(int(L_min), int(L_max), quad_rule_flags(False, mindist_l2))
    r.precision, r.ms, r.solver, r.rtol, r.max_iter = int(precision), int(ms), int(solver), float(rtol), int(max_iter)
    r.u_out = None if u_out is None else u_out.ctypes.data
    return r


class Server(_Handle):
    """nl_serve_*: a continuous-batching server on the current device."""
    _destroy = "nl_serve_destroy"

    def __init__(self, device_mem_budget: int, max_slots: int):
        h = ctypes.c_void_p()
        _check(lib().nl_serve_create(int(device_mem_budget), int(max_slots), ctypes.byref(h)),
               "nl_serve_create")
        super().__init__(h)
        self._keep = {}

    def submit(self, req: Request, u_out=None) -> int:
        t = ctypes.c_uint64()
        _check(lib().nl_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t)), "nl_serve_submit")
        self._keep[t.value] = u_out  # keeps the output array alive until the result is taken
        return t.value

    def poll(self, ticket: int):
        r = Result()
        s = lib().nl_serve_poll(self.h, ticket, ctypes.byref(r))
        if s == NL_EBUSY:
            return None
        _check(s, "nl_serve_poll")
        self._keep.pop(ticket, None)
        return r

    def wait(self, ticket: int, timeout_ms: float = 600000.0) -> Result:
        r = Result()
        _check(lib().nl_serve_wait(self.h, ticket, float(timeout_ms), ctypes.byref(r)), "nl_serve_wait")
        self._keep.pop(ticket, None)
        return r

    def stats(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().nl_serve_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


# ---- batched assembly -----------------------------------------------------------------------

NL_PLAN_AUTOTUNE = 1
NL_PLAN_GRAPH = 2


class Plan(_Handle):
    """nl_plan_*: n problems of one dimension and precision assembled by one launch.

    problems: sequence of (mesh, pairs, delta, eps, L_max, L_min, kernel) tuples (L_min and
    kernel may be left out: 1 and NL_KERNEL_CONST)."""
    _destroy = "nl_plan_destroy"

    def __init__(self, problems, precision=NL_PREC_FP64, flags=0, stream=None):
        n = len(problems)
        meshes = (ctypes.c_void_p * n)()
        pairs = (ctypes.c_void_p * n)()
        kps = (KernelParams * n)()
        qps = (QuadParams * n)()
        self._nnz = []
        for k, pr in enumerate(problems):
            mesh, pr_pairs, delta, eps, L_max = pr[:5]
            L_min = pr[5] if len(pr) > 5 else 1
            kernel = pr[6] if len(pr) > 6 else NL_KERNEL_CONST
            meshes[k] = mesh.h.value
            pairs[k] = pr_pairs.h.value
            kps[k] = KernelParams(float(delta), float(eps), 0.0, int(kernel), 0.0)
            qps[k] = QuadParams(int(L_min), int(L_max), 0)
            self._nnz.append(pr_pairs.info()[1])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else ctypes.c_void_p(0)
        _check(lib().nl_plan_create(n, meshes, pairs, kps, qps, int(precision), int(flags), st,
                                    ctypes.byref(h)), "nl_plan_create")
        super().__init__(h)
        self.n = n

    def execute(self):
        _check(lib().nl_plan_execute(self.h), "nl_plan_execute")

    def sync(self):
        stats = (AssembleStats * self.n)()
        _check(lib().nl_plan_sync(self.h, stats), "nl_plan_sync")
        return list(stats)

    def export(self, k: int) -> np.ndarray:
        out = np.zeros(self._nnz[k], dtype=np.float64)
        _check(lib().nl_plan_export(self.h, int(k), _ptr(out)), "nl_plan_export")
        return out

    def device_values(self, k: int) -> int:
        v = ctypes.c_void_p()
        _check(lib().nl_plan_values(self.h, int(k), ctypes.byref(v), None), "nl_plan_values")
        return v.value or 0

    def matrix(self, k: int) -> Matrix:
        h = ctypes.c_void_p()
        _check(lib().nl_plan_matrix(self.h, int(k), ctypes.byref(h)), "nl_plan_matrix")
        return Matrix(h, self._nnz[k])

    def shape(self):
        w, c, ch, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        _check(lib().nl_plan_shape(self.h, ctypes.byref(w), ctypes.byref(c), ctypes.byref(ch),
                                   ctypes.byref(ms), ctypes.byref(g)), "nl_plan_shape")
        return {"warps": w.value, "ctas_per_sm": c.value, "chunk": ch.value,
                "tuned_ms": ms.value, "graph": bool(g.value)}
