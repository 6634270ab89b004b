"""Workload descriptions: the shapes and parameters of the paper's tests and of the
benchmark configurations, as plain data.

Every mesh is a structured P1 mesh of a box Omega with an interaction layer of
ceil((delta + eps)/h) whole cells, so the mollified kernel (support radius delta + eps)
never reaches past the meshed region from a point of Omega.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

from .mesh import Mesh, hex_mesh, p2_mesh, q2_hex_mesh, q2_mesh, quad_mesh, s20_hex_mesh, structured_mesh

KERNEL_CONST = 0
KERNEL_GAUSS = 1

MS_LINEAR = 0
MS_QUADRATIC = 1
MS_CUBIC = 2
MS_QUARTIC = 3


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    cells: tuple
    h: float
    lo: tuple
    delta: float
    eps: float
    L_max: int
    L_min: int = 1
    kernel: int = KERNEL_CONST
    ms: int = MS_QUADRATIC
    jitter: float = 0.0
    seed: int = 0
    layer_cells: int = 0  # 0: ceil((delta + eps)/h); otherwise the given number of cells
    order: int = 1        # 1: P1 elements; 2: P2 simplices on the same triangulation
    # "quad": one quadrilateral per grid cell (2D; Q1, or Q2 with order 2); "hex": one
    # hexahedron per grid cell (3D; Q1, Q2 with order 2, the 20-node serendipity element with
    # order 3)
    cell: str = "simplex"

    @property
    def layer(self) -> int:
        if self.layer_cells:
            return int(self.layer_cells)
        return int(math.ceil((self.delta + self.eps) / self.h - 1e-9))

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _unit_box(name, dim, n, delta, eps, L_max, **kw) -> Workload:
    return Workload(name=name, dim=dim, cells=(n,) * dim, h=1.0 / n, lo=(0.0,) * dim,
                    delta=delta, eps=eps, L_max=L_max, **kw)


def table2_tri(ml: int) -> Workload:
    """Sec. 6, Table 2: Omega = [-0.6, 0.6] x [-0.4, 0.4], h = 0.1 (1/2)^(ml-2),
    delta = 0.2, eps = 0.0125 (2/3)^(ml-2), L_min = 1, L_max = 3, u = x^3 + y^3.  The layer
    Gamma is meshed delta wide (Sec. 2, eq. interaction-domain), 2^(ml-1) cells."""
    s = 2 ** (ml - 2)
    return Workload(name=f"table2_tri_ml{ml}", dim=2, cells=(12 * s, 8 * s), h=0.1 / s,
                    lo=(-0.6, -0.4), delta=0.2, eps=0.0125 * (2.0 / 3.0) ** (ml - 2), L_max=3,
                    ms=MS_CUBIC, layer_cells=2 * s)


def table7_hex(ml: int) -> Workload:
    """Sec. 6, Table 7 (3D h-convergence, u = x^3 + y^3 + z^3): Omega = [-0.6, 0.6] x
    [-0.4, 0.4] x [-0.4, 0.4], h = 0.2 (1/2)^(ml-1), delta = 0.2, eps = 0.01875 (2/3)^(ml-1),
    L_min = 1, L_max = 2, one hexahedron per grid cell (Q1); the layer Gamma is meshed delta
    wide (2^(ml-1) cells), as for the 2D tables."""
    s = 2 ** (ml - 1)
    return Workload(name=f"table7_hex_ml{ml}", dim=3, cells=(6 * s, 4 * s, 4 * s), h=0.2 / s,
                    lo=(-0.6, -0.4, -0.4), delta=0.2, eps=0.01875 * (2.0 / 3.0) ** (ml - 1),
                    L_max=2, ms=MS_CUBIC, layer_cells=s, cell="hex")


def table6_hex(L_max: int) -> Workload:
    """Sec. 6, Table 6 (3D consistency, Q2 hexahedra): Omega = [-0.6, 0.6] x [-0.4, 0.4] x
    [-0.4, 0.4], h = 0.1, delta = 0.2, L_min = 1, u = x^2 + y^2 + z^2 (f = -6); the layer
    Gamma is meshed delta wide (2 cells).  eps = 0.0125 (3/4)^(L_max-3), the schedule of the
    2D consistency test (Table 1): it reproduces the printed errors at L_max = 3, 4, where the
    3D caption's exponent L_max - 2 gives 2.5 times the printed error at L_max = 3."""
    return Workload(name=f"table6_hex_L{L_max}", dim=3, cells=(12, 8, 8), h=0.1,
                    lo=(-0.6, -0.4, -0.4), delta=0.2, eps=0.0125 * 0.75 ** (L_max - 3),
                    L_max=L_max, ms=MS_QUADRATIC, layer_cells=2, cell="hex", order=2)


def table3_tri(ml: int) -> Workload:
    """Sec. 6, Table 3: the setting of Table 2 with u = x^4 + y^4."""
    return table2_tri(ml).with_(name=f"table3_tri_ml{ml}", ms=MS_QUARTIC)


_H2 = 1.0 / 256.0
WORKLOADS = {
    # 2D, h = 1/16, delta = 0.1, eps = delta/10, 3 levels, u = x^2 + y^2
    "c1_2d": _unit_box("c1_2d", 2, 16, 0.1, 0.01, 3),
    # 2D at scale, h = 1/256, delta = 4h, eps in {delta/5, delta/20}, 4 levels, jitter 0.1h
    "c2_2d": _unit_box("c2_2d", 2, 256, 4 * _H2, 4 * _H2 / 5, 4, jitter=0.1),
    "c2_2d_eps20": _unit_box("c2_2d_eps20", 2, 256, 4 * _H2, 4 * _H2 / 20, 4, jitter=0.1),
    "c2_2d_h128": _unit_box("c2_2d_h128", 2, 128, 4 / 128, 4 / 128 / 5, 4, jitter=0.1),
    "c2_2d_gauss": _unit_box("c2_2d_gauss", 2, 256, 4 * _H2, 4 * _H2 / 5, 4, jitter=0.1,
                             kernel=KERNEL_GAUSS),
    "c2_2d_gauss_eps20": _unit_box("c2_2d_gauss_eps20", 2, 256, 4 * _H2, 4 * _H2 / 20, 4,
                                   jitter=0.1, kernel=KERNEL_GAUSS),
    # 3D, h = 1/16, delta = 0.125, eps = delta/10, 2 levels, u = x^2 + y^2 + z^2
    "c3_3d": _unit_box("c3_3d", 3, 16, 0.125, 0.0125, 2),
    # 3D, h = 1/10, delta = 0.125, eps = delta/10, 2 levels: a small case of the 3D kernel for
    # profiler captures (12 M pairs, an 0.8 GB block buffer: larger than L2, a few GB at most)
    "c3_3d_h10": _unit_box("c3_3d_h10", 3, 10, 0.125, 0.0125, 2),
    # 3D, h = 1/32, delta = 3h, eps = delta/10, 2 levels
    "c4_3d": _unit_box("c4_3d", 3, 32, 3.0 / 32, 0.3 / 32, 2),
    # the c2_2d triangulation with P2 elements (Sec. 6, the quadratic columns of Tables 1-3)
    "c2_2d_p2": _unit_box("c2_2d_p2", 2, 256, 4 * _H2, 4 * _H2 / 5, 4, jitter=0.1, order=2),
    # the c2_2d_h128 triangulation with P2 elements: a small case for profiler captures
    "c2_2d_h128_p2": _unit_box("c2_2d_h128_p2", 2, 128, 4 / 128, 4 / 128 / 5, 4, jitter=0.1,
                               order=2),
    # the c2_2d grid with one Q1 quadrilateral per cell (Sec. 6, QUAD meshes)
    "c2_2d_q1": _unit_box("c2_2d_q1", 2, 256, 4 * _H2, 4 * _H2 / 5, 4, jitter=0.1, cell="quad"),
    "c2_2d_h128_q1": _unit_box("c2_2d_h128_q1", 2, 128, 4 / 128, 4 / 128 / 5, 4, jitter=0.1,
                               cell="quad"),
    # the c3_3d tetrahedra with P2 elements
    "c3_3d_p2": _unit_box("c3_3d_p2", 3, 16, 0.125, 0.0125, 2, order=2),
    "c3_3d_h10_p2": _unit_box("c3_3d_h10_p2", 3, 10, 0.125, 0.0125, 2, order=2),
    # the c3_3d grid with one Q1 hexahedron per cell (Sec. 6, the HEX meshes of the 3D tests)
    "c3_3d_hex": _unit_box("c3_3d_hex", 3, 16, 0.125, 0.0125, 2, cell="hex"),
    "c3_3d_h10_hex": _unit_box("c3_3d_h10_hex", 3, 10, 0.125, 0.0125, 2, cell="hex"),
    # the same grids with Q2 (27-node) hexahedra
    "c3_3d_hex_q2": _unit_box("c3_3d_hex_q2", 3, 16, 0.125, 0.0125, 2, cell="hex", order=2),
    "c3_3d_h10_hex_q2": _unit_box("c3_3d_h10_hex_q2", 3, 10, 0.125, 0.0125, 2, cell="hex",
                                  order=2),
    # the same grid with Q2 (biquadratic) quadrilaterals
    "c2_2d_q2": _unit_box("c2_2d_q2", 2, 256, 4 * _H2, 4 * _H2 / 5, 4, jitter=0.1, cell="quad",
                          order=2),
    "c2_2d_h128_q2": _unit_box("c2_2d_h128_q2", 2, 128, 4 / 128, 4 / 128 / 5, 4, jitter=0.1,
                               cell="quad", order=2),
}


def workload_mesh(w: Workload) -> Mesh:
    m = structured_mesh(w.dim, w.cells, w.h, w.lo, w.layer, jitter=w.jitter, seed=w.seed)
    if w.cell == "quad":
        q = quad_mesh(m)
        return q2_mesh(q) if w.order == 2 else q
    if w.cell == "hex":
        if w.order == 1:
            return hex_mesh(m)
        q2 = q2_hex_mesh(hex_mesh(m))
        return s20_hex_mesh(q2) if w.order == 3 else q2
    return p2_mesh(m) if w.order == 2 else m
