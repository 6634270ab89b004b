"""Structured P1 meshes of Omega = [lo, lo + cells*h] with an interaction layer.

Layout (the same on both sides of every parity test):

* vertices are numbered lexicographically, x fastest: v = i + (nx+1)*(j + (ny+1)*k),
  where i, j, k count grid lines from the outer corner of the layer;
* ``coords`` is SoA, shape (dim, n_vert), float64;
* cells are numbered lexicographically, x fastest; each square is cut along its
  "/" diagonal into (v00, v10, v11) and (v00, v11, v01); each cube is cut into the six
  Kuhn tetrahedra (v000, v000+e_a, v000+e_a+e_b, v111) for the permutations (a, b, c)
  of the axes in lexicographic order; ``conn`` has shape (n_elem, dim+1), int32;
* an element belongs to Omega when its cell does; a vertex is a degree of freedom
  ("free") when it lies strictly inside Omega (grid index strictly between the Omega
  faces), so the vertices on the boundary of Omega belong to the volume constraint;
* optional jitter moves every vertex that lies neither on the boundary of Omega nor on
  the outer boundary of the layer by ``jitter * h * (2u - 1)`` per coordinate, with u the
  splitmix64 counter generator of :func:`splitmix64_unit`.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_unit(seed: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from splitmix64 (Steele, Lea, Flood 2014) at position
    ``seed + (counter + 1) * golden``: z ^= z>>30; z *= M1; z ^= z>>27; z *= M2; z ^= z>>31;
    u = (z >> 11) * 2^-53."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Mesh:
    dim: int
    coords: np.ndarray  # (dim, n_vert) float64, SoA
    conn: np.ndarray  # (n_elem, dim+1) int32
    elem_in_omega: np.ndarray  # (n_elem,) uint8
    node_free: np.ndarray  # (n_vert,) uint8
    h: float
    meta: dict = field(default_factory=dict)

    @property
    def n_vert(self) -> int:
        return int(self.coords.shape[1])

    @property
    def n_elem(self) -> int:
        return int(self.conn.shape[0])

    def points(self) -> np.ndarray:
        """(n_vert, dim) copy of the coordinates."""
        return np.ascontiguousarray(self.coords.T)


def structured_mesh(dim: int, cells, h: float, lo, layer: int, jitter: float = 0.0,
                    seed: int = 0) -> Mesh:
    """Mesh of Omega = prod_k [lo_k, lo_k + cells_k*h] plus ``layer`` cells on every side."""
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    cells = [int(c) for c in (cells if np.iterable(cells) else [cells] * dim)]
    lo = [float(v) for v in (lo if np.iterable(lo) else [lo] * dim)]
    if len(cells) != dim or len(lo) != dim or layer < 0 or min(cells) < 1:
        raise ValueError("bad mesh description")
    nc = [c + 2 * layer for c in cells]  # cells per axis including the layer
    nl = [c + 1 for c in nc]  # grid lines per axis
    n_vert = int(np.prod(nl))
    # grid index of every vertex, x fastest
    idx = np.indices(nl[::-1]).reshape(dim, -1)[::-1]  # idx[k] = index along axis k
    coords = np.empty((dim, n_vert), dtype=np.float64)
    for k in range(dim):
        coords[k] = lo[k] + (idx[k] - layer).astype(np.float64) * h
    faces = [(0, layer, layer + cells[k], nc[k]) for k in range(dim)]
    on_face = np.zeros(n_vert, dtype=bool)
    inside = np.ones(n_vert, dtype=bool)
    for k in range(dim):
        on_face |= np.isin(idx[k], faces[k])
        inside &= (idx[k] > layer) & (idx[k] < layer + cells[k])
    if jitter != 0.0:
        vid = np.arange(n_vert, dtype=np.int64)
        move = ~on_face
        for k in range(dim):
            u = splitmix64_unit(seed, vid * 4 + k)
            off = (jitter * h) * (2.0 * u - 1.0)
            coords[k] = np.where(move, coords[k] + off, coords[k])
    # elements
    cidx = np.indices(nc[::-1]).reshape(dim, -1)[::-1]  # cell index per axis, x fastest
    n_cells = cidx.shape[1]
    stride = [int(np.prod(nl[:k])) for k in range(dim)]
    base = sum(cidx[k] * stride[k] for k in range(dim))
    in_omega = np.ones(n_cells, dtype=bool)
    for k in range(dim):
        in_omega &= (cidx[k] >= layer) & (cidx[k] < layer + cells[k])
    if dim == 2:
        v00 = base
        v10 = base + stride[0]
        v01 = base + stride[1]
        v11 = base + stride[0] + stride[1]
        tris = [(v00, v10, v11), (v00, v11, v01)]
        conn = np.stack([np.stack(t, axis=1) for t in tris], axis=1).reshape(-1, 3)
        per_cell = 2
    else:
        tets = []
        for perm in itertools.permutations(range(3)):
            a = base + stride[perm[0]]
            b = a + stride[perm[1]]
            tets.append((base, a, b, base + stride[0] + stride[1] + stride[2]))
        conn = np.stack([np.stack(t, axis=1) for t in tets], axis=1).reshape(-1, 4)
        per_cell = 6
    elem_in_omega = np.repeat(in_omega, per_cell).astype(np.uint8)
    return Mesh(dim=dim, coords=coords, conn=np.ascontiguousarray(conn.astype(np.int32)),
                elem_in_omega=elem_in_omega, node_free=inside.astype(np.uint8), h=float(h),
                meta=dict(cells=cells, lo=lo, layer=layer, jitter=jitter, seed=seed))


def p2_mesh(mesh: Mesh) -> Mesh:
    """The P2 (quadratic Lagrange) mesh on the simplices of a structured mesh.

    Nodes: the vertices (same numbers), then one node per edge at its midpoint (a + b) * 0.5,
    numbered after the vertices in the lexicographic order of the edges' (smaller vertex,
    larger vertex) pairs.  ``conn`` rows are (v0, v1, v2, m01, m12, m02) for triangles and
    (v0, v1, v2, v3, m01, m12, m02, m03, m13, m23) for tetrahedra.  A node is a degree of
    freedom when it lies strictly inside the open Omega of ``mesh.meta`` (vertices on the
    boundary of Omega are never moved by the jitter, so midpoints of boundary edges lie
    exactly on it)."""
    if mesh.conn.shape[1] != mesh.dim + 1:
        raise ValueError("P2 meshes are built from P1 simplex meshes")
    c = mesh.conn.astype(np.int64)
    edges = [(0, 1), (1, 2), (0, 2)] if mesh.dim == 2 else [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
    ne = len(edges)
    pairs = np.stack([c[:, list(e)] for e in edges], axis=1)  # (n_elem, ne, 2)
    lo_hi = np.sort(pairs, axis=2).reshape(-1, 2)
    key = lo_hi[:, 0] * mesh.n_vert + lo_hi[:, 1]
    ukey, inv = np.unique(key, return_inverse=True)
    ea, eb = ukey // mesh.n_vert, ukey % mesh.n_vert
    mid = (mesh.coords[:, ea] + mesh.coords[:, eb]) * 0.5
    coords = np.concatenate([mesh.coords, mid], axis=1)
    edge_node = (mesh.n_vert + inv).reshape(-1, ne)
    conn = np.concatenate([c, edge_node], axis=1).astype(np.int32)
    lo = np.array(mesh.meta["lo"], dtype=np.float64)
    hi = lo + np.array(mesh.meta["cells"], dtype=np.float64) * mesh.h
    free = np.all((coords > lo[:, None]) & (coords < hi[:, None]), axis=0)
    free[: mesh.n_vert] = mesh.node_free.astype(bool)
    meta = dict(mesh.meta, order=2)
    return Mesh(dim=mesh.dim, coords=coords, conn=np.ascontiguousarray(conn), elem_in_omega=mesh.elem_in_omega.copy(),
                node_free=free.astype(np.uint8), h=mesh.h, meta=meta)


def quad_mesh(mesh: Mesh) -> Mesh:
    """The quadrilateral (Q1) mesh of the cells of a structured 2D mesh: the same vertices, one
    element per cell with vertices (v00, v10, v11, v01) counterclockwise (the images of the
    unit square's corners (0,0), (1,0), (1,1), (0,1)); a cell of Omega is an element of
    Omega.  With jitter the cells are general convex quadrilaterals."""
    if mesh.dim != 2 or mesh.conn.shape[1] != 3:
        raise ValueError("quadrilateral meshes are built from structured P1 triangle meshes")
    t = mesh.conn.reshape(-1, 2, 3)  # the two triangles (v00, v10, v11), (v00, v11, v01) per cell
    conn = np.stack([t[:, 0, 0], t[:, 0, 1], t[:, 0, 2], t[:, 1, 2]], axis=1).astype(np.int32)
    eio = mesh.elem_in_omega.reshape(-1, 2)[:, 0].copy()
    return Mesh(dim=2, coords=mesh.coords.copy(), conn=np.ascontiguousarray(conn),
                elem_in_omega=eio, node_free=mesh.node_free.copy(), h=mesh.h,
                meta=dict(mesh.meta, cell="quad"))


def q2_mesh(mesh: Mesh) -> Mesh:
    """The Q2 (biquadratic Lagrange) mesh on the cells of a quadrilateral mesh: the vertices
    (same numbers), one node per edge at its midpoint (a + b) * 0.5 (numbered after the
    vertices in the lexicographic order of the edges' (smaller, larger) vertex pairs), then
    one node per cell at the image of the unit square's centre ((v0 + v1) * 0.5 + (v2 + v3) *
    0.5) * 0.5.  ``conn`` rows are (v0, v1, v2, v3, m01, m12, m23, m30, centre).  A node is a
    degree of freedom when it lies strictly inside the open Omega."""
    if mesh.dim != 2 or mesh.conn.shape[1] != 4:
        raise ValueError("Q2 meshes are built from quadrilateral meshes")
    c = mesh.conn.astype(np.int64)
    edges = np.stack([c[:, [0, 1]], c[:, [1, 2]], c[:, [2, 3]], c[:, [3, 0]]], axis=1)
    lo_hi = np.sort(edges, axis=2).reshape(-1, 2)
    key = lo_hi[:, 0] * mesh.n_vert + lo_hi[:, 1]
    ukey, inv = np.unique(key, return_inverse=True)
    ea, eb = ukey // mesh.n_vert, ukey % mesh.n_vert
    mid = (mesh.coords[:, ea] + mesh.coords[:, eb]) * 0.5
    x = mesh.coords
    cen = ((x[:, c[:, 0]] + x[:, c[:, 1]]) * 0.5 + (x[:, c[:, 2]] + x[:, c[:, 3]]) * 0.5) * 0.5
    coords = np.concatenate([mesh.coords, mid, cen], axis=1)
    edge_node = (mesh.n_vert + inv).reshape(-1, 4)
    cen_node = mesh.n_vert + len(ukey) + np.arange(mesh.n_elem)
    conn = np.concatenate([c, edge_node, cen_node[:, None]], axis=1).astype(np.int32)
    lo = np.array(mesh.meta["lo"], dtype=np.float64)
    hi = lo + np.array(mesh.meta["cells"], dtype=np.float64) * mesh.h
    free = np.all((coords > lo[:, None]) & (coords < hi[:, None]), axis=0)
    free[: mesh.n_vert] = mesh.node_free.astype(bool)
    return Mesh(dim=2, coords=coords, conn=np.ascontiguousarray(conn),
                elem_in_omega=mesh.elem_in_omega.copy(), node_free=free.astype(np.uint8),
                h=mesh.h, meta=dict(mesh.meta, order=2))


def s2_mesh(mesh: Mesh) -> Mesh:
    """The 8-node serendipity mesh of a Q2 mesh: the same nodes and elements without the
    cells' centre nodes (the last n_elem nodes of q2_mesh); rows (v0, v1, v2, v3, m01, m12,
    m23, m30)."""
    if mesh.dim != 2 or mesh.conn.shape[1] != 9:
        raise ValueError("serendipity meshes are built from Q2 meshes")
    n_keep = mesh.n_vert - mesh.n_elem
    if not np.array_equal(mesh.conn[:, 8], np.arange(n_keep, mesh.n_vert)):
        raise ValueError("the centre nodes must be the last n_elem nodes")
    return Mesh(dim=2, coords=np.ascontiguousarray(mesh.coords[:, :n_keep]),
                conn=np.ascontiguousarray(mesh.conn[:, :8]), elem_in_omega=mesh.elem_in_omega.copy(),
                node_free=mesh.node_free[:n_keep].copy(), h=mesh.h, meta=dict(mesh.meta, order=3))


def hex_mesh(mesh: Mesh) -> Mesh:
    """The hexahedral (Q1) mesh of the cells of a structured 3D mesh: the same vertices, one
    element per cell with vertices (v000, v100, v110, v010, v001, v101, v111, v011) (the
    images of the unit cube's corners (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1),
    (1,1,1), (0,1,1)); a cell of Omega is an element of Omega."""
    if mesh.dim != 3 or mesh.conn.shape[1] != 4:
        raise ValueError("hexahedral meshes are built from structured P1 tetrahedral meshes")
    cells, layer = mesh.meta["cells"], mesh.meta["layer"]
    nc = [c + 2 * layer for c in cells]
    nl = [c + 1 for c in nc]
    stride = [1, nl[0], nl[0] * nl[1]]
    cidx = np.indices(nc[::-1]).reshape(3, -1)[::-1]  # x fastest, the order of the tetrahedra
    base = sum(cidx[k] * stride[k] for k in range(3))
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    conn = np.stack([base + sum(c[k] * stride[k] for k in range(3)) for c in corners], 1).astype(np.int32)
    assert np.array_equal(conn[:, 0], mesh.conn[::6, 0]) and np.array_equal(conn[:, 6], mesh.conn[::6, 3])
    eio = mesh.elem_in_omega[::6].copy()
    return Mesh(dim=3, coords=mesh.coords.copy(), conn=np.ascontiguousarray(conn), elem_in_omega=eio,
                node_free=mesh.node_free.copy(), h=mesh.h, meta=dict(mesh.meta, cell="hex"))


# The 27 nodes of the Q2 hexahedron as lattice points (i, j, k) of half steps: the 8 vertices in
# the Q1 order, then the 12 edge midpoints, the 6 face centres and the centre, each group in
# the order of (k, j, i) (z slowest)
HEX27 = [(0, 0, 0), (2, 0, 0), (2, 2, 0), (0, 2, 0), (0, 0, 2), (2, 0, 2), (2, 2, 2), (0, 2, 2),
         (1, 0, 0), (0, 1, 0), (2, 1, 0), (1, 2, 0), (0, 0, 1), (2, 0, 1), (0, 2, 1), (2, 2, 1),
         (1, 0, 2), (0, 1, 2), (2, 1, 2), (1, 2, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1), (2, 1, 1),
         (1, 2, 1), (1, 1, 2), (1, 1, 1)]


def q2_hex_mesh(mesh: Mesh) -> Mesh:
    """The Q2 (triquadratic Lagrange) mesh on the cells of a hexahedral mesh: every node of the
    cells' lattices of half steps (the vertices keep their numbers; the other points are
    numbered after them by their position on the grid of half steps, x fastest), placed at
    the image of its lattice point under the cell's trilinear map.  ``conn`` rows list the 27
    nodes in the order HEX27.  A node is a degree of freedom when it lies strictly inside the
    open Omega."""
    if mesh.dim != 3 or mesh.conn.shape[1] != 8:
        raise ValueError("Q2 hexahedral meshes are built from Q1 hexahedral meshes")
    cells, layer = mesh.meta["cells"], mesh.meta["layer"]
    nc = [c + 2 * layer for c in cells]
    n2 = [2 * c + 1 for c in nc]  # half-step grid points per axis
    x = mesh.coords
    V = x[:, mesh.conn]  # (3, n_elem, 8)
    cidx = np.indices(nc[::-1]).reshape(3, -1)[::-1]  # cell index per axis, x fastest
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    gid = np.zeros((mesh.n_elem, 27), dtype=np.int64)
    pos = np.zeros((3, mesh.n_elem, 27))
    for a, (i, j, k) in enumerate(HEX27):
        g = [2 * cidx[0] + i, 2 * cidx[1] + j, 2 * cidx[2] + k]
        gid[:, a] = g[0] + n2[0] * (g[1] + n2[1] * g[2])
        w = [(1 - i / 2 if c[0] == 0 else i / 2) * (1 - j / 2 if c[1] == 0 else j / 2) *
             (1 - k / 2 if c[2] == 0 else k / 2) for c in corners]
        pos[:, :, a] = sum(w[b] * V[:, :, b] for b in range(8))
    # vertices keep their numbers; the other grid points follow in grid order
    vert_gid = np.unique(gid[:, :8])
    other = np.setdiff1d(np.unique(gid), vert_gid)
    number = {}
    # a vertex's grid id -> its mesh number
    for a in range(8):
        for e_gid, v in zip(gid[:, a], mesh.conn[:, a]):
            number[int(e_gid)] = int(v)
    base = mesh.n_vert
    for t, g in enumerate(other):
        number[int(g)] = base + t
    conn = np.vectorize(number.get)(gid).astype(np.int32)
    n_vert = base + len(other)
    coords = np.zeros((3, n_vert))
    coords[:, conn.ravel()] = pos.reshape(3, -1)
    coords[:, :mesh.n_vert] = x
    lo = np.array(mesh.meta["lo"], dtype=np.float64)
    hi = lo + np.array(mesh.meta["cells"], dtype=np.float64) * mesh.h
    free = np.all((coords > lo[:, None] + 1e-12) & (coords < hi[:, None] - 1e-12), axis=0)
    free[: mesh.n_vert] = mesh.node_free.astype(bool)
    return Mesh(dim=3, coords=coords, conn=np.ascontiguousarray(conn), elem_in_omega=mesh.elem_in_omega.copy(),
                node_free=free.astype(np.uint8), h=mesh.h, meta=dict(mesh.meta, order=2))


def s20_hex_mesh(mesh: Mesh) -> Mesh:
    """The 20-node serendipity mesh of a Q2 hexahedral mesh: the first 20 nodes of each
    element (the vertices and the edge midpoints, in the order HEX27), the face-centre and
    centre nodes dropped and the remaining nodes renumbered in their order (the vertices keep
    their numbers)."""
    if mesh.dim != 3 or mesh.conn.shape[1] != 27:
        raise ValueError("serendipity hexahedral meshes are built from Q2 hexahedral meshes")
    keep = np.unique(mesh.conn[:, :20])
    new = np.full(mesh.n_vert, -1, dtype=np.int64)
    new[keep] = np.arange(len(keep))
    conn = new[mesh.conn[:, :20]].astype(np.int32)
    return Mesh(dim=3, coords=np.ascontiguousarray(mesh.coords[:, keep]), conn=np.ascontiguousarray(conn),
                elem_in_omega=mesh.elem_in_omega.copy(), node_free=mesh.node_free[keep].copy(),
                h=mesh.h, meta=dict(mesh.meta, order=3))
