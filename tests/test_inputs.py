"""The seeded input generators (CPU): the structured meshes of the four workloads have the
sizes their construction fixes, and the jitter leaves the topology, the inner/outer split and
the element pairs of the small workload unchanged.

Construction (the structured meshes of Sec. 6): (0,1)^n split into cubes of side h, each cut
into n! simplices (2 triangles, 6 Kuhn tetrahedra), surrounded by an outer layer of
ceil((delta + eps)/h) cells, so that every point within delta + eps of Omega is meshed (the
layer width is this implementation's reading of the interaction domain's extent); unknowns
are the nodes strictly inside Omega."""
import math

import numpy as np
import pytest

import oracle as O
from nl_inputs import WORKLOADS, workload_mesh


@pytest.mark.parametrize("name", ["c1_2d", "c2_2d", "c3_3d", "c4_3d"])
def test_workload_mesh_sizes(name):
    w = WORKLOADS[name]
    m = workload_mesh(w)
    n, d = w.cells[0], w.dim
    assert all(c == n for c in w.cells)
    assert w.layer * w.h >= w.delta + w.eps - 1e-12 > (w.layer - 1) * w.h
    N = n + 2 * w.layer
    assert m.n_vert == (N + 1) ** d
    assert m.n_elem == math.factorial(d) * N ** d
    assert int(m.elem_in_omega.sum()) == math.factorial(d) * n ** d
    assert int(m.node_free.sum()) == (n - 1) ** d
    # every simplex has positive volume and the volumes fill the meshed box
    x = m.coords
    V = np.stack([x[:, m.conn[:, a]].T for a in range(d + 1)], axis=1)  # (elem, d+1, d)
    vol = np.abs(np.linalg.det(V[:, 1:, :] - V[:, :1, :])) / math.factorial(d)
    assert vol.min() > 0.2 * w.h ** d / math.factorial(d)
    assert abs(vol.sum() - (N * w.h) ** d) < 1e-9 * (N * w.h) ** d


def test_jitter_keeps_the_small_workload_pairs():
    # the small 2D workload without and with jitter: same element pairs and CSR pattern
    w = WORKLOADS["c1_2d"]
    counts = []
    for jit in (0.0, w.jitter or 0.1):
        m = workload_mesh(w.with_(jitter=jit))
        off, pl = O.pairs(m, w.delta, w.eps)
        rp, col = O.csr(m, off, pl)
        counts.append((len(pl), len(col)))
    assert counts[0] == counts[1] and counts[0][0] > 0


def test_serving_stream_mix_and_reproducibility():
    # the seeded request stream: reproducible, both dimensions and kernels, Omega element
    # counts within 1e3..2e5 (2D) / 1e3..1e5 (3D) up to the rounding to whole cells, delta in
    # [2h, 6h], eps = delta/10, increasing arrival times
    from nl_inputs.requests import serving_stream
    a, b = serving_stream(512, seed=0), serving_stream(512, seed=0)
    assert a == b and serving_stream(512, seed=1) != a
    dims = {r.dim for r in a}
    kernels = {r.kernel for r in a}
    assert dims == {2, 3} and kernels == {0, 1}
    for r in a:
        per_cell = 2 if r.dim == 2 else 6
        omega = per_cell * r.n ** r.dim
        hi = 2e5 if r.dim == 2 else 1e5
        assert 0.5e3 <= omega <= 1.6 * hi, r
        h = 1.0 / r.n
        assert 2 * h - 1e-12 <= r.delta <= 6 * h + 1e-12 and abs(r.eps - r.delta / 10) < 1e-15
        assert r.layer * h >= r.delta + r.eps - 1e-12 > (r.layer - 1) * h
        assert r.n_elem == per_cell * (r.n + 2 * r.layer) ** r.dim
    t = np.array([r.arrival_s for r in a])
    assert np.all(np.diff(t) > 0)
    # log-uniform sizes: the median Omega element count of each dimension lies near the
    # geometric mean of its range
    for dim, hi in ((2, 2e5), (3, 1e5)):
        sizes = [(2 if dim == 2 else 6) * r.n ** dim for r in a if r.dim == dim]
        gm = math.sqrt(1e3 * hi)
        assert gm / 3 < float(np.median(sizes)) < gm * 3


def test_splitmix64_matches_its_published_sequence():
    # splitmix64 (Steele, Lea, Flood 2014) from state 0 gives 0xE220A8397B1DCDAF,
    # 0x6E789E6AA1B965F4, 0x06C45D188009454F; the unit doubles are their top 53 bits / 2^53
    from nl_inputs.mesh import splitmix64_unit
    u = splitmix64_unit(0, np.arange(3))
    for got, z in zip(u, (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F)):
        assert got == (z >> 11) / 2.0 ** 53


def test_p2_workload_mesh():
    # the P2 workload: the c2_2d triangulation with one node per edge at its midpoint, so the
    # nodes are the points of the grid of spacing h/2 over the meshed box ((2N+1)^2 of them,
    # N cells per side), the free ones the (2n-1)^2 strictly inside Omega; every element's
    # edge nodes sit at the midpoints of its edges (v0v1, v1v2, v0v2)
    w = WORKLOADS["c2_2d_p2"]
    m = workload_mesh(w)
    n, N = w.cells[0], w.cells[0] + 2 * w.layer
    assert m.conn.shape == (2 * N * N, 6)
    assert m.n_vert == (2 * N + 1) ** 2
    assert int(m.node_free.sum()) == (2 * n - 1) ** 2
    x = m.coords
    for j, (a, b) in enumerate(((0, 1), (1, 2), (0, 2))):
        mid = (x[:, m.conn[:, a]] + x[:, m.conn[:, b]]) * 0.5
        assert np.array_equal(x[:, m.conn[:, 3 + j]], mid)
    # the vertices and the P1 mesh are those of c2_2d
    p1 = workload_mesh(WORKLOADS["c2_2d"])
    assert np.array_equal(m.conn[:, :3], p1.conn)
    assert np.array_equal(x[:, :p1.n_vert], p1.coords)


@pytest.mark.parametrize("order", [2, 3])
def test_quadratic_hex_workload_meshes(order):
    # Table 6's grid (12 x 8 x 8 cells of Omega and a 2-cell layer) with Q2 (27-node) or
    # serendipity (20-node) hexahedra: the Q2 nodes are the points of the grid of spacing h/2
    # over the meshed box, the serendipity nodes those with at most one odd half-step index
    # (vertices and edge midpoints); node a of every element sits at the trilinear image of
    # its lattice point HEX27[a] / 2, and the free nodes are those strictly inside Omega
    from nl_inputs import HEX27
    from nl_inputs.configs import table6_hex
    w = table6_hex(3).with_(order=order)
    m = workload_mesh(w)
    nb = 27 if order == 2 else 20
    cells = [c + 2 * w.layer for c in w.cells]
    assert m.conn.shape == (int(np.prod(cells)), nb)
    pts = [2 * c + 1 for c in cells]
    inner = [2 * c - 1 for c in w.cells]
    if order == 2:
        assert m.n_vert == int(np.prod(pts))
        assert int(m.node_free.sum()) == int(np.prod(inner))
    else:
        def count(even, odd):  # half-step grid points with at most one odd index
            return (even[0] * even[1] * even[2] + odd[0] * even[1] * even[2] +
                    even[0] * odd[1] * even[2] + even[0] * even[1] * odd[2])
        # the whole box: c + 1 even and c odd indices per axis; strictly inside Omega: n - 1
        # even and n odd
        assert m.n_vert == count([c + 1 for c in cells], cells)
        assert int(m.node_free.sum()) == count([c - 1 for c in w.cells], list(w.cells))
    assert len(np.unique(m.conn)) == m.n_vert
    x = m.coords
    V = x[:, m.conn[:, :8]]  # (3, elem, 8)
    corners = HEX27[:8]
    for a in range(8, nb):
        i, j, k = HEX27[a]
        w8 = [(1 - i / 2 if c[0] == 0 else i / 2) * (1 - j / 2 if c[1] == 0 else j / 2) *
              (1 - k / 2 if c[2] == 0 else k / 2) for c in [(p // 2, q // 2, r // 2) for p, q, r in corners]]
        pos = sum(w8[b] * V[:, :, b] for b in range(8))
        assert np.abs(x[:, m.conn[:, a]] - pos).max() < 1e-12, a
