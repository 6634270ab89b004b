"""P2 tetrahedra on the GPU (the quadratic simplex in 3D), through the C ABI, against the oracle
on the same seeded meshes.

Tolerances as for the other elements (test_gpu_parity): pair lists, CSR pattern and
Algorithm-1 work counts bit-exact; A within 1e-12 relative (Frobenius, and per entry against
the largest entry) in FP64 and 2e-6 in FP32; the whole GPU path's solution equal to the
oracle's dense solve to 1e-9.
"""
import numpy as np
import pytest

import oracle as O
from nl_inputs import WORKLOADS, p2_mesh, structured_mesh, workload_mesh
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6


def _m(jitter, seed, n=2, layer=1):
    return p2_mesh(structured_mesh(3, n, 1 / n, 0.0, layer, jitter=jitter, seed=seed))


CASES = [
    # (name, mesh factory, delta, eps, L_max, L_min, kernel, mindist_l2)
    ("jit_L1", lambda: _m(0.1, 1), 0.3, 0.03, 1, 1, 0, False),
    ("jit_L2", lambda: _m(0.1, 2), 0.3, 0.03, 2, 1, 0, False),
    ("jit_Lmin2", lambda: _m(0.1, 3), 0.3, 0.03, 2, 2, 0, False),
    ("gauss", lambda: _m(0.1, 4), 0.3, 0.015, 2, 1, 1, False),
    ("euclid", lambda: _m(0.1, 5), 0.3, 0.03, 2, 1, 0, True),
]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_p2_tet_pairs_pattern_counts_and_values(case):
    name, mk, delta, eps, L_max, L_min, kernel, l2 = case
    mesh = mk()
    off0, pl0 = O.pairs(mesh, delta, eps)
    rp0, col0 = O.csr(mesh, off0, pl0)
    v0, st0 = O.assemble(mesh, off0, pl0, rp0, col0, delta, eps, L_max, L_min, kernel, mindist_l2=l2)
    m = nl.mesh_from(mesh)
    assert m.order() == (2, 10)
    p = nl.nl_pairs_build(m, delta, eps)
    off, pl, rp, col = p.export(mesh.n_elem, mesh.n_vert)
    assert np.array_equal(off, off0)
    assert np.array_equal(pl, pl0)
    assert np.array_equal(rp, rp0)
    assert np.array_equal(col, col0)
    for prec, tol in ((nl.NL_PREC_FP64, TOL64), (nl.NL_PREC_FP32, TOL32)):
        A, st = nl.nl_assemble(m, p, delta, eps, L_max, L_min, kernel, prec, mindist_l2=l2)
        vals = A.export()
        assert st.precision_run == prec
        assert st.n_items == st0.n_integrations, (name, prec)
        assert st.n_point_pairs == st0.n_point_pairs, (name, prec)
        assert st.n_eval_point_pairs + 196 * st.n_closed_items <= st.n_point_pairs
        assert _rel(vals, v0) < tol, (name, prec, _rel(vals, v0))
        assert _maxrel(vals, v0) < tol, (name, prec, _maxrel(vals, v0))


def test_p2_tet_mesh_validation_and_solve():
    mesh = _m(0.0, 0)
    bad = mesh.coords.copy()
    bad[2, mesh.conn[3, 9]] += 1e-3  # edge node (2,3) of element 3 off its midpoint
    with pytest.raises(nl.NLError):
        nl.nl_mesh_create_p2(3, bad, mesh.conn, mesh.elem_in_omega, mesh.node_free)
    # the whole GPU path (pairs, assembly, right-hand side with lifting, BiCGStab) against the
    # oracle's dense solve, for u = x^2 + y^2 + z^2 (in the FE space; f = -6)
    delta, eps, L = 0.3, 0.03, 1
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, delta, eps)
    A, _ = nl.nl_assemble(m, p, delta, eps, L)
    g = np.array([O.ms_u(1, mesh.coords[:, i]) for i in range(mesh.n_vert)])
    C = O.kernel_constant(3, 0, delta, eps)
    f = np.array([O.ms_f(1, mesh.coords[:, i], 0, delta, eps, C) for i in range(mesh.n_vert)])
    b = nl.nl_rhs(m, A, g, f_nodes=f)
    u, *_ = nl.nl_solve(A, b, g, solver=1, rtol=1e-13)
    ref = O.solve_problem(mesh, delta, eps, L, 1)
    assert np.abs(u - ref["u_h"]).max() / np.abs(ref["u_h"]).max() < 1e-9


def test_p2_tet_full_size_sampled_rows():
    # the 3D workload at h = 1/16 with P2 elements (63,888 tetrahedra): whole matrix on the GPU,
    # rows of two seeded nodes (a vertex inside Omega and an edge node in the layer) against
    # the oracle assembling only the elements around them
    w = WORKLOADS["c3_3d_p2"]
    mesh = workload_mesh(w)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    rng = np.random.default_rng(29)
    x = mesh.coords
    lo = np.array(w.lo)
    hi = lo + np.array(w.cells) * w.h
    inside = np.all((x > lo[:, None] + 1e-9) & (x < hi[:, None] - 1e-9), axis=0)
    layer = ~np.all((x >= lo[:, None] - 1e-9) & (x <= hi[:, None] + 1e-9), axis=0)
    is_vertex = np.arange(mesh.n_vert) <= mesh.conn[:, :4].max()
    nodes = [int(rng.choice(np.flatnonzero(inside & is_vertex))),
             int(rng.choice(np.flatnonzero(layer & ~is_vertex)))]
    mask = np.zeros(mesh.n_elem, np.uint8)
    for i in nodes:
        mask[np.any(mesh.conn == i, axis=1)] = 1
    ooff, opl = O.pairs(mesh, w.delta, w.eps, m_mask=mask)
    orp, ocol = O.csr(mesh, ooff, opl)
    ovals, _ = O.assemble(mesh, ooff, opl, orp, ocol, w.delta, w.eps, w.L_max, w.L_min, w.kernel,
                          m_mask=mask)
    _, _, rp, col = p.export(mesh.n_elem, mesh.n_vert)
    for prec, tol in ((nl.NL_PREC_FP64, TOL64), (nl.NL_PREC_FP32, TOL32)):
        A, _ = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, prec)
        vals = A.export()
        for i in nodes:
            assert np.array_equal(col[rp[i]:rp[i + 1]], ocol[orp[i]:orp[i + 1]]), i
            g_row, o_row = vals[rp[i]:rp[i + 1]], ovals[orp[i]:orp[i + 1]]
            assert np.linalg.norm(g_row - o_row) / np.linalg.norm(o_row) < tol, (prec, i)
