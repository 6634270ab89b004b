"""The oracle's P2 tetrahedra (quadratic Lagrange: the vertices, then the midpoints of the
edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3)) against what the mathematics fixes: Algorithm 1
against brute-force uniform Bey refinement with the P2 basis written out independently, zero
row sums, symmetry at one level, linear consistency, and the quadratic solution (in the FE
space) reproduced up to errors that fall with L_max.  The paper prints no P2 tetrahedron
values (its 3D tests use hexahedra).
"""
import numpy as np
import pytest

import oracle as O
from nl_inputs import p2_mesh, structured_mesh
from nl_inputs.mesh import Mesh
from test_oracle_pins import _bey_children, _tet_vol

EDGES = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]


def _p2_basis(lam):
    """(n, 4) barycentric coordinates -> (n, 10) P2 basis values."""
    cols = [lam[:, a] * (2 * lam[:, a] - 1) for a in range(4)]
    cols += [4 * lam[:, i] * lam[:, j] for i, j in EDGES]
    return np.stack(cols, 1)


def _uniform_p2_blocks(Vl, Vm, delta, eps, C, depth):
    """Outer integral over E_l split uniformly by Bey's rule `depth` times (14-point rule on
    every piece), inner 14-point rule on E_m, P2 bases: the blocks 2 S and -2 X."""
    b, w = O.quad_rule(3)
    tets = [np.array(Vl)]
    for _ in range(depth):
        tets = [c for T in tets for c in _bey_children(T)]
    X = np.concatenate([b @ T for T in tets])
    WX = np.concatenate([w * _tet_vol(T) for T in tets])
    Vl = np.array(Vl)
    Tl = np.stack([Vl[1] - Vl[0], Vl[2] - Vl[0], Vl[3] - Vl[0]], axis=1)
    l123 = np.linalg.solve(Tl, (X - Vl[0]).T).T
    PL = _p2_basis(np.column_stack([1 - l123.sum(1), l123]))
    Vm = np.array(Vm)
    Y = b @ Vm
    WY = w * _tet_vol(Vm)
    PM = _p2_basis(b)
    R = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    MU = np.vectorize(lambda r: O.mu(r, delta, eps))(R)
    G = WX[:, None] * WY[None, :] * C * MU
    return 2 * np.einsum("xy,ya,yb->ab", G, PM, PM), -2 * np.einsum("xy,ya,xc->ac", G, PM, PL)


@pytest.mark.parametrize("offset", [0.16, 0.2])
def test_algorithm1_p2_tets_equal_uniform_refinement(offset):
    # constant kernel: Algorithm 1 at L_max = L and uniform Bey refinement to level L give the
    # same sums up to rounding (an INT sub-element's integrand is the quadratic phi^l_d, which
    # the degree-5 rule integrates exactly; dropped ones have mu = 0 at every point pair)
    Vm = np.array([[0.0, 0.0, 0.0], [0.05, 0.01, 0.0], [0.01, 0.05, 0.01], [0.01, 0.01, 0.05]])
    Vl = np.array([[offset, 0.02, 0.0], [offset + 0.05, 0.0, 0.01], [offset + 0.02, 0.05, 0.0],
                   [offset + 0.01, 0.02, 0.05]])
    pts, conn = [], []
    for e, V in enumerate((Vm, Vl)):
        base = len(pts)
        pts += list(V) + [(V[i] + V[j]) / 2 for i, j in EDGES]
        conn.append(list(range(base, base + 10)))
    coords = np.array(pts).T.copy()
    mesh = Mesh(dim=3, coords=coords, conn=np.array(conn, np.int32),
                elem_in_omega=np.ones(2, np.uint8), node_free=np.ones(20, np.uint8), h=0.05)
    delta, eps = 0.2, 0.01
    C = O.kernel_constant(3, O.KERNEL_CONST, delta, eps)
    off, pl = O.pairs(mesh, delta, eps)
    assert len(pl) == 4
    rp, col = O.csr(mesh, off, pl)
    for L in (1, 2, 3):
        vals, st = O.assemble(mesh, off, pl, rp, col, delta, eps, L)
        got = np.zeros((20, 20))
        for i in range(20):
            got[i, col[rp[i]:rp[i + 1]]] = vals[rp[i]:rp[i + 1]]
        ref = np.zeros((20, 20))
        for (mi, li) in ((0, 0), (0, 1), (1, 0), (1, 1)):
            S2, X2 = _uniform_p2_blocks((Vm, Vl)[li], (Vm, Vl)[mi], delta, eps, C, L - 1)
            ref[np.ix_(conn[mi], conn[mi])] += S2
            ref[np.ix_(conn[mi], conn[li])] += X2
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), L


def test_p2_tets_zero_row_sums_symmetry_and_consistency():
    # the P2 basis sums to one (zero row sums); one level makes the rules coincide (symmetry);
    # u = 1 + x + y + z is reproduced; u = x^2 + y^2 + z^2 (in the FE space) up to the
    # integration and mollifier errors, smaller with one more level
    m = p2_mesh(structured_mesh(3, 2, 0.5, 0.0, 1, jitter=0.1, seed=3))
    off, pl = O.pairs(m, 0.3, 0.03)
    rp, col = O.csr(m, off, pl)
    v1, _ = O.assemble(m, off, pl, rp, col, 0.3, 0.03, 1)
    rows = np.repeat(np.arange(m.n_vert), np.diff(rp))
    assert np.abs(np.bincount(rows, weights=v1, minlength=m.n_vert)).max() < 1e-12 * np.abs(v1).max()
    import scipy.sparse as sp
    A = sp.csr_matrix((v1, col, rp), shape=(m.n_vert, m.n_vert))
    assert abs(A - A.T).max() < 1e-14 * np.abs(v1).max()
    m2 = p2_mesh(structured_mesh(3, 2, 0.5, 0.0, 1))
    assert O.solve_problem(m2, 0.3, 0.03, 1, 0)["err_all"] < 1e-12
    e1 = O.solve_problem(m2, 0.3, 0.03, 1, 1)["err_all"]
    e2 = O.solve_problem(m2, 0.3, 0.03, 2, 1)["err_all"]
    assert e2 < 0.6 * e1, (e1, e2)
