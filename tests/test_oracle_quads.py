"""The oracle's quadrilateral elements (Sec. 6: QUAD meshes, Q1 bilinear and Q2 biquadratic
Lagrange elements, Gauss-Legendre 3x3 for the inner and the outer integral) against what the
paper and the mathematics fix: the printed QUAD columns of Tables 1-3, exact integrals,
closed-form local matrices of fully-interior pairs, Algorithm 1 against brute-force uniform
refinement, zero row sums, symmetry at one level and linear consistency.
"""
import math

import numpy as np
import pytest

import oracle as O
from nl_inputs import q2_mesh, quad_mesh, s2_mesh, structured_mesh, workload_mesh
from nl_inputs.configs import table2_tri, table3_tri
from nl_inputs.mesh import Mesh


def _golden(name, col=1):
    import os
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if line.strip() and not line.startswith("#"):
            parts = line.split()
            rows[int(parts[0])] = float(parts[col])
    return rows


def _quads(w, order=1):
    # order 1: Q1, 2: Q2, 3: the 8-node serendipity element
    m = quad_mesh(workload_mesh(w))
    if order == 1:
        return m
    return q2_mesh(m) if order == 2 else s2_mesh(q2_mesh(m))


# ---- geometry and rule ------------------------------------------------------------------------

@pytest.mark.parametrize("order", [1, 2, 3])
def test_l2_norm_of_a_quadratic_over_jittered_quadrilaterals(order):
    # ||x^2 + y^2||_{L2} over the meshed box, through the error routine with u_h = 0: the
    # bilinear maps of the jittered cells tile the box exactly (boundary vertices stay), and
    # Gauss-Legendre 3x3 integrates (x^2 + y^2)^2 |det DF| exactly (degree <= 5 per reference
    # variable), so the result is the closed form whatever the jitter
    w = table2_tri(2).with_(jitter=0.2, seed=3, ms=1)
    m = _quads(w, order)
    x0, x1 = -0.6 - 0.2, 0.6 + 0.2
    y0, y1 = -0.4 - 0.2, 0.4 + 0.2

    def I(a, b, p):
        return (b ** (p + 1) - a ** (p + 1)) / (p + 1)
    exact = (I(x0, x1, 4) * (y1 - y0) + 2 * I(x0, x1, 2) * I(y0, y1, 2) + (x1 - x0) * I(y0, y1, 4))
    got = O.l2_error(m, np.zeros(m.n_vert), 1, omega_only=False)
    assert abs(got ** 2 / exact - 1) < 1e-13


# ---- local matrices ------------------------------------------------------------------------

def test_fully_interior_quad_pairs_closed_form():
    # two h x h squares well inside delta - eps of each other: mu = 1 at every point pair and
    # A is the closed form of the constant kernel with the Q1 mass matrix of a square,
    # M(a,b) = h^2/36 (4 same node, 2 neighbours, 1 opposite), and int phi_a = h^2 / 4:
    #   +2 C |E_l| M(a,b) on (m_a, m_b),  -2 C (h^2/4)^2 on (m_a, l_c)
    h, delta, eps = 0.05, 1.0, 0.1
    sq = np.array([[0, 0], [h, 0], [h, h], [0, h]], float)
    coords = np.concatenate([sq, sq + [0.3, 0.1]]).T.copy()
    mesh = Mesh(dim=2, coords=coords, conn=np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32),
                elem_in_omega=np.ones(2, np.uint8), node_free=np.ones(8, np.uint8), h=h)
    off, pl = O.pairs(mesh, delta, eps)
    rp, col = O.csr(mesh, off, pl)
    C = O.kernel_constant(2, O.KERNEL_CONST, delta, eps)
    Mq = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) * h * h / 36
    ref = np.zeros((8, 8))
    for mm in range(2):
        for ll in range(2):
            nm, nl = np.arange(4) + 4 * mm, np.arange(4) + 4 * ll
            ref[np.ix_(nm, nm)] += 2 * C * h * h * Mq
            ref[np.ix_(nm, nl)] -= 2 * C * (h * h / 4) ** 2
    for L in (1, 3):
        vals, st = O.assemble(mesh, off, pl, rp, col, delta, eps, L)
        got = np.zeros((8, 8))
        for i in range(8):
            got[i, col[rp[i]:rp[i + 1]]] = vals[rp[i]:rp[i + 1]]
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), L
        assert st.n_integrations == 4 and st.n_point_pairs == 4 * 81 and st.n_band_pairs == 0


def _lagrange1d(order, s):
    if order == 2:
        return np.stack([2 * (s - 0.5) * (s - 1), 4 * s * (1 - s), 2 * s * (s - 0.5)], -1)
    return np.stack([1 - s, s], -1)


def _qbasis(order, s, t):
    if order == 3:  # serendipity: corners and edge midpoints of [-1, 1]^2
        xi, eta = 2 * s - 1, 2 * t - 1
        nd = [(-1, -1), (1, -1), (1, 1), (-1, 1), (0, -1), (1, 0), (0, 1), (-1, 0)]
        out = []
        for xa, ya in nd:
            if xa != 0 and ya != 0:
                out.append((1 + xi * xa) * (1 + eta * ya) * (xi * xa + eta * ya - 1) / 4)
            elif xa == 0:
                out.append((1 - xi * xi) * (1 + eta * ya) / 2)
            else:
                out.append((1 + xi * xa) * (1 - eta * eta) / 2)
        return np.stack(out, -1)
    Ls, Lt = _lagrange1d(order, s), _lagrange1d(order, t)
    ij = [(0, 0), (1, 0), (1, 1), (0, 1)] if order == 1 else \
        [(0, 0), (2, 0), (2, 2), (0, 2), (1, 0), (2, 1), (1, 2), (0, 1), (1, 1)]
    return np.stack([Ls[..., i] * Lt[..., j] for i, j in ij], -1)


def _bilinear(V, s, t):
    N = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], -1)
    X = N @ V
    xs = (1 - t)[:, None] * (V[1] - V[0]) + t[:, None] * (V[2] - V[3])
    xt = (1 - s)[:, None] * (V[3] - V[0]) + s[:, None] * (V[2] - V[1])
    return X, np.abs(xs[:, 0] * xt[:, 1] - xs[:, 1] * xt[:, 0])


def _uniform_quad_blocks(Vl, Vm, order, delta, eps, C, depth):
    """Outer integral over E_l on the 4^depth sub-squares of its unit square (Gauss-Legendre
    3x3 on each), inner Gauss-Legendre 3x3 on E_m: the blocks 2 S and -2 X."""
    x, w = np.polynomial.legendre.leggauss(3)
    g, gw = (x + 1) / 2, w / 2
    n = 2 ** depth
    i, j, a, b = np.meshgrid(np.arange(n), np.arange(n), np.arange(3), np.arange(3), indexing="ij")
    s, t = ((i + g[a]) / n).ravel(), ((j + g[b]) / n).ravel()
    X, detl = _bilinear(Vl, s, t)
    WX = (gw[a] * gw[b]).ravel() / (n * n) * detl
    PL = _qbasis(order, s, t)
    a2, b2 = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    sm, tm = g[a2].ravel(), g[b2].ravel()
    Y, detm = _bilinear(Vm, sm, tm)
    WY = (gw[a2] * gw[b2]).ravel() * detm
    PM = _qbasis(order, sm, tm)
    R = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    MU = np.vectorize(lambda r: O.mu(r, delta, eps))(R)
    G = WX[:, None] * WY[None, :] * C * MU
    return 2 * np.einsum("xy,ya,yb->ab", G, PM, PM), -2 * np.einsum("xy,ya,xc->ac", G, PM, PL)


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("offset", [0.17, 0.205, 0.215])
def test_algorithm1_quads_equal_uniform_refinement(order, offset):
    # Constant kernel: Algorithm 1 at L_max = L and uniform refinement of l's unit square to
    # level L give the same sums up to rounding (an INT sub-element's integrand phi^l_d |det
    # DF_l| has degree <= 3 per reference variable, which Gauss-Legendre 3 integrates exactly;
    # dropped sub-elements have mu = 0 at every point pair).  General (non-parallelogram)
    # quadrilaterals, so the bilinear map's Jacobian varies.
    Vm = np.array([[0.0, 0.0], [0.06, 0.01], [0.055, 0.05], [-0.004, 0.045]])
    Vl = np.array([[offset, 0.02], [offset + 0.05, 0.0], [offset + 0.06, 0.055], [offset + 0.01, 0.06]])
    coords = np.concatenate([Vm, Vl]).T.copy()
    conn = np.array([[0, 1, 2, 3], [4, 5, 6, 7]], np.int32)
    if order >= 2:
        ne = 5 if order == 2 else 4  # Q2: edge midpoints and centre; serendipity: edges only
        extra, cz = [], []
        for e, V in enumerate((Vm, Vl)):
            mids = [(V[0] + V[1]) / 2, (V[1] + V[2]) / 2, (V[2] + V[3]) / 2, (V[3] + V[0]) / 2,
                    ((V[0] + V[1]) / 2 + (V[2] + V[3]) / 2) / 2][:ne]
            cz.append(list(conn[e]) + [8 + ne * e + k for k in range(ne)])
            extra += mids
        coords = np.concatenate([np.concatenate([Vm, Vl]), np.array(extra)]).T.copy()
        conn = np.array(cz, np.int32)
    nn = coords.shape[1]
    mesh = Mesh(dim=2, coords=coords, conn=conn, elem_in_omega=np.ones(2, np.uint8),
                node_free=np.ones(nn, np.uint8), h=0.05)
    delta, eps = 0.2, 0.01
    C = O.kernel_constant(2, O.KERNEL_CONST, delta, eps)
    off, pl = O.pairs(mesh, delta, eps)
    assert len(pl) == 4
    rp, col = O.csr(mesh, off, pl)
    for L in (1, 3, 4):
        vals, _ = O.assemble(mesh, off, pl, rp, col, delta, eps, L)
        got = np.zeros((nn, nn))
        for i in range(nn):
            got[i, col[rp[i]:rp[i + 1]]] = vals[rp[i]:rp[i + 1]]
        ref = np.zeros((nn, nn))
        for (mi, li) in ((0, 0), (0, 1), (1, 0), (1, 1)):
            S2, X2 = _uniform_quad_blocks((Vm, Vl)[li], (Vm, Vl)[mi], order, delta, eps, C, L - 1)
            ref[np.ix_(conn[mi], conn[mi])] += S2
            ref[np.ix_(conn[mi], conn[li])] += X2
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (order, L)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_quad_zero_row_sums_symmetry_and_linear_consistency(order):
    # the Q1 / Q2 / serendipity basis sums to one, so every row sums to zero; at L_max = 1 the inner and
    # outer rules coincide and A is symmetric; u = 1 + x + y (f = 0) is reproduced
    w = table2_tri(2).with_(jitter=0.15, seed=5)
    m = _quads(w, order)
    off, pl = O.pairs(m, 0.2, 0.0125)
    rp, col = O.csr(m, off, pl)
    v1, _ = O.assemble(m, off, pl, rp, col, 0.2, 0.0125, 1)
    rows = np.repeat(np.arange(m.n_vert), np.diff(rp))
    assert np.abs(np.bincount(rows, weights=v1, minlength=m.n_vert)).max() < 1e-12 * np.abs(v1).max()
    import scipy.sparse as sp
    A = sp.csr_matrix((v1, col, rp), shape=(m.n_vert, m.n_vert))
    assert abs(A - A.T).max() < 1e-14 * np.abs(v1).max()
    r = O.solve_problem(_quads(table2_tri(2), order), 0.2, 0.0125, 3, 0)
    assert r["err_all"] < 1e-6


# ---- the printed QUAD columns of Sec. 6 ---------------------------------------------------------

@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("L_max", [3, 4])
def test_table1_quad_consistency(L_max, order):
    # Table 1, QUAD (quadratic FE, u = x^2 + y^2 in the FE space, h = 0.1, delta = 0.2,
    # eps = 0.0125 (3/4)^(L_max - 3)): only the integration and mollifier errors remain;
    # printed 8.123e-5, 1.278e-5 (and 3.453e-7 at L_max = 5, reproduced by Q2 to 3.4544e-7,
    # 10 s, not in the suite).  The serendipity element contains u as well and gives the same
    # errors to 0.02 %.
    gold = _golden("table1_quad_quadratic.txt")
    m2 = _quads(table2_tri(2), order)
    eps = 0.0125 * 0.75 ** (L_max - 3)
    err = O.solve_problem(m2, 0.2, eps, L_max, 1)["err_all"]
    assert abs(err / gold[L_max] - 1) < 2e-3, err


@pytest.mark.parametrize("ml", [2, 3])
@pytest.mark.parametrize("table,fn,gold_file", [("2", table2_tri, "table2_quad.txt"),
                                                 ("3", table3_tri, "table3_quad.txt")])
def test_tables_2_3_quad_bilinear(table, fn, gold_file, ml):
    # Tables 2 and 3, QUAD bilinear column: the printed errors to 0.2 % (the quartic case
    # carries the kernel's fourth moment in its forcing)
    gold = _golden(gold_file, 1)
    w = fn(ml)
    err = O.solve_problem(_quads(w, 1), w.delta, w.eps, w.L_max, w.ms)["err_all"]
    assert abs(err / gold[ml] - 1) < 2e-3, (table, ml, err)


@pytest.mark.parametrize("table,fn,gold_file", [("2", table2_tri, "table2_quad.txt"),
                                                 ("3", table3_tri, "table3_quad.txt")])
def test_tables_2_3_quad_quadratic_order(table, fn, gold_file):
    # Tables 2 and 3, QUAD quadratic column at ml = 2, 3: third order (printed 3.090 and
    # 2.892; P1 would give 2) and the printed errors within 25 % (the oracle gives 7.12e-5,
    # 8.51e-6 and 1.16e-4, 1.38e-5; the consistency test of Table 1 on the same elements
    # matches to four digits, so the h-convergence runs differ in a detail the text leaves
    # open, listed among the readings)
    gold = _golden(gold_file, 3)
    errs = {}
    for ml in (2, 3):
        w = fn(ml)
        errs[ml] = O.solve_problem(_quads(w, 2), w.delta, w.eps, w.L_max, w.ms)["err_all"]
        assert abs(errs[ml] / gold[ml] - 1) < 0.25, (table, ml, errs[ml])
    p = math.log2(errs[2] / errs[3])
    assert 2.8 < p < 3.3, (table, p)
