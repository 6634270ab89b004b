"""Parity of the CUDA path (through the C ABI) with the oracle, on the same seeded inputs.

Tolerances: pair lists, CSR pattern and Algorithm-1 work counts bit-exact; A within 1e-12
relative Frobenius in FP64; A within 2e-6 relative Frobenius in the FP32 paths (the
point-pair values carry FP32 rounding ~6e-8 relative and the per-pair sums of up to a few
thousand terms add a few more ulps; the band terms use an FP32 square root near the
mollifier's steepest slope).
"""
import numpy as np
import pytest

import oracle as O
from nl_inputs import WORKLOADS, structured_mesh, workload_mesh
from nl_inputs.configs import table2_tri
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6


def _oracle(mesh, delta, eps, L_max, L_min=1, kernel=0, m_mask=None):
    off, pl = O.pairs(mesh, delta, eps)
    rp, col = O.csr(mesh, off, pl)
    vals, st = O.assemble(mesh, off, pl, rp, col, delta, eps, L_max, L_min, kernel, m_mask=m_mask)
    return off, pl, rp, col, vals, st


def _gpu(mesh, delta, eps, L_max, L_min=1, kernel=0, precision=nl.NL_PREC_FP64):
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, delta, eps)
    A, st = nl.nl_assemble(m, p, delta, eps, L_max, L_min, kernel, precision)
    off, pl, rp, col = p.export(mesh.n_elem, mesh.n_vert)
    return off, pl, rp, col, A.export(), st, (m, p, A)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _maxrel(a, b):
    # per entry: a few wrong entries among many cannot hide under the Frobenius norm
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [
    # (name, mesh factory, delta, eps, L_max, L_min, kernel)
    ("c1", lambda: workload_mesh(WORKLOADS["c1_2d"]), 0.1, 0.01, 3, 1, 0),
    ("jit2d_L4", lambda: structured_mesh(2, 9, 1 / 9, 0.0, 3, jitter=0.1, seed=11), 0.25, 0.03, 4, 1, 0),
    ("jit2d_L1", lambda: structured_mesh(2, 7, 1 / 7, 0.0, 2, jitter=0.1, seed=3), 0.2, 0.04, 1, 1, 0),
    ("jit2d_Lmin2", lambda: structured_mesh(2, 7, 1 / 7, 0.0, 2, jitter=0.1, seed=4), 0.2, 0.04, 3, 2, 0),
    ("gauss2d", lambda: structured_mesh(2, 8, 1 / 8, 0.0, 2, jitter=0.1, seed=5), 0.2, 0.01, 3, 1, 1),
    ("rect2d", lambda: workload_mesh(table2_tri(2)), 0.2, 0.0125, 3, 1, 0),
    ("jit3d", lambda: structured_mesh(3, 3, 1 / 3, 0.0, 1, jitter=0.1, seed=7), 0.22, 0.02, 2, 1, 0),
    ("gauss3d", lambda: structured_mesh(3, 2, 0.5, 0.0, 1, jitter=0.1, seed=8), 0.3, 0.06, 2, 1, 1),
    ("deep3d", lambda: structured_mesh(3, 2, 0.5, 0.0, 0, jitter=0.05, seed=9), 0.4, 0.05, 3, 1, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pairs_pattern_and_fp64_values(case):
    name, mk, delta, eps, L_max, L_min, kernel = case
    mesh = mk()
    ooff, opl, orp, ocol, ovals, ost = _oracle(mesh, delta, eps, L_max, L_min, kernel)
    off, pl, rp, col, vals, st, _ = _gpu(mesh, delta, eps, L_max, L_min, kernel)
    assert np.array_equal(off, ooff)
    assert np.array_equal(pl, opl)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    assert st.n_pairs == len(opl)
    assert st.n_point_pairs == ost.n_point_pairs
    assert st.n_items == ost.n_integrations
    assert _rel(vals, ovals) < TOL64
    assert _maxrel(vals, ovals) < TOL64


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp32_values(case):
    name, mk, delta, eps, L_max, L_min, kernel = case
    mesh = mk()
    *_, ovals, ost = _oracle(mesh, delta, eps, L_max, L_min, kernel)
    off, pl, rp, col, vals, st, _ = _gpu(mesh, delta, eps, L_max, L_min, kernel, nl.NL_PREC_FP32)
    assert st.n_point_pairs == ost.n_point_pairs  # FP32 screening keeps the FP64 decisions
    assert _rel(vals, ovals) < TOL32
    assert _maxrel(vals, ovals) < TOL32


def test_deep_refinement_2d():
    # L_max = 7 on a tiny mesh: deep LIFO and many FP32 screens near the thresholds; the
    # decisions must agree exactly (identical Algorithm-1 counts).  Every pair sums ~1.3e5
    # point pairs, so the FP64 values agree only to the rounding of sums that long
    # (sequential in the oracle, tree-shaped on the GPU): 1e-11 here.  In FP32 each lane
    # accumulates ~600 point pairs per inner point and pair, so the FP32 tolerance grows with
    # that count: 2e-5 here.
    mesh = structured_mesh(2, 2, 0.5, 0.0, 1, jitter=0.1, seed=2)
    *_, ovals, ost = _oracle(mesh, 0.3, 0.02, 7)
    for prec, tol in ((nl.NL_PREC_FP64, 1e-11), (nl.NL_PREC_FP32, 2e-5)):
        *_, vals, st, _ = _gpu(mesh, 0.3, 0.02, 7, precision=prec)
        assert st.n_point_pairs == ost.n_point_pairs
        assert st.n_items == ost.n_integrations
        assert _rel(vals, ovals) < tol
        assert _maxrel(vals, ovals) < tol


def test_single_element_and_two_far_elements():
    from nl_inputs.mesh import Mesh
    one = Mesh(dim=2, coords=np.array([[0.0, 0.1, 0.0], [0.0, 0.0, 0.1]]),
               conn=np.array([[0, 1, 2]], np.int32), elem_in_omega=np.ones(1, np.uint8),
               node_free=np.ones(3, np.uint8), h=0.1)
    *_, ovals, _ = _oracle(one, 0.2, 0.01, 3)
    off, pl, rp, col, vals, st, _ = _gpu(one, 0.2, 0.01, 3)
    assert list(pl) == [0] and _rel(vals, ovals) < TOL64
    two = Mesh(dim=2, coords=np.array([[0.0, 0.1, 0.0, 5.0, 5.1, 5.0], [0.0, 0.0, 0.1, 0, 0, 0.1]]),
               conn=np.array([[0, 1, 2], [3, 4, 5]], np.int32), elem_in_omega=np.ones(2, np.uint8),
               node_free=np.ones(6, np.uint8), h=0.1)
    off, pl, rp, col, vals, st, _ = _gpu(two, 0.2, 0.01, 3)
    assert list(off) == [0, 1, 2] and list(pl) == [0, 1]


def test_reassemble_into_same_matrix_and_invalid_arguments():
    mesh = structured_mesh(2, 4, 0.25, 0.0, 2)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, 0.4, 0.05)
    A, _ = nl.nl_assemble(m, p, 0.4, 0.05, 2)
    v1 = A.export()
    nl.nl_assemble(m, p, 0.4, 0.05, 2, into=A)
    assert _rel(A.export(), v1) < 1e-14
    with pytest.raises(nl.NLError) as e:
        nl.nl_assemble(m, p, 0.4, 0.05, 20)
    assert e.value.status == nl.NL_EINVAL
    with pytest.raises(nl.NLError) as e:
        nl.nl_pairs_build(m, 0.1, 0.2)
    assert e.value.status == nl.NL_EINVAL
    with pytest.raises(nl.NLError) as e:
        nl.nl_assemble(m, p, 0.41, 0.05, 2)
    assert e.value.status == nl.NL_EINVAL
    bad = structured_mesh(2, 2, 0.5, 0.0, 0)
    bad.conn[0, 0] = 10 ** 6
    with pytest.raises(nl.NLError) as e:
        nl.mesh_from(bad)
    assert e.value.status == nl.NL_EINVAL
    nan = structured_mesh(2, 2, 0.5, 0.0, 0)
    nan.coords[0, 0] = np.nan
    with pytest.raises(nl.NLError):
        nl.mesh_from(nan)


def test_box_generator_matches_input_module():
    for dim, cells, h, lo, layer, jit, seed in ((2, (5, 3), 0.2, (-0.5, 0.1), 2, 0.1, 7),
                                                (3, (3, 2, 4), 0.25, (0.0, 0.5, -1.0), 1, 0.1, 3)):
        ref = structured_mesh(dim, cells, h, lo, layer, jitter=jit, seed=seed)
        m = nl.nl_mesh_create_box(dim, cells, h, lo, layer, jit, seed)
        coords, conn, eio, nf = m.export()
        assert np.array_equal(coords, ref.coords)
        assert np.array_equal(conn, ref.conn)
        assert np.array_equal(eio, ref.elem_in_omega) and np.array_equal(nf, ref.node_free)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", [nl.NL_PREC_FP64, nl.NL_PREC_FP32])
def test_solve_matches_dense_oracle(solver, prec):
    w = WORKLOADS["c1_2d"]
    mesh = workload_mesh(w)
    ref = O.solve_problem(mesh, w.delta, w.eps, w.L_max, w.ms)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    A, _ = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max, precision=prec)
    g = np.array([O.ms_u(w.ms, mesh.coords[:, i]) for i in range(mesh.n_vert)])
    b = nl.nl_rhs(m, A, g, f_const=-4.0)
    F = b.export()
    tolF = 1e-12 if prec == nl.NL_PREC_FP64 else 5e-6
    assert np.linalg.norm(F - ref["F"]) <= tolF * np.linalg.norm(ref["F"])
    u, it, rr, _ = nl.nl_solve(A, b, g, solver=solver, rtol=1e-12, precision=nl.NL_PREC_FP64)
    assert rr <= 1e-12
    tolu = 1e-9 if prec == nl.NL_PREC_FP64 else 1e-5
    assert np.abs(u - ref["u_h"]).max() <= tolu * np.abs(ref["u_h"]).max()
    err = O.l2_error(mesh, u, w.ms, omega_only=True)
    assert abs(err / ref["err_omega"] - 1) < (1e-8 if prec == nl.NL_PREC_FP64 else 1e-3)


def test_mixed_solver_refinement():
    w = WORKLOADS["c1_2d"]
    mesh = workload_mesh(w)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    A, _ = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max)
    g = np.array([O.ms_u(w.ms, mesh.coords[:, i]) for i in range(mesh.n_vert)])
    b = nl.nl_rhs(m, A, g, f_const=-4.0)
    u64, *_ = nl.nl_solve(A, b, g, solver=1, rtol=1e-12)
    u32, it, rr, _ = nl.nl_solve(A, b, g, solver=1, rtol=1e-12, precision=nl.NL_PREC_FP32)
    assert rr <= 1e-12
    assert np.abs(u32 - u64).max() <= 1e-10 * np.abs(u64).max()


def test_table2_tri_linear_on_gpu():
    gold = {2: 4.373e-3, 3: 1.094e-3}
    for ml in (2, 3):
        w = table2_tri(ml)
        mesh = workload_mesh(w)
        m = nl.mesh_from(mesh)
        p = nl.nl_pairs_build(m, w.delta, w.eps)
        A, _ = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max)
        g = np.array([O.ms_u(w.ms, mesh.coords[:, i]) for i in range(mesh.n_vert)])
        f = np.array([O.ms_f(w.ms, mesh.coords[:, i], 0, w.delta, w.eps,
                             O.kernel_constant(2, 0, w.delta, w.eps)) for i in range(mesh.n_vert)])
        b = nl.nl_rhs(m, A, g, f_nodes=f)  # f = -6(x+y) is linear: its P1 interpolant is exact
        u, *_ = nl.nl_solve(A, b, g, solver=1, rtol=1e-13)
        err = O.l2_error(mesh, u, w.ms, omega_only=False)
        assert abs(err / gold[ml] - 1) < 2e-3, (ml, err)


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in ("c1", "jit2d_L4", "gauss2d", "jit3d")],
                         ids=lambda c: c[0])
def test_band_point_pair_counts(case):
    # the band counter feeds the benchmark's algorithmic flop count: point pairs with
    # delta - eps <= r <= delta + eps, against the oracle's count (only the rounding of r at
    # the two band edges may differ)
    name, mk, delta, eps, L_max, L_min, kernel = case
    mesh = mk()
    off, pl = O.pairs(mesh, delta, eps)
    rp, col = O.csr(mesh, off, pl)
    _, ost = O.assemble(mesh, off, pl, rp, col, delta, eps, L_max, L_min, kernel)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, delta, eps)
    for prec, tol in ((nl.NL_PREC_FP64, 1e-9), (nl.NL_PREC_FP32, 1e-4)):
        _, st = nl.nl_assemble(m, p, delta, eps, L_max, L_min, kernel, prec, count_band=True)
        assert abs(st.n_band_point_pairs - ost.n_band_pairs) <= tol * ost.n_band_pairs + 2, (
            name, prec, st.n_band_point_pairs, ost.n_band_pairs)


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in ("c1", "jit2d_L4", "jit2d_Lmin2",
                                                               "gauss2d", "jit3d", "deep3d")],
                         ids=lambda c: c[0])
def test_euclidean_min_dist_counts_and_values(case):
    # NL_QUAD_MINDIST_L2: Algorithm 1's refinement test with the Euclidean minimum distance of
    # Sec. 5.1; the work counts equal the oracle's with the same test, bit for bit, in both
    # precisions (FP32 screen with its own margin, FP64 decision inside it), and the matrix is
    # the default one (only contributions that are exactly zero are left out)
    name, mk, delta, eps, L_max, L_min, kernel = case
    mesh = mk()
    off, pl = O.pairs(mesh, delta, eps)
    rp, col = O.csr(mesh, off, pl)
    ovals, ost = O.assemble(mesh, off, pl, rp, col, delta, eps, L_max, L_min, kernel,
                            mindist_l2=True)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, delta, eps)
    for prec, tol in ((nl.NL_PREC_FP64, TOL64), (nl.NL_PREC_FP32, TOL32)):
        A, st = nl.nl_assemble(m, p, delta, eps, L_max, L_min, kernel, prec, mindist_l2=True)
        vals = A.export()
        assert st.n_items == ost.n_integrations, (name, prec)
        assert st.n_point_pairs == ost.n_point_pairs, (name, prec)
        assert _rel(vals, ovals) < tol and _maxrel(vals, ovals) < tol, (name, prec)


# The tensor-core paths (NL_PREC_MIXED_TF32 / BF16): the contraction over the outer points on
# mma.sync with two-part split operands, everything else as in NL_PREC_FP32.  Tolerances
# against the FP64 oracle, relative Frobenius and per entry: the TF32 parts carry about 22
# significant bits, and the tensor cores' FP32 accumulation over each batch of 32 outer
# points rounds less tightly than the ALU's FMAs (the deep 3D case measured 5.4e-6 with
# unbounded accumulation chains): 1e-5; the BF16 parts carry about 16 bits: 1e-4.
MMA_TOL = {nl.NL_PREC_MIXED_TF32: 1e-5, nl.NL_PREC_MIXED_BF16: 1e-4}


@pytest.mark.parametrize("prec", [nl.NL_PREC_MIXED_TF32, nl.NL_PREC_MIXED_BF16],
                         ids=["tf32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_values(case, prec):
    name, mk, delta, eps, L_max, L_min, kernel = case
    mesh = mk()
    *_, ovals, ost = _oracle(mesh, delta, eps, L_max, L_min, kernel)
    off, pl, rp, col, vals, st, _ = _gpu(mesh, delta, eps, L_max, L_min, kernel, prec)
    assert st.precision_run == prec
    assert st.n_point_pairs == ost.n_point_pairs and st.n_items == ost.n_integrations
    tol = MMA_TOL[prec]
    assert _rel(vals, ovals) < tol, (name, _rel(vals, ovals))
    assert _maxrel(vals, ovals) < tol, (name, _maxrel(vals, ovals))


def test_precision_run_is_reported():
    mesh = structured_mesh(2, 4, 0.25, 0.0, 2)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, 0.4, 0.05)
    for prec in (nl.NL_PREC_FP64, nl.NL_PREC_FP32, nl.NL_PREC_MIXED_TF32, nl.NL_PREC_MIXED_BF16):
        _, st = nl.nl_assemble(m, p, 0.4, 0.05, 2, precision=prec)
        assert st.precision_run == prec
    # the no-allocation entry point and plans run the mixed precisions in FP32 and say so
    pl = nl.Plan([(m, p, 0.4, 0.05, 2, 1, 0)], precision=nl.NL_PREC_MIXED_TF32)
    pl.execute()
    assert pl.sync()[0].precision_run == nl.NL_PREC_FP32


def test_matrix_apply_equals_csr_product():
    # nl_matrix_apply: y = A x over every row on the device, against the CSR product of the
    # exported values (FP64; only the summation order differs)
    import torch
    mesh = structured_mesh(3, 3, 1 / 3, 0.0, 1, jitter=0.1, seed=7)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, 0.22, 0.02)
    A, _ = nl.nl_assemble(m, p, 0.22, 0.02, 2)
    vals = A.export()
    _, _, rp, col = p.export(mesh.n_elem, mesh.n_vert)
    x = np.random.default_rng(3).standard_normal(mesh.n_vert)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    A.apply(xd.data_ptr(), yd.data_ptr())
    torch.cuda.synchronize()
    rows = np.repeat(np.arange(mesh.n_vert), np.diff(rp))
    ref = np.bincount(rows, weights=vals * x[col], minlength=mesh.n_vert)
    assert np.abs(yd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(vals).max() * np.abs(x).max() * 64
    with pytest.raises(nl.NLError) as e:
        A.apply(xd.data_ptr(), xd.data_ptr())
    assert e.value.status == nl.NL_EINVAL
