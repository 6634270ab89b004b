"""Batched assembly (nl_plan_*): many problems of different sizes, kernels and refinement
depths in one launch must give, problem by problem, the matrix that nl_assemble gives alone,
and the oracle's matrix for a problem small enough to run it.

Tolerances: FP64 1e-12 relative Frobenius (only the order of FP64 additions differs); FP32
2e-6 (the chunking of the work counter decides how the FP32 self-block sums of one inner
element are grouped, so the FP32 rounding differs from a single-problem run at the level of
the FP32 path's own error); work counts bit-exact (the int/ref/drop decisions do not depend
on the batching)."""
import numpy as np
import pytest

import oracle as O
from nl_inputs import structured_mesh
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu

TOL = {nl.NL_PREC_FP64: 1e-12, nl.NL_PREC_FP32: 2e-6}

# (dim, cells, delta/h, eps/delta, L_max, L_min, kernel, jitter seed)
MIX2 = [(2, 12, 3.0, 0.1, 4, 1, 0, 1), (2, 20, 2.5, 0.2, 2, 1, 0, 2), (2, 8, 4.0, 0.1, 5, 1, 1, 3),
        (2, 5, 2.0, 0.25, 3, 2, 0, 4), (2, 16, 3.5, 0.05, 3, 1, 1, 5)]
MIX3 = [(3, 3, 2.0, 0.1, 2, 1, 0, 6), (3, 4, 1.5, 0.2, 2, 1, 1, 7), (3, 2, 2.5, 0.1, 3, 1, 0, 8)]


def _problem(dim, n, dh, er, L_max, L_min, kernel, seed):
    h = 1.0 / n
    delta = dh * h
    eps = er * delta
    layer = int(np.ceil((delta + eps) / h - 1e-9))
    mesh = structured_mesh(dim, n, h, 0.0, layer, jitter=0.1, seed=seed)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, delta, eps)
    return mesh, m, p, delta, eps, L_max, L_min, kernel


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [nl.NL_PREC_FP64, nl.NL_PREC_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("mix", [MIX2, MIX3], ids=["2d", "3d"])
def test_plan_equals_single_problem_assembly(mix, prec):
    probs = [_problem(*spec) for spec in mix]
    plan = nl.Plan([(m, p, d, e, L, Lm, k) for (_, m, p, d, e, L, Lm, k) in probs], precision=prec)
    plan.execute()
    stats = plan.sync()
    for k, (mesh, m, p, d, e, L, Lm, kern) in enumerate(probs):
        A, st = nl.nl_assemble(m, p, d, e, L, Lm, kern, prec)
        ref = A.export()
        got = plan.export(k)
        assert _rel(got, ref) < TOL[prec], (k, _rel(got, ref))
        assert stats[k].n_pairs == st.n_pairs
        assert stats[k].n_items == st.n_items
        assert stats[k].n_eval_point_pairs == st.n_eval_point_pairs
        assert stats[k].n_closed_items == st.n_closed_items


@pytest.mark.parametrize("prec", [nl.NL_PREC_FP64, nl.NL_PREC_FP32], ids=["fp64", "fp32"])
def test_plan_problem_matches_oracle(prec):
    # a small problem batched behind a larger one, checked against the oracle
    big = _problem(2, 14, 3.0, 0.1, 3, 1, 0, 11)
    small = _problem(2, 6, 2.5, 0.15, 3, 1, 1, 12)
    plan = nl.Plan([big[1:], small[1:]], precision=prec)
    plan.execute()
    plan.sync()
    mesh, _, _, d, e, L, Lm, kern = small
    off, pl = O.pairs(mesh, d, e)
    rp, col = O.csr(mesh, off, pl)
    vals, _ = O.assemble(mesh, off, pl, rp, col, d, e, L, Lm, kern)
    assert _rel(plan.export(1), vals) < TOL[prec]


def test_autotuned_graph_plan_repeats_and_feeds_the_solver():
    probs = [_problem(*spec) for spec in MIX2]
    spec = [(m, p, d, e, L, Lm, k) for (_, m, p, d, e, L, Lm, k) in probs]
    plain = nl.Plan(spec, precision=nl.NL_PREC_FP32)
    plain.execute()
    plain.sync()
    plan = nl.Plan(spec, precision=nl.NL_PREC_FP32, flags=nl.NL_PLAN_AUTOTUNE | nl.NL_PLAN_GRAPH)
    sh = plan.shape()
    assert sh["graph"] and sh["warps"] in (2, 4, 8) and sh["chunk"] in (8, 32, 128) and sh["tuned_ms"] > 0
    for rep in range(3):
        plan.execute()
        st = plan.sync()
        for k in range(len(spec)):
            assert _rel(plan.export(k), plain.export(k)) < TOL[nl.NL_PREC_FP32], (rep, k)
        assert st[0].ms_assemble > 0
    # problem 0's matrix through the right-hand side and the solver equals the direct path's
    mesh, m, p, d, e, L, Lm, kern = probs[0]
    A_plan = plan.matrix(0)
    A_ref, _ = nl.nl_assemble(m, p, d, e, L, Lm, kern, nl.NL_PREC_FP32)
    g = (mesh.coords ** 2).sum(axis=0)
    outs = []
    for A in (A_plan, A_ref):
        rhs = nl.nl_rhs(m, A, g, f_const=-2.0 * mesh.dim)
        u, it, rr, status = nl.nl_solve(A, rhs, g, solver=1, rtol=1e-11, precision=nl.NL_PREC_FP32)
        outs.append(u)
    assert np.abs(outs[0] - outs[1]).max() <= 1e-6 * np.abs(outs[1]).max()


def test_plan_rejects_bad_batches():
    a = _problem(2, 6, 2.0, 0.1, 2, 1, 0, 1)
    b = _problem(3, 2, 2.0, 0.1, 2, 1, 0, 2)
    with pytest.raises(nl.NLError) as e:
        nl.Plan([a[1:], b[1:]])
    assert e.value.status == nl.NL_EINVAL
    _, m, p, d, e_, L, Lm, k = a
    with pytest.raises(nl.NLError) as e:
        nl.Plan([(m, p, d * 1.01, e_, L, Lm, k)])  # delta differs from the pairs'
    assert e.value.status == nl.NL_EINVAL
    with pytest.raises(nl.NLError) as e:
        nl.Plan([(m, p, d, e_, 0, 1, k)])  # L_max < L_min
    assert e.value.status == nl.NL_EINVAL
