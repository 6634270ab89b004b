"""Parity at the full workload sizes, in the launch configuration the benchmark times: the
whole matrix is assembled on the GPU, and sampled rows are compared with the oracle, which
assembles only the inner elements around the sampled nodes (a row i receives contributions
only from the elements m that contain node i, so masking in exactly those elements gives the
complete row).  Sampled nodes: seeded, one inside Omega, one on its boundary, one in the
layer, one at the outer corner of the layer.

Tolerances as in test_gpu_parity: 1e-12 relative (FP64), 2e-6 relative (FP32) per row; the
row's column list must be identical."""
import numpy as np
import pytest

import oracle as O
from nl_inputs import WORKLOADS, workload_mesh
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu

TOL = {nl.NL_PREC_FP64: 1e-12, nl.NL_PREC_FP32: 2e-6}

CASES = [
    ("c2_2d", nl.NL_PREC_FP32), ("c2_2d", nl.NL_PREC_FP64), ("c2_2d_eps20", nl.NL_PREC_FP32),
    ("c2_2d_gauss", nl.NL_PREC_FP32), ("c3_3d", nl.NL_PREC_FP32), ("c4_3d", nl.NL_PREC_FP32),
]


def _sample_nodes(mesh, w, seed, n_3d):
    rng = np.random.default_rng(seed)
    x = mesh.coords
    lo = np.array(w.lo)
    hi = lo + np.array(w.cells) * w.h
    inside = np.all((x > lo[:, None] + 1e-9) & (x < hi[:, None] - 1e-9), axis=0)
    on_bd = np.all((x >= lo[:, None] - 1e-9) & (x <= hi[:, None] + 1e-9), axis=0) & ~inside
    layer = ~np.all((x >= lo[:, None] - 1e-9) & (x <= hi[:, None] + 1e-9), axis=0)
    corner = int(np.argmin(x.sum(axis=0)))
    nodes = [int(rng.choice(np.flatnonzero(inside))), int(rng.choice(np.flatnonzero(on_bd))),
             int(rng.choice(np.flatnonzero(layer))), corner]
    return nodes[:n_3d] if mesh.dim == 3 else nodes


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{'fp64' if c[1] == nl.NL_PREC_FP64 else 'fp32'}" for c in CASES])
def test_full_size_sampled_rows(case):
    name, prec = case
    w = WORKLOADS[name]
    mesh = workload_mesh(w)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    A, st = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, prec)
    vals = A.export()
    n_pairs, nnz = p.info()
    _, _, rp, col = p.export(mesh.n_elem, mesh.n_vert)
    nodes = _sample_nodes(mesh, w, seed=7, n_3d=2)
    mask = np.zeros(mesh.n_elem, np.uint8)
    for i in nodes:
        mask[np.any(mesh.conn == i, axis=1)] = 1
    ooff, opl = O.pairs(mesh, w.delta, w.eps, m_mask=mask)
    orp, ocol = O.csr(mesh, ooff, opl)
    ovals, _ = O.assemble(mesh, ooff, opl, orp, ocol, w.delta, w.eps, w.L_max, w.L_min, w.kernel,
                          m_mask=mask)
    # the masked pair lists equal the GPU's for the masked elements
    goff, gpl = p.export(mesh.n_elem, mesh.n_vert)[:2]
    for mm in np.flatnonzero(mask)[:8]:
        assert np.array_equal(gpl[goff[mm]:goff[mm + 1]], opl[ooff[mm]:ooff[mm + 1]])
    for i in nodes:
        g_cols, o_cols = col[rp[i]:rp[i + 1]], ocol[orp[i]:orp[i + 1]]
        assert np.array_equal(g_cols, o_cols), (name, i)
        g_row, o_row = vals[rp[i]:rp[i + 1]], ovals[orp[i]:orp[i + 1]]
        rel = np.linalg.norm(g_row - o_row) / np.linalg.norm(o_row)
        assert rel < TOL[prec], (name, i, rel)
