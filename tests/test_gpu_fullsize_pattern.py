"""Element-pair lists and CSR pattern at the workloads' full sizes, bit for bit against the
oracle's brute-force search (eq. k_l with eq. mindist, every l tested for every m; run on all
host cores by tests/oracle_pool.py).

The GPU search screens candidates in FP32 with a margin that grows with the largest
coordinate and the reach, and re-tests in FP64 only inside that margin: the full-size meshes
are where a margin too small would show.  Checked here:

* 2D at h = 1/256 (eps = delta/5 and delta/20) and 3D at h = 1/16: the complete pair_off,
  pair_l, row_ptr and col arrays;
* 3D at h = 1/32 (1.41e9 pairs): the complete lists of a seeded 5% of the inner elements and
  of every element around 16 seeded nodes, and the complete rows of those nodes; for the
  whole mesh, the GPU pattern equals the set unions of the GPU's own (sample-checked) pair
  lists at 64 more nodes, and every element occurs as often as l as it has pairs as m
  (the relation is symmetric).
"""
import numpy as np
import pytest

import oracle as O
import oracle_pool
from nl_inputs import WORKLOADS, workload_mesh
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["c2_2d", "c2_2d_eps20", "c3_3d"])
def test_full_pair_lists_and_pattern_bit_exact(name):
    w = WORKLOADS[name]
    mesh = workload_mesh(w)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    goff, gpl, grp, gcol = p.export(mesh.n_elem, mesh.n_vert)
    ooff, opl = oracle_pool.pairs(mesh, w.delta, w.eps)
    assert np.array_equal(goff, ooff), name
    assert np.array_equal(gpl, opl), name
    orp, ocol = O.csr(mesh, ooff, opl)
    assert np.array_equal(grp, orp), name
    assert np.array_equal(gcol, ocol), name


def test_c4_sampled_lists_and_rows_bit_exact():
    w = WORKLOADS["c4_3d"]
    mesh = workload_mesh(w)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    goff, gpl, grp, gcol = p.export(mesh.n_elem, mesh.n_vert)
    assert goff[-1] == len(gpl) == 1_414_944_000
    rng = np.random.default_rng(2024)
    mask = (rng.random(mesh.n_elem) < 0.05).astype(np.uint8)
    nodes = rng.choice(mesh.n_vert, size=16, replace=False)
    around = np.isin(mesh.conn, nodes).any(axis=1)
    mask[around] = 1
    ooff, opl = oracle_pool.pairs(mesh, w.delta, w.eps, m_mask=mask)
    sel = np.flatnonzero(mask)
    glen = goff[sel + 1] - goff[sel]
    olen = ooff[sel + 1] - ooff[sel]
    assert np.array_equal(glen, olen)
    gidx = np.concatenate([np.arange(goff[e], goff[e + 1]) for e in sel])
    assert np.array_equal(gpl[gidx], opl)
    # complete rows of the sampled nodes: the oracle's pattern over the masked elements holds
    # every column of a row whose elements are all masked
    orp, ocol = O.csr(mesh, ooff, opl)
    for i in nodes:
        assert np.array_equal(gcol[grp[i]:grp[i + 1]], ocol[orp[i]:orp[i + 1]]), i
    # whole mesh: the pair relation is symmetric (eq. mindist is symmetric in the two boxes),
    # so every element appears as often as l as it has pairs as m ...
    assert np.array_equal(np.bincount(gpl, minlength=mesh.n_elem), np.diff(goff))
    # ... and every row of the pattern at 64 more seeded nodes is the union of the nodes of
    # l over the GPU's own pair lists of the elements around the node
    for i in rng.choice(mesh.n_vert, size=64, replace=False):
        cols = set()
        for e in np.flatnonzero((mesh.conn == i).any(axis=1)):
            cols.update(mesh.conn[gpl[goff[e]:goff[e + 1]]].ravel().tolist())
        assert np.array_equal(gcol[grp[i]:grp[i + 1]], np.array(sorted(cols), np.int32)), i
