"""The FP32 screen of Algorithm 1's decisions in the FP32 assembly path (CPU, numpy float32
emulation): sub-element vertices relative to the first vertex of E_m (the FP64 offset of the
first vertices rebuilt from float-float pairs, per-element FP32 vertex offsets, FP32
midpoints), box distances of Sec. 5.1 (eqs. maxdist, mindist, and the Euclidean minimum
distance stated after eq. mindistin) in FP32, compared against delta -/+ eps with the margin
2e-5 (delta + eps + 2 max_ext) (twice that for the Euclidean distance).  Every decision the screen
takes must equal the FP64 decision on the exact sub-element, at every refinement level up
to 12, on the workloads' meshes and on a mesh far from the origin; likewise for the
quadrilaterals and hexahedra (sub-squares and sub-cubes on the lattice of half steps, to
level 10), on the 2D grids, the 3D workload's grid and Table 6's grid.  The closed forms of
FINAL items (simplices, Q1 quadrilaterals) are taken only where every point pair clears
delta - eps or delta + eps by half a margin."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from nl_inputs import structured_mesh

f32 = np.float32


def _children(dim):
    if dim == 2:
        # (v0, m01, m02), (m01, v1, m12), (m02, m12, v2), (m01, m12, m02); points 3.. = midpoints
        # m01, m02, m12
        return [(0, 3, 4), (3, 1, 5), (4, 5, 2), (3, 5, 4)], [(0, 1), (0, 2), (1, 2)]
    # Bey: x0..x3, then x01, x02, x03, x12, x13, x23 as points 4..9
    return ([(0, 4, 5, 6), (4, 1, 7, 8), (5, 7, 2, 9), (6, 8, 9, 3), (4, 5, 6, 8), (4, 5, 7, 8),
             (5, 6, 8, 9), (5, 7, 8, 9)], [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])


def _refine(V, c, dim, dtype):
    kids, mids = _children(dim)
    half = dtype(0.5)
    pts = [V[:, a, :] for a in range(dim + 1)]
    pts += [((V[:, i, :] + V[:, j, :]) * half).astype(dtype) for i, j in mids]
    P = np.stack(pts, axis=1)
    sel = np.array(kids)[c]  # (n, dim+1)
    return np.take_along_axis(P, sel[:, :, None].repeat(dim, axis=2), axis=1)


def _dists(V, lo2, hi2, dtype):
    lo, hi = V.min(axis=1), V.max(axis=1)
    d1 = (lo - hi2).astype(dtype)
    d2 = (lo2 - hi).astype(dtype)
    sq = np.maximum(d1 * d1, d2 * d2).astype(dtype)
    s = np.zeros(len(V), dtype)
    for k in range(V.shape[2]):
        s = (s + sq[:, k]).astype(dtype)
    t = np.maximum(np.maximum(d1, d2), dtype(0))
    amin = t.max(axis=1)
    # squared Euclidean min-dist (the variant after eq. mindistin), accumulated as the kernel's
    # fused multiply-adds: the product of two FP32 values is exact in FP64, one rounding per add
    e = np.zeros(len(V), dtype)
    for k in range(V.shape[2]):
        tk = t[:, k].astype(np.float64)
        e = (e.astype(np.float64) + tk * tk).astype(dtype)
    return s, amin, e  # squared max-dist, min-dist, squared Euclidean min-dist


@pytest.mark.parametrize("dim,cells,h,lo,delta,eps,jitter", [
    (2, 256, 1 / 256, (0.0, 0.0), 4 / 256, 4 / 256 / 5, 0.1),
    (2, 64, 1 / 64, (1000.0, -350.0), 4 / 64, 4 / 64 / 20, 0.1),
    (3, 16, 1 / 16, (0.0, 0.0, 0.0), 0.125, 0.0125, 0.1),
])
def test_fp32_screen_decisions_equal_fp64(dim, cells, h, lo, delta, eps, jitter):
    layer = int(np.ceil((delta + eps) / h - 1e-9))
    mesh = structured_mesh(dim, (cells,) * dim, h, lo, layer, jitter=jitter, seed=3)
    X = mesh.coords.T  # (n_vert, dim)
    EV = X[mesh.conn]  # (n_elem, dim+1, dim) FP64
    rng = np.random.default_rng(5)
    max_ext = float((EV.max(axis=1) - EV.min(axis=1)).max())
    cen = EV.mean(axis=1)
    tree = cKDTree(cen)
    n = 4000
    ms = rng.integers(0, mesh.n_elem, n)
    near = tree.query_ball_point(cen[ms], delta + eps + 2 * max_ext)
    ls = np.array([rng.choice(c) for c in near])
    # per-element FP32 record: vertex offsets and the first vertex as a float-float pair
    off = (EV[:, 1:, :] - EV[:, :1, :]).astype(f32)
    v0 = EV[:, 0, :]
    v0h = v0.astype(f32)
    v0l = (v0 - v0h.astype(np.float64)).astype(f32)
    # E_m relative to its first vertex, and its FP64 box
    Vm32 = np.concatenate([np.zeros((n, 1, dim), f32), off[ms]], axis=1)
    lo_m32, hi_m32 = Vm32.min(axis=1), Vm32.max(axis=1)
    lo_m64, hi_m64 = EV[ms].min(axis=1), EV[ms].max(axis=1)
    # E_l relative to m's first vertex: (hi_l - hi_m) + (lo_l - lo_m), then the offsets
    Vl0 = ((v0h[ls] - v0h[ms]).astype(f32) + (v0l[ls] - v0l[ms]).astype(f32)).astype(f32)
    V32 = np.concatenate([Vl0[:, None, :], (Vl0[:, None, :] + off[ls]).astype(f32)], axis=1)
    V64 = EV[ls].copy()
    dme, dpe = delta - eps, delta + eps
    margin = f32(2e-5 * (delta + eps + 2.0 * max_ext))
    fdme, fdpe = f32(dme), f32(dpe)
    lo_t, hi_t = float(fdme) - float(margin), float(fdme) + float(margin)
    fint2 = f32(lo_t * lo_t) if lo_t > 0 else f32(-1)
    fnotint2 = f32(hi_t * hi_t)
    decided = checked = 0
    for level in range(1, 13):
        if level > 1:
            c = rng.integers(0, 2 ** dim, n)
            V32 = _refine(V32, c, dim, f32)
            V64 = _refine(V64, c, dim, np.float64)
        fam, fan, fe2 = _dists(V32, lo_m32, hi_m32, f32)
        s64, amin64, e64 = _dists(V64, lo_m64, hi_m64, np.float64)
        amax64, aminl2 = np.sqrt(s64), np.sqrt(e64)
        is_int, is_ref = amax64 < dme, amin64 < dpe
        c_int, c_notint = fam < fint2, fam > fnotint2
        c_ref, c_out = fan < f32(fdpe - margin), fan > f32(fdpe + margin)
        assert np.all(is_int[c_int]) and not np.any(is_int[c_notint]), level
        assert np.all(is_ref[c_ref]) and not np.any(is_ref[c_out]), level
        # the Euclidean refinement test (NL_QUAD_MINDIST_L2) against (delta + eps -+ 2 margin)^2
        fref2 = f32((float(fdpe) - 2.0 * float(margin)) ** 2)
        fout2 = f32((float(fdpe) + 2.0 * float(margin)) ** 2)
        is_ref2 = aminl2 < dpe
        c_ref2, c_out2 = fe2 < fref2, fe2 > fout2
        assert np.all(is_ref2[c_ref2]) and not np.any(is_ref2[c_out2]), level
        decided += int((c_int | c_notint).sum() + (c_ref | c_out).sum())
        # adversarial thresholds placed at each sub-element's own distances: within a few
        # margins (the screen's window edges) and within FP32 precision (where only the
        # FP64 test may decide)
        for scale in (float(margin), 2.0 ** -20 * (delta + eps)):
            for dist, kind in ((amax64, "max"), (amin64, "min"), (aminl2, "l2")):
                T = dist + rng.uniform(-3, 3, n) * scale
                fT = T.astype(f32)
                exact = dist < T
                if kind == "max":
                    lo_t = fT.astype(np.float64) - float(margin)
                    t2 = np.where(lo_t > 0, (lo_t * lo_t), -1.0).astype(f32)
                    hi2 = ((fT.astype(np.float64) + float(margin)) ** 2).astype(f32)
                    yes, no = fam < t2, fam > hi2
                elif kind == "l2":
                    lo_t = fT.astype(np.float64) - 2.0 * float(margin)
                    t2 = np.where(lo_t > 0, (lo_t * lo_t), -1.0).astype(f32)
                    hi2 = ((fT.astype(np.float64) + 2.0 * float(margin)) ** 2).astype(f32)
                    yes, no = fe2 < t2, fe2 > hi2
                else:
                    yes, no = fan < (fT - margin).astype(f32), fan > (fT + margin).astype(f32)
                assert np.all(exact[yes]) and not np.any(exact[no]), (level, scale, kind)
                checked += int((yes | no).sum())
    assert decided > 0.9 * 2 * 12 * n  # the FP64 fallback is rare
    assert checked > 0


@pytest.mark.parametrize("eps_div", [5, 20])
def test_closed_form_final_items_have_mu_exactly_0_or_1(eps_div):
    # 2D FINAL sub-elements taken in closed form: every inner point y of m with
    # |c - y| < delta - eps - R - margin (or > delta + eps + R + margin), c the centroid and
    # R = rad(E_l) 2^(1-L) (midpoint children are the parent scaled by 1/2), must have all of
    # the sub-element's quadrature points x within delta - eps (beyond delta + eps) by a
    # clear gap, so that the FP32 mollifier clamps to exactly 1 (0) at every point pair.
    import oracle as O
    delta = 4 / 256
    eps = delta / eps_div
    layer = int(np.ceil((delta + eps) * 256 - 1e-9))
    mesh = structured_mesh(2, (256, 256), 1 / 256, (0.0, 0.0), layer, jitter=0.1, seed=4)
    EV = mesh.coords.T[mesh.conn]
    rng = np.random.default_rng(9)
    max_ext = float((EV.max(axis=1) - EV.min(axis=1)).max())
    cen_e = EV.mean(axis=1)
    tree = cKDTree(cen_e)
    n = 3000
    ms = rng.integers(0, mesh.n_elem, n)
    ls = np.array([rng.choice(c) for c in tree.query_ball_point(cen_e[ms], delta + eps + 2 * max_ext)])
    b, _ = O.quad_rule(2)
    bf = b.astype(f32)
    off = (EV[:, 1:, :] - EV[:, :1, :]).astype(f32)
    v0 = EV[:, 0, :]
    v0h = v0.astype(f32)
    v0l = (v0 - v0h.astype(np.float64)).astype(f32)
    Vm = np.concatenate([np.zeros((n, 1, 2), f32), off[ms]], axis=1)
    Y = np.einsum("qa,nak->nqk", bf, Vm).astype(f32)  # inner points of m (FP32, relative)
    Vl0 = ((v0h[ls] - v0h[ms]).astype(f32) + (v0l[ls] - v0l[ms]).astype(f32)).astype(f32)
    V = np.concatenate([Vl0[:, None, :], (Vl0[:, None, :] + off[ls]).astype(f32)], axis=1)
    ct = (V.sum(axis=1) * f32(1 / 3)).astype(f32)
    rad_l = np.sqrt((((V - ct[:, None, :]) ** 2).sum(-1)).max(axis=1)).astype(f32)
    margin = f32(2e-5 * (delta + eps + 2.0 * max_ext))
    dme, dpe = f32(delta - eps), f32(delta + eps)
    n_in = n_out = 0
    for level in range(1, 5):
        if level > 1:
            V = _refine(V, rng.integers(0, 4, n), 2, f32)
        cen = (V.sum(axis=1) * f32(1 / 3)).astype(f32)
        rad = (rad_l * f32(2.0 ** (1 - level))).astype(f32)
        lo = (dme - rad - margin).astype(f32)
        hi = (dpe + rad + margin).astype(f32)
        lo2 = np.where(lo > 0, lo * lo, f32(-1)).astype(f32)
        hi2 = (hi * hi).astype(f32)
        d2 = (((cen[:, None, :] - Y) ** 2).sum(-1)).astype(f32)  # (n, 7)
        inside, outside = d2 < lo2[:, None], d2 > hi2[:, None]
        X = np.einsum("qa,nak->nqk", bf, V).astype(f32)  # outer points of the sub-element
        r = np.sqrt(((X[:, :, None, :].astype(np.float64) - Y[:, None, :, :]) ** 2).sum(-1))
        gap = 0.5 * float(margin)
        assert np.all(r.max(axis=1)[inside] < float(dme) - gap), level
        assert np.all(r.min(axis=1)[outside] > float(dpe) + gap), level
        n_in += int(inside.sum())
        n_out += int(outside.sum())
    assert n_in > 0 and n_out > 0



def _tensor_child(V, c, dim, dtype):
    """Children of quadrilaterals (dim 2: vertices (0,0), (1,0), (1,1), (0,1); child c = 0..3
    the sub-squares (0,0), (1,0), (1,1), (0,1)) and hexahedra (dim 3: the Q1 vertex order,
    child c with bits (x, y, z)), their vertices on the lattice of half steps: a lattice point
    with a middle index is the midpoint of its two neighbours along the first such axis (x,
    then y, then z); the quadrilateral's centre is the midpoint of the midpoints of its edges
    (0,1) and (2,3)."""
    half = dtype(0.5)

    def mid(a, b):
        return ((a + b) * half).astype(dtype)
    n = len(V)
    idx = np.arange(n)
    if dim == 2:
        P = [V[:, a, :] for a in range(4)]
        m01, m12, m23, m30 = mid(P[0], P[1]), mid(P[1], P[2]), mid(P[2], P[3]), mid(P[3], P[0])
        ce = mid(m01, m23)
        kids = np.stack([np.stack([P[0], m01, ce, m30], 1), np.stack([m01, P[1], m12, ce], 1),
                         np.stack([ce, m12, P[2], m23], 1), np.stack([m30, ce, m23, P[3]], 1)], 1)
        return kids[idx, c]
    corner = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    L = {}
    for a, (i, j, k) in enumerate(corner):
        L[(2 * i, 2 * j, 2 * k)] = V[:, a, :]
    for i in (0, 2):
        for j in (0, 2):
            L[(i, j, 1)] = mid(L[(i, j, 0)], L[(i, j, 2)])
        for k in range(3):
            L[(i, 1, k)] = mid(L[(i, 0, k)], L[(i, 2, k)])
    for j in range(3):
        for k in range(3):
            L[(1, j, k)] = mid(L[(0, j, k)], L[(2, j, k)])
    kids = np.stack([np.stack([L[(cx + i, cy + j, cz + k)] for i, j, k in corner], 1)
                     for cx, cy, cz in [(q & 1, (q >> 1) & 1, (q >> 2) & 1) for q in range(8)]], 1)
    return kids[idx, c]


@pytest.mark.parametrize("dim,cells,h,lo,delta,eps", [
    (2, 128, 1 / 128, (0.0, 0.0), 4 / 128, 4 / 128 / 5),
    (2, 64, 1 / 64, (1000.0, -350.0), 4 / 64, 4 / 64 / 20),
    (3, 16, 1 / 16, (0.0, 0.0, 0.0), 0.125, 0.0125),
    (3, 12, 0.1, (-0.6, -0.4, -0.4), 0.2, 0.0125),
])
def test_fp32_screen_of_quadrilaterals_and_hexahedra(dim, cells, h, lo, delta, eps):
    # the same screen on the tensor-product elements: the FP32 record holds the vertex offsets
    # and the float-float first vertex; sub-elements come from the lattice midpoints in FP32
    # (the kernels' child rule) and are compared with the FP64 ones built the same way
    from nl_inputs import hex_mesh, quad_mesh
    layer = int(np.ceil((delta + eps) / h - 1e-9))
    base = structured_mesh(dim, (cells,) * dim, h, lo, layer, jitter=0.1, seed=4)
    mesh = quad_mesh(base) if dim == 2 else hex_mesh(base)
    nv = 4 if dim == 2 else 8
    X = mesh.coords.T
    EV = X[mesh.conn[:, :nv]]  # (n_elem, nv, dim)
    rng = np.random.default_rng(6)
    max_ext = float((EV.max(axis=1) - EV.min(axis=1)).max())
    cen = EV.mean(axis=1)
    tree = cKDTree(cen)
    n = 3000
    ms = rng.integers(0, mesh.n_elem, n)
    near = tree.query_ball_point(cen[ms], delta + eps + 2 * max_ext)
    ls = np.array([rng.choice(c) for c in near])
    off = (EV[:, 1:, :] - EV[:, :1, :]).astype(f32)
    v0 = EV[:, 0, :]
    v0h = v0.astype(f32)
    v0l = (v0 - v0h.astype(np.float64)).astype(f32)
    Vm32 = np.concatenate([np.zeros((n, 1, dim), f32), off[ms]], axis=1)
    lo_m32, hi_m32 = Vm32.min(axis=1), Vm32.max(axis=1)
    lo_m64, hi_m64 = EV[ms].min(axis=1), EV[ms].max(axis=1)
    Vl0 = ((v0h[ls] - v0h[ms]).astype(f32) + (v0l[ls] - v0l[ms]).astype(f32)).astype(f32)
    V32 = np.concatenate([Vl0[:, None, :], (Vl0[:, None, :] + off[ls]).astype(f32)], axis=1)
    V64 = EV[ls].copy()
    dme, dpe = delta - eps, delta + eps
    margin = f32(2e-5 * (delta + eps + 2.0 * max_ext))
    fdme, fdpe = f32(dme), f32(dpe)
    lo_t, hi_t = float(fdme) - float(margin), float(fdme) + float(margin)
    fint2 = f32(lo_t * lo_t) if lo_t > 0 else f32(-1)
    fnotint2 = f32(hi_t * hi_t)
    fref2 = f32((float(fdpe) - 2.0 * float(margin)) ** 2)
    fout2 = f32((float(fdpe) + 2.0 * float(margin)) ** 2)
    decided = 0
    for level in range(1, 11):
        if level > 1:
            c = rng.integers(0, 2 ** dim, n)
            V32 = _tensor_child(V32, c, dim, f32)
            V64 = _tensor_child(V64, c, dim, np.float64)
        fam, fan, fe2 = _dists(V32, lo_m32, hi_m32, f32)
        s64, amin64, e64 = _dists(V64, lo_m64, hi_m64, np.float64)
        amax64, aminl2 = np.sqrt(s64), np.sqrt(e64)
        is_int, is_ref, is_ref2 = amax64 < dme, amin64 < dpe, aminl2 < dpe
        c_int, c_notint = fam < fint2, fam > fnotint2
        c_ref, c_out = fan < f32(fdpe - margin), fan > f32(fdpe + margin)
        c_ref2, c_out2 = fe2 < fref2, fe2 > fout2
        assert np.all(is_int[c_int]) and not np.any(is_int[c_notint]), level
        assert np.all(is_ref[c_ref]) and not np.any(is_ref[c_out]), level
        assert np.all(is_ref2[c_ref2]) and not np.any(is_ref2[c_out2]), level
        decided += int((c_int | c_notint).sum() + (c_ref | c_out).sum())
        # thresholds at the sub-elements' own distances, a few margins away
        for dist, kind in ((amax64, "max"), (amin64, "min")):
            T = dist + rng.uniform(-3, 3, n) * float(margin)
            fT = T.astype(f32)
            exact = dist < T
            if kind == "max":
                lt = fT.astype(np.float64) - float(margin)
                t2 = np.where(lt > 0, lt * lt, -1.0).astype(f32)
                yes, no = fam < t2, fam > ((fT.astype(np.float64) + float(margin)) ** 2).astype(f32)
            else:
                yes, no = fan < (fT - margin).astype(f32), fan > (fT + margin).astype(f32)
            assert np.all(exact[yes]) and not np.any(exact[no]), (level, kind)
    assert decided > 0.9 * 2 * 10 * n


@pytest.mark.parametrize("eps_div", [5, 20])
def test_closed_form_final_quadrilaterals_have_mu_exactly_0_or_1(eps_div):
    # Q1 quadrilaterals: a FINAL sub-square is taken in closed form at inner point y when
    # |c - y| < delta - eps - R - margin (or > delta + eps + R + margin), c the mean of its
    # four FP32 vertices and R = max |v - c| (the bilinear image lies in the vertices' convex
    # hull, inside that ball); every Gauss-Legendre 3x3 point x of the exact sub-square must
    # then lie within delta - eps of y (beyond delta + eps) by a clear gap
    from nl_inputs import quad_mesh
    delta = 4 / 128
    eps = delta / eps_div
    layer = int(np.ceil((delta + eps) * 128 - 1e-9))
    mesh = quad_mesh(structured_mesh(2, (128, 128), 1 / 128, (0.0, 0.0), layer, jitter=0.1, seed=4))
    EV = mesh.coords.T[mesh.conn]  # (n_elem, 4, 2)
    rng = np.random.default_rng(11)
    max_ext = float((EV.max(axis=1) - EV.min(axis=1)).max())
    cen_e = EV.mean(axis=1)
    tree = cKDTree(cen_e)
    n = 3000
    ms = rng.integers(0, mesh.n_elem, n)
    ls = np.array([rng.choice(c) for c in tree.query_ball_point(cen_e[ms], delta + eps + 2 * max_ext)])
    g = (np.polynomial.legendre.leggauss(3)[0] + 1) / 2
    S, T = np.meshgrid(g, g, indexing="ij")
    s, t = S.ravel(), T.ravel()
    N = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], 1)  # (9, 4)
    off = (EV[:, 1:, :] - EV[:, :1, :]).astype(f32)
    v0 = EV[:, 0, :]
    v0h = v0.astype(f32)
    v0l = (v0 - v0h.astype(np.float64)).astype(f32)
    # inner points of m in FP64 relative to m's first vertex, rounded to FP32
    Y = np.einsum("qa,nak->nqk", N, EV[ms] - EV[ms][:, :1, :]).astype(f32)
    Vl0 = ((v0h[ls] - v0h[ms]).astype(f32) + (v0l[ls] - v0l[ms]).astype(f32)).astype(f32)
    V = np.concatenate([Vl0[:, None, :], (Vl0[:, None, :] + off[ls]).astype(f32)], axis=1)
    V64 = EV[ls] - EV[ms][:, :1, :]  # the exact sub-square in the same frame
    margin = f32(2e-5 * (delta + eps + 2.0 * max_ext))
    dme, dpe = f32(delta - eps), f32(delta + eps)
    n_in = n_out = 0
    for level in range(1, 6):
        if level > 1:
            c = rng.integers(0, 4, n)
            V = _tensor_child(V, c, 2, f32)
            V64 = _tensor_child(V64, c, 2, np.float64)
        cen = (V.sum(axis=1) * f32(0.25)).astype(f32)
        rad = np.sqrt((((V - cen[:, None, :]) ** 2).sum(-1)).max(axis=1).astype(f32)).astype(f32)
        lo = (dme - rad - margin).astype(f32)
        hi = (dpe + rad + margin).astype(f32)
        lo2 = np.where(lo > 0, lo * lo, f32(-1)).astype(f32)
        hi2 = (hi * hi).astype(f32)
        d2 = (((cen[:, None, :] - Y) ** 2).sum(-1)).astype(f32)  # (n, 9)
        inside, outside = d2 < lo2[:, None], d2 > hi2[:, None]
        X = np.einsum("qa,nak->nqk", N, V64)  # outer points of the exact sub-square
        r = np.sqrt(((X[:, :, None, :] - Y[:, None, :, :].astype(np.float64)) ** 2).sum(-1))
        gap = 0.5 * float(margin)
        assert np.all(r.max(axis=1)[inside] < float(dme) - gap), level
        assert np.all(r.min(axis=1)[outside] > float(dpe) + gap), level
        n_in += int(inside.sum())
        n_out += int(outside.sum())
    assert n_in > 0 and n_out > 0
