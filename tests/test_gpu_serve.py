"""Serving loop: requests admitted by memory and slots, run concurrently (small ones batched
into one plan launch with others), and each result equal to the same request run alone, and to
the oracle.

Alone vs in the mix: FP64 requests agree to the solver's tolerance (u to 1e-9 relative, the
L2 error to 1e-6); FP32 requests may be assembled in a batched plan in the mix, whose work
counter regroups the FP32 sums of the assembly (the matrices differ at the 1e-7 level), so u
agrees to 1e-6 and the L2 error to 1e-4."""
import numpy as np
import pytest

from nl_inputs import structured_mesh
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu


def _req(dim, n, delta_h, kernel, prec, u=None, seed=0):
    h = 1.0 / n
    delta = delta_h * h
    eps = delta / 10
    layer = int(np.ceil((delta + eps) / h - 1e-9))
    return nl.make_request(dim, (n,) * dim, h, (0.0,) * dim, layer, delta, eps,
                           3 if dim == 2 else 2, kernel=kernel, precision=prec, ms=1, solver=1,
                           rtol=1e-11, jitter=0.1, seed=seed, u_out=u)


MIX = [(2, 24, 3.0, 0, nl.NL_PREC_FP32), (3, 6, 2.5, 1, nl.NL_PREC_FP32),
       (2, 40, 4.0, 1, nl.NL_PREC_FP64), (2, 16, 2.0, 0, nl.NL_PREC_FP32),
       (3, 5, 2.0, 0, nl.NL_PREC_FP64), (2, 32, 5.0, 0, nl.NL_PREC_FP32)]


def _nvert(dim, n, delta_h):
    layer = int(np.ceil(1.1 * delta_h - 1e-9))
    return (n + 2 * layer + 1) ** dim


def test_results_alone_equal_results_in_the_mix():
    alone = []
    with nl.Server(8 << 30, 1) as S:
        for (dim, n, dh, k, prec) in MIX:
            u = np.zeros(_nvert(dim, n, dh))
            r = S.wait(S.submit(_req(dim, n, dh, k, prec, u), u))
            assert r.status == nl.NL_OK, r.message
            alone.append((u, r))
    for rep in range(2):  # two rounds of concurrent requests on fresh workers
        with nl.Server(8 << 30, 4) as S:
            outs = [np.zeros(_nvert(d, n, dh)) for (d, n, dh, k, p) in MIX]
            tickets = [S.submit(_req(*spec, u=u), u) for spec, u in zip(MIX, outs)]
            res = [S.wait(t) for t in tickets]
            starts = sorted(r.t_start_ms for r in res)
            dones = sorted(r.t_done_ms for r in res)
            assert starts[1] < dones[0], "requests did not overlap"
            for (u0, r0), u1, r1, spec in zip(alone, outs, res, MIX):
                assert r1.status == nl.NL_OK, (rep, r1.message)
                assert r1.n_pairs == r0.n_pairs and r1.n_point_pairs == r0.n_point_pairs
                tu, te = (1e-9, 1e-6) if spec[4] == nl.NL_PREC_FP64 else (1e-6, 1e-4)
                assert np.abs(u1 - u0).max() <= tu * np.abs(u0).max(), (spec, r1.group)
                assert abs(r1.l2_err_omega / r0.l2_err_omega - 1) < te, (spec, r1.group)
            p50, p99, sps = S.stats()
            assert 0 < p50 <= p99 and sps > 0


def test_admission_by_memory_budget_serialises_large_requests():
    # a budget below two requests' footprint: the second waits for the first to finish
    with nl.Server(64 << 20, 4) as S:
        t = [S.submit(_req(2, 64, 4.0, 0, nl.NL_PREC_FP32)) for _ in range(3)]
        res = [S.wait(x) for x in t]
        assert all(r.status == nl.NL_OK for r in res)
        res.sort(key=lambda r: r.t_start_ms)
        for a, b in zip(res, res[1:]):
            assert b.t_start_ms >= a.t_done_ms - 1e-3


def test_poll_wait_timeout_and_bad_ticket():
    with nl.Server(1 << 30, 1) as S:
        t = S.submit(_req(2, 48, 4.0, 0, nl.NL_PREC_FP64))
        with pytest.raises(nl.NLError) as e:
            S.wait(t, timeout_ms=0.01)
        assert e.value.status == nl.NL_ETIMEOUT
        r = S.wait(t)
        assert r.status == nl.NL_OK and r.l2_err_omega > 0
        with pytest.raises(nl.NLError) as e:
            S.poll(t)  # a result is taken once
        assert e.value.status == nl.NL_EINVAL


# Served results against the oracle's dense solve of the same problem (pairs, pattern,
# Algorithm 1, right-hand side with lifting and Gaussian elimination, all in FP64 on the CPU),
# at the tolerances of the single-problem solver tests: u_h to 1e-9 (FP64 assembly) or 1e-5
# (FP32 assembly) of max |u_h|, the L2 error over Omega to 1e-8 or 1e-3 relative.
# (The 3D meshes are small, delta = 0.8h, because the oracle's 3D assembly is slow.)
ORACLE_MIX = [(2, 16, 3.0, 0, nl.NL_PREC_FP64, 21), (2, 12, 2.5, 1, nl.NL_PREC_FP32, 22),
              (3, 4, 0.8, 0, nl.NL_PREC_FP32, 23), (3, 3, 0.8, 1, nl.NL_PREC_FP64, 24)]


def test_served_results_match_the_oracle():
    import oracle as O
    with nl.Server(8 << 30, 4) as S:
        outs, tickets, specs = [], [], []
        for (dim, n, dh, kern, prec, seed) in ORACLE_MIX:
            u = np.zeros(_nvert(dim, n, dh))
            tickets.append(S.submit(_req(dim, n, dh, kern, prec, u, seed=seed), u))
            outs.append(u)
        res = [S.wait(t) for t in tickets]
    for (dim, n, dh, kern, prec, seed), u, r in zip(ORACLE_MIX, outs, res):
        assert r.status == nl.NL_OK, r.message
        h = 1.0 / n
        delta = dh * h
        eps = delta / 10
        layer = int(np.ceil((delta + eps) / h - 1e-9))
        mesh = structured_mesh(dim, n, h, 0.0, layer, jitter=0.1, seed=seed)
        ref = O.solve_problem(mesh, delta, eps, 3 if dim == 2 else 2, 1, kernel=kern)
        assert r.n_pairs == len(ref["pair_l"]) and r.nnz == len(ref["col"])
        assert r.n_point_pairs == ref["stats"].n_point_pairs
        tolu, tole = (1e-9, 1e-8) if prec == nl.NL_PREC_FP64 else (1e-5, 1e-3)
        assert np.abs(u - ref["u_h"]).max() <= tolu * np.abs(ref["u_h"]).max(), (dim, n, prec)
        assert abs(r.l2_err_omega / ref["err_omega"] - 1) < tole, (dim, n, prec)


def test_small_requests_share_one_launch():
    # 12 small 2D requests submitted at once to a one-slot server: the first is admitted alone
    # (nothing else is waiting yet, or a group starts), the rest that wait are batched into
    # plans; every grouped result matches the oracle-checked single path to the FP32
    # tolerance, and results of one group share its id
    specs = [(2, 8 + (i % 4) * 2, 2.0 + (i % 3), i % 2, nl.NL_PREC_FP32) for i in range(12)]
    alone = []
    with nl.Server(4 << 30, 1) as S:
        for sp in specs:
            u = np.zeros(_nvert(*sp[:3]))
            r = S.wait(S.submit(_req(*sp, u=u), u))
            assert r.status == nl.NL_OK and r.group == -1
            alone.append((u, r))
    with nl.Server(4 << 30, 1) as S:
        outs = [np.zeros(_nvert(*sp[:3])) for sp in specs]
        tickets = [S.submit(_req(*sp, u=u), u) for sp, u in zip(specs, outs)]
        res = [S.wait(t) for t in tickets]
    groups = [r.group for r in res]
    assert sum(g >= 0 for g in groups) >= 8, groups
    for (u0, r0), u1, r1 in zip(alone, outs, res):
        assert r1.status == nl.NL_OK, r1.message
        assert r1.n_pairs == r0.n_pairs and r1.n_point_pairs == r0.n_point_pairs
        assert np.abs(u1 - u0).max() <= 1e-6 * np.abs(u0).max(), r1.group
