"""The oracle's brute-force element-pair search (eq. k_l with eq. mindist: every l tested
for every m) spread over the host's cores, for parity checks at the workloads' full sizes.

The oracle itself stays single-threaded and literal: the inner elements m are cut into
contiguous ranges, each range is searched by one spawned process through the oracle's
``m_mask`` argument, and the lists are concatenated in m order, which is the order the
oracle produces for the whole mesh.  Processes are spawned (never forked), so a pool started
after the test process has used the GPU does not inherit its CUDA state.

Test infrastructure: only tests/ import this module.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from types import SimpleNamespace

import numpy as np


def _pairs_range(args):
    dim, coords, conn, delta, eps, m0, m1, keep = args
    import oracle as O
    mesh = SimpleNamespace(dim=dim, coords=coords, conn=conn,
                           elem_in_omega=np.ones(conn.shape[0], np.uint8),
                           node_free=np.ones(coords.shape[1], np.uint8))
    mask = np.zeros(conn.shape[0], np.uint8)
    mask[m0:m1] = 1 if keep is None else keep
    off, pl = O.pairs(mesh, delta, eps, m_mask=mask)
    return m0, np.diff(off[m0:m1 + 1]), pl


def cores() -> int:
    return max(1, os.cpu_count() or 1)


def pairs(mesh, delta: float, eps: float, m_mask=None, procs: int | None = None):
    """(pair_off, pair_l) of the oracle for the whole mesh, or for the selected inner
    elements m when m_mask is given (the other lists are empty), computed on all cores."""
    n = mesh.n_elem
    sel = np.arange(n) if m_mask is None else np.flatnonzero(np.asarray(m_mask))
    procs = procs or cores()
    # contiguous ranges of m holding about the same number of selected elements
    nchunks = max(1, min(len(sel), 4 * procs))
    bounds = []
    for part in np.array_split(sel, nchunks):
        if len(part):
            bounds.append((int(part[0]), int(part[-1]) + 1))
    coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    masked = None if m_mask is None else np.asarray(m_mask).astype(np.uint8)
    tasks = [(mesh.dim, coords, conn, delta, eps, a, b, None if masked is None else masked[a:b])
             for a, b in bounds]
    counts = np.zeros(n, np.int64)
    segs = {}
    # a worker that fails to start raises BrokenProcessPool here instead of being restarted
    with ProcessPoolExecutor(max_workers=min(procs, len(tasks)),
                             mp_context=mp.get_context("spawn")) as pool:
        for m0, cnt, pl in pool.map(_pairs_range, tasks):
            counts[m0:m0 + len(cnt)] = cnt
            segs[m0] = pl
    off = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    pl = np.concatenate([segs[k] for k in sorted(segs)]) if segs else np.zeros(0, np.int32)
    return off, pl.astype(np.int32, copy=False)
