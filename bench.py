#!/usr/bin/env python
"""Benchmark of the nonlocal assembly + solve hot path on one GB300 (or N replicas).

One step = the whole path on the 3D workload at h = 1/32 (Omega = (0,1)^3 with a 4-cell
layer, 384,000 Kuhn tetrahedra, delta = 3h, eps = delta/10, L_max = 2, constant kernel;
1.41e9 element pairs, 2.2e12 quad-pt pairs): element-pair search and CSR pattern,
Algorithm 1 assembly, right-hand side with lifting (u = x^2 + y^2 + z^2, f = -6) and
BiCGStab solve to 1e-10, with the mesh resident on the device.  The headline runs the FP32
point-pair path with the solve in FP32 inside FP64 iterative refinement ("mixed"); the same
step in FP64 is measured next to it with the solution error of both against the manufactured
solution and the difference of the two matrices.

Beside the headline the JSON line carries: the FP64 step, the roofline of the assembly kernel
(FP32 and FP64), the achieved bandwidth of the HBM-bound kernels (scatter, SpMV), the
public-API end-to-end rate from pinned host buffers (e2e), the 2D workload at h = 1/256 in its
four (eps, kernel) combinations (mixed and FP64 steps), an eps-convergence study (the P1
analogue of the paper's Table 4: error against cost over eps and L_max), a batching leg (128 small problems:
sequential assembly against one plan), a serving leg (the first --serve-requests requests of
the seeded stream, closed loop and then open loop at 70% load) and the oracle timed on all
host cores on a bounded sample (cpu_baseline).

Output: one JSON line (rank 0).  --impl reference times the plain CPU oracle on bounded
samples of the same workload instead.  Under torchrun every rank runs its own replica.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("element pairs/s & quad-pt pairs/s, mixed vs FP64 at equal error; "
          "p50/p99 solve ms")
WORKLOAD = "c4_3d"
C2_BLOCK = ["c2_2d", "c2_2d_eps20", "c2_2d_gauss", "c2_2d_gauss_eps20"]

# DRAM traffic of the FP32 assembly kernel per element pair: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the current kernel version on a small case of the
# same dimension (profiles/k_quad_2d_fp32_c2_h128.md, profiles/k_quad_3d_fp32_c3_h10.md)
# divided by its element pairs.  Almost all of it is the block buffer, written once per pair,
# so it scales with the pairs of a launch.  None: no capture of the current version.
TRAFFIC_BYTES_PER_PAIR = {2: 35.37, 3: 63.45}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed FP64 steps of the headline workload (0 = leave the FP64 path out)")
    ap.add_argument("--c2-steps", type=int, default=5,
                    help="timed mixed steps per combination of the 2D block (0 = skip the block)")
    ap.add_argument("--c2-fp64-steps", type=int, default=1,
                    help="timed FP64 steps per combination of the 2D block")
    ap.add_argument("--p2-steps", type=int, default=2,
                    help="timed FP32 steps of the P2 leg (the 2D workload with P2 triangles; "
                         "0 = skip the leg)")
    ap.add_argument("--p2-fp64-steps", type=int, default=1,
                    help="timed FP64 steps of the P2 leg")
    ap.add_argument("--quad-steps", type=int, default=2,
                    help="timed FP32 steps of each quadrilateral leg (Q1, Q2 on the 2D workload's "
                         "grid; 0 = skip)")
    ap.add_argument("--quad-fp64-steps", type=int, default=1,
                    help="timed FP64 steps of each quadrilateral leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="wall seconds of the oracle sample on all host cores")
    ap.add_argument("--ref-step-seconds", type=float, default=3.0,
                    help="--impl reference: wall seconds of one step's oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mindist-l2", type=int, default=1,
                    help="Algorithm 1's refinement test with the Euclidean minimum distance "
                         "(NL_QUAD_MINDIST_L2; the matrix is the same) in the timed steps")
    ap.add_argument("--eps-study", type=int, default=1,
                    help="the eps-convergence leg (0 = skip)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the seeded 512-request serving stream replayed by the "
                         "serving leg (0 = skip; 512 = the whole stream)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-open-loop", type=int, default=1,
                    help="also replay the requests open loop at 70%% load (0 = closed loop only)")
    ap.add_argument("--serve-l2", type=int, default=1,
                    help="serving requests use NL_QUAD_MINDIST_L2 (same matrices, less work)")
    ap.add_argument("--batch-problems", type=int, default=128,
                    help="small problems of the batching leg (0 = skip)")
    ap.add_argument("--profile", action="store_true",
                    help="one pair build and one FP32 (and FP64) assembly of a small workload "
                         "(--profile-workload) for ncu, then exit")
    ap.add_argument("--profile-workload", default="c2_2d_h128")
    ap.add_argument("--profile-fp64", type=int, default=1,
                    help="with --profile: also run the FP64 assembly (0 = FP32 only)")
    ap.add_argument("--profile-precs", default="",
                    help="with --profile: comma list of fp64, fp32, tf32, bf16 (overrides "
                         "--profile-fp64)")
    return ap.parse_args()


def measured_peaks():
    """MEASURED_PEAKS.json (HBM copy GB/s, cuBLAS BF16 TFLOP/s) when present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---- distributed plumbing -------------------------------------------------------------------

def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks ----------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        self.idx = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- workload --------------------------------------------------------------------------------

def workload(name):
    from nl_inputs import WORKLOADS, workload_mesh
    w = WORKLOADS[name]
    mesh = workload_mesh(w)
    return w, mesh


def describe(w, mesh):
    shape = "triangles" if mesh.dim == 2 else "tetrahedra"
    if _is_quad(mesh):
        shape = "quadrilaterals"
    if _is_hex(mesh):
        shape = "hexahedra"
    n_omega = int(mesh.elem_in_omega.sum())
    kern = "constant" if w.kernel == 0 else "truncated Gaussian"
    order = {6: "P2", 10: "P2", 4: "Q1" if mesh.dim == 2 else "P1", 9: "Q2", 27: "Q2", 20: "serendipity",
             8: "Q1" if mesh.dim == 3 else "serendipity"}.get(mesh.conn.shape[1], "P1")
    return (f"{w.name}: Omega=(0,1)^{mesh.dim}, h=1/{round(1 / w.h)}, {mesh.n_elem} {order} {shape} "
            f"({n_omega} in Omega), delta={w.delta / w.h:g}h, eps=delta/{w.delta / w.eps:g}, "
            f"layer {w.layer} cells, L_max={w.L_max}, {kern} kernel, jitter {w.jitter:g}h "
            f"seed {w.seed}; "
            f"u=sum x_k^2; BiCGStab to 1e-10")


def u_exact(mesh):
    return (mesh.coords ** 2).sum(axis=0)  # u = x^2 + y^2 (+ z^2)


def _is_quad(mesh):
    return mesh.dim == 2 and mesh.conn.shape[1] in (4, 8, 9)


def _is_hex(mesh):
    return mesh.dim == 3 and mesh.conn.shape[1] in (8, 20, 27)


def l2_err_omega_quads(mesh, u_h):
    """||u - u_h||_{L2(Omega)} on quadrilaterals (u = sum x_k^2): Gauss-Legendre 3x3 on each
    element's unit square mapped by its bilinear map; Q1 / Q2 basis (tensor products of the 1D
    Lagrange bases on {0, 1} or {0, 1/2, 1}, nodes: vertices, edge midpoints, centre)."""
    x, gw = np.polynomial.legendre.leggauss(3)
    g, gw = (x + 1) / 2, gw / 2
    S, T = np.meshgrid(g, g, indexing="ij")
    W = np.outer(gw, gw).ravel()
    s, t = S.ravel(), T.ravel()
    conn = mesh.conn[mesh.elem_in_omega.astype(bool)]
    V = mesh.points()[conn[:, :4]]  # (ne, 4, 2)
    N = np.stack([(1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], 1)  # (9, 4)
    X = np.einsum("qa,eak->eqk", N, V)
    xs = (1 - t)[None, :, None] * (V[:, 1] - V[:, 0])[:, None] + t[None, :, None] * (V[:, 2] - V[:, 3])[:, None]
    xt = (1 - s)[None, :, None] * (V[:, 3] - V[:, 0])[:, None] + s[None, :, None] * (V[:, 2] - V[:, 1])[:, None]
    det = np.abs(xs[..., 0] * xt[..., 1] - xs[..., 1] * xt[..., 0])
    if conn.shape[1] == 9:
        def L(v):
            return np.stack([2 * (v - 0.5) * (v - 1), 4 * v * (1 - v), 2 * v * (v - 0.5)], 1)
        Ls, Lt = L(s), L(t)
        ij = [(0, 0), (2, 0), (2, 2), (0, 2), (1, 0), (2, 1), (1, 2), (0, 1), (1, 1)]
        phi = np.stack([Ls[:, i] * Lt[:, j] for i, j in ij], 1)
    else:
        phi = N
    uh = np.einsum("qa,ea->eq", phi, u_h[conn])
    d = (X ** 2).sum(-1) - uh
    return float(math.sqrt(np.sum(det * W[None, :] * d * d)))


def l2_err_omega_hexes(mesh, u_h):
    """||u - u_h||_{L2(Omega)} on hexahedra (u = sum x_k^2): Gauss-Legendre 3x3x3 on each
    element's unit cube mapped by its trilinear map; Q1, Q2 (products of the 1D Lagrange
    bases on {0, 1/2, 1}, nodes in the order of nl_inputs.HEX27) or the 20-node serendipity
    element (the first 20 of those nodes)."""
    x, gw = np.polynomial.legendre.leggauss(3)
    g, gw = (x + 1) / 2, gw / 2
    S, T, U = np.meshgrid(g, g, g, indexing="ij")
    s, t, u = S.ravel(), T.ravel(), U.ravel()
    W = np.einsum("i,j,k->ijk", gw, gw, gw).ravel()
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    N, dN = [], []
    for c in corners:
        fs, ft, fu = (s if c[0] else 1 - s), (t if c[1] else 1 - t), (u if c[2] else 1 - u)
        ds, dt, du = (1 if c[0] else -1), (1 if c[1] else -1), (1 if c[2] else -1)
        N.append(fs * ft * fu)
        dN.append(np.stack([ds * ft * fu, fs * dt * fu, fs * ft * du], -1))
    N, dN = np.stack(N, 1), np.stack(dN, 1)  # (27, 8), (27, 8, 3)
    conn = mesh.conn[mesh.elem_in_omega.astype(bool)]
    V = mesh.points()[conn[:, :8]]  # (ne, 8, 3)
    X = np.einsum("qa,eak->eqk", N, V)
    J = np.einsum("qar,eak->eqkr", dN, V)
    det = np.abs(np.linalg.det(J))
    phi = N
    if conn.shape[1] == 27:
        from nl_inputs import HEX27

        def L(v):
            return np.stack([2 * (v - 0.5) * (v - 1), 4 * v * (1 - v), 2 * v * (v - 0.5)], 1)
        Ls, Lt, Lu = L(s), L(t), L(u)
        phi = np.stack([Ls[:, i] * Lt[:, j] * Lu[:, k] for i, j, k in HEX27], 1)
    elif conn.shape[1] == 20:
        from nl_inputs import HEX27
        c = np.stack([2 * s - 1, 2 * t - 1, 2 * u - 1], 1)
        cols = []
        for a, node in enumerate(HEX27[:20]):
            f = np.array(node, float) - 1
            lin = [1 - c[:, k] ** 2 if f[k] == 0 else 1 + f[k] * c[:, k] for k in range(3)]
            p = lin[0] * lin[1] * lin[2]
            cols.append(p * (c @ f - 2) / 8 if a < 8 else p / 4)
        phi = np.stack(cols, 1)
    uh = np.einsum("qa,ea->eq", phi, u_h[conn])
    d = (X ** 2).sum(-1) - uh
    return float(math.sqrt(np.sum(det * W[None, :] * d * d)))


def l2_err_omega(mesh, u_h, rule):
    """||u - u_h||_{L2(Omega)} with the degree-5 rule per element (u = sum x_k^2); P1, or P2
    simplices when the elements have more nodes than vertices (basis lambda_a (2 lambda_a - 1)
    at the vertices, 4 lambda_a lambda_b at the edge nodes (0,1), (1,2), (0,2) (, (0,3), (1,3),
    (2,3))); quadrilaterals and hexahedra with their own routines."""
    if _is_quad(mesh):
        return l2_err_omega_quads(mesh, u_h)
    if _is_hex(mesh):
        return l2_err_omega_hexes(mesh, u_h)
    b, w = rule
    P = mesh.points()
    conn = mesh.conn[mesh.elem_in_omega.astype(bool)]
    nv = mesh.dim + 1
    V = P[conn[:, :nv]]  # (ne, nv, dim)
    if mesh.dim == 2:
        vol = 0.5 * np.abs((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1]) -
                           (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    else:
        vol = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])) / 6.0
    X = np.einsum("qv,evk->eqk", b, V)
    if conn.shape[1] > nv:  # P2: vertices, then the edge nodes in the mesh's edge order
        edges = [(0, 1), (1, 2), (0, 2)] if mesh.dim == 2 else [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
        phi = np.concatenate([b * (2 * b - 1)] + [4 * b[:, [i]] * b[:, [j]] for i, j in edges], axis=1)
    else:
        phi = b
    uh = np.einsum("qv,ev->eq", phi, u_h[conn])
    d = (X ** 2).sum(-1) - uh
    return float(math.sqrt(np.sum(vol[:, None] * w[None, :] * d * d)))


# ---- our implementation ----------------------------------------------------------------------

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x 2 flops x max SM clock
FP64_PEAK_TFLOPS = 1.19  # measured FP64 FMA chain of this GPU model


def _measure(nl, torch, stream, dmesh, mesh, w, prec, steps, warmup, flush, world,
             keep_last=False, l2=False):
    """Times `steps` whole steps (pairs, pattern, assembly, right-hand side, BiCGStab) after
    `warmup` untimed ones; the L2 is flushed before every timed step, outside the timing.
    Returns per-step times, solve times, the last step's stats, solution and (keep_last)
    the last matrix, and the launches of this library in the timed region."""
    g = u_exact(mesh)
    f_const = -2.0 * mesh.dim
    sprec = nl.NL_PREC_FP64 if prec == nl.NL_PREC_FP64 else nl.NL_PREC_FP32

    def step():
        p = nl.nl_pairs_build(dmesh, w.delta, w.eps)
        A, st = nl.nl_assemble(dmesh, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, prec,
                               mindist_l2=l2)
        b = nl.nl_rhs(dmesh, A, g, f_const=f_const)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        u, it, rr, _ = nl.nl_solve(A, b, g, solver=1, rtol=1e-10, max_iter=20000, precision=sprec)
        t1.record(stream)
        t1.synchronize()
        return dict(st=st, u=u, it=it, rr=rr, solve_ms=t0.elapsed_time(t1), A=A, p=p)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    times, solve_ms, stats, last = [], [], [], None
    launches0 = nl.lib().nl_launch_count()
    for k in range(steps):
        if last is not None:
            last.pop("A", None)
            last.pop("p", None)
        flush.zero_()  # L2 flush (256 MB > 129 MB L2) between steps, outside the timing
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        solve_ms.append(last["solve_ms"])
        stats.append(last["st"])
    launches = nl.lib().nl_launch_count() - launches0
    A = last.pop("A")
    last.pop("p")
    if keep_last:
        last["values"] = A.export()
    del A
    return dict(times=times, solve_ms=solve_ms, stats=stats, last=last, launches=launches)


def _roofline(nl, dmesh, mesh, w, prec, stats, l2=False, stb=None):
    """Algorithmic flops of the assembly kernel over the measured steps against the FP32 ALU
    (or FP64 pipe) peak; the band count comes from one extra untimed launch with
    NL_QUAD_COUNT_BAND (stb: the counters of such a launch already made; the FP64 kernel
    reuses the FP32 launch's, whose Algorithm-1 decisions are the same and whose band count
    differs only by the rounding of r at the band edges)."""
    if stb is None:
        pb = nl.nl_pairs_build(dmesh, w.delta, w.eps)
        _, stb = nl.nl_assemble(dmesh, pb, w.delta, w.eps, w.L_max, w.L_min, w.kernel, prec,
                                count_band=True, mindist_l2=l2)
    nb = mesh.conn.shape[1]
    flops = roofline_flops(mesh.dim, stb, nb=nb)
    flops_ev = roofline_flops(mesh.dim, stb, evaluated_only=True, nb=nb)
    quad_ms = statistics.mean(s.ms_quad for s in stats)
    f32 = prec != nl.NL_PREC_FP64
    peak = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
    achieved = flops / (quad_ms / 1e3) / 1e12
    achieved_ev = flops_ev / (quad_ms / 1e3) / 1e12
    rtype = "float" if f32 else "double"
    return stb, {
        "bound": "alu" if f32 else "fp64 pipe", "achieved": round(achieved, 3),
        "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
        "units": "Algorithm-1 quadrature point pairs (closed-form ones included)",
        "frac_evaluated_only": round(achieved_ev / peak, 4),
        "kernel": (f"k_quad_p2<{rtype},{w.kernel}>" if nb == 6 else
                   f"k_quad_p2t<{rtype},{w.kernel}>" if nb == 10 else
                   f"k_quad_h<{rtype},{w.kernel},{nb}>" if _is_hex(mesh) else
                   f"k_quad_q<{rtype},{w.kernel},{ {4: 1, 9: 2, 8: 3}[nb] }>" if _is_quad(mesh) else
                   f"k_quad<{mesh.dim},{rtype},{w.kernel}>"), "flops_per_assembly": flops,
        "kernel_ms_per_assembly": round(quad_ms, 3),
        "launches_per_assembly": int(stats[-1].n_quad_launches),
        "peak_source": ("152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (derived)" if f32 else
                        "FP64 FMA-chain microbenchmark on GB300 (measured)")}


def _scatter_bytes(mesh, pairs_info, rp, dim, rsize):
    """Algorithmic bytes of the scatter over one assembly: every cross block read once (with
    its pair_l entry and l's nodes), and per inner element the rows of its nodes: their
    column lists read and their values updated (FP64 read + write) once."""
    n_pairs = pairs_info[0]
    nv = dim + 1
    deg = np.bincount(mesh.conn.ravel(), minlength=mesh.n_vert)
    rowlen = np.diff(rp)
    per_elem_rows = int(np.sum(deg.astype(np.int64) * rowlen))
    return int(n_pairs * (nv * nv * rsize + 4 + 4 * nv) + per_elem_rows * (4 + 16))


def _spmv_rate(nl, torch, stream, A, mesh, nnz, reps=20):
    """nl_matrix_apply (FP64 y = A x over all rows): CUDA-event time per call and achieved
    HBM bandwidth for the algorithmic bytes (values 8 + col 4 per entry, row_ptr, x and y
    once)."""
    x = torch.rand(mesh.n_vert, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    A.apply(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        A.apply(x.data_ptr(), y.data_ptr())
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    byts = 12 * nnz + 8 * (mesh.n_vert + 1) + 16 * mesh.n_vert
    return {"kernel": "k_spmv<double,double>", "ms": round(ms, 4), "bytes": int(byts),
            "achieved_gbs": round(byts / (ms / 1e3) / 1e9, 1)}


def run_ours(args, rank, world, local):
    import torch
    from paper_2101_08825_gb300 import nl
    from paper_2101_08825_gb300.build import build

    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build()
    barrier(world)
    nl.lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(int(256 * 2 ** 20) // 4, dtype=torch.float32, device="cuda")
    peaks = measured_peaks()

    w, mesh = workload(args.workload)
    rule = nl.nl_quad_rule(mesh.dim)
    dmesh = nl.mesh_from(mesh)

    # mixed headline (timed with clock sampling)
    clk = ClockSampler(local)
    clk.start()
    L2 = bool(args.mindist_l2)
    mx = _measure(nl, torch, stream, dmesh, mesh, w, nl.NL_PREC_FP32, args.steps, args.warmup,
                  flush, world, keep_last=args.fp64_steps > 0, l2=L2)
    clocks = clk.stop()
    ms = statistics.mean(mx["times"])
    ms_max = allmax(world, ms)
    st = mx["stats"][-1]
    n_pairs, n_pp = st.n_pairs, st.n_point_pairs
    value = world * n_pairs / (ms_max / 1e3)
    err_mixed = l2_err_omega(mesh, mx["last"]["u"], rule)
    kern_ms = statistics.mean(s.ms_assemble for s in mx["stats"])
    stb, roof = _roofline(nl, dmesh, mesh, w, nl.NL_PREC_FP32, mx["stats"], l2=L2)
    tb = TRAFFIC_BYTES_PER_PAIR.get(mesh.dim)
    roof["traffic"] = round(tb * n_pairs / roof["launches_per_assembly"]) if tb else None
    roof["traffic_per_launch_note"] = ("DRAM bytes per element pair of the ncu capture of the "
                                       "current kernel on the small case of this dimension, "
                                       "times the pairs of one launch")

    # the FP64 step on the same workload (the FP64 kernels are warmed on a tiny case first)
    fp64 = None
    if args.fp64_steps > 0:
        wc1, mc1 = workload("c1_2d" if mesh.dim == 2 else "c3_3d_h10")
        dc1 = nl.mesh_from(mc1)
        _measure(nl, torch, stream, dc1, mc1, wc1, nl.NL_PREC_FP64, 1, 0, flush, world)
        del dc1
        f64 = _measure(nl, torch, stream, dmesh, mesh, w, nl.NL_PREC_FP64, args.fp64_steps, 0,
                       flush, world, keep_last=True, l2=L2)
        ms64 = allmax(world, statistics.mean(f64["times"]))
        err64 = l2_err_omega(mesh, f64["last"]["u"], rule)
        v32, v64 = mx["last"]["values"], f64["last"]["values"]
        a_rel = float(np.linalg.norm(v32 - v64) / np.linalg.norm(v64))
        a_max = float(np.abs(v32 - v64).max() / np.abs(v64).max())
        _, roof64 = _roofline(nl, dmesh, mesh, w, nl.NL_PREC_FP64, f64["stats"], l2=L2, stb=stb)
        fp64 = {"dtype": "f64", "ms_per_step": round(ms64, 3), "steps": args.fp64_steps,
                "value": round(world * n_pairs / (ms64 / 1e3), 1),
                "assembly_ms": round(statistics.mean(s.ms_assemble for s in f64["stats"]), 3),
                "l2_err_omega": err64, "roofline": roof64}
        mx["last"].pop("values", None)

    # HBM-bound kernels of the step: the scatter (from the assembly's own CUDA events) and the
    # SpMV (nl_matrix_apply, FP64)
    p = nl.nl_pairs_build(dmesh, w.delta, w.eps)
    pinfo = p.info()
    rp = p.export(mesh.n_elem, mesh.n_vert)[2]
    sc_bytes = _scatter_bytes(mesh, pinfo, rp, mesh.dim, 4)
    sc_ms = statistics.mean(s.ms_scatter for s in mx["stats"])
    A, _ = nl.nl_assemble(dmesh, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, nl.NL_PREC_FP32,
                          mindist_l2=L2)
    # the same FP32 assembly with the paper's default refinement test (eq. mindist) and with the
    # tensor-core contraction (TF32, BF16), one timed call each
    variants = {}
    for vname, vprec, vl2 in (("fp32_eq_mindist", nl.NL_PREC_FP32, False),
                              ("mixed_tf32", nl.NL_PREC_MIXED_TF32, L2),
                              ("mixed_bf16", nl.NL_PREC_MIXED_BF16, L2)):
        _, vst = nl.nl_assemble(dmesh, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, vprec,
                                mindist_l2=vl2)
        variants[vname] = {"assembly_ms": round(vst.ms_assemble, 3),
                           "kernel_ms": round(vst.ms_quad, 3),
                           "quad_pt_pairs": vst.n_point_pairs,
                           "evaluated_point_pairs": vst.n_eval_point_pairs,
                           "precision_run": int(vst.precision_run)}
    hbm_peak = peaks.get("hbm_gbs", 6746.0)
    spmv = _spmv_rate(nl, torch, stream, A, mesh, pinfo[1])
    spmv["frac"] = round(spmv["achieved_gbs"] / hbm_peak, 4)
    hbm = {"peak_gbs": hbm_peak, "peak_source": "measured STREAM-style copy",
           "scatter": {"kernel": f"k_scatter<{mesh.dim},float>", "ms_per_assembly": round(sc_ms, 3),
                       "bytes": sc_bytes,
                       "achieved_gbs": round(sc_bytes / (sc_ms / 1e3) / 1e9, 1) if sc_ms > 0 else None,
                       "frac": round(sc_bytes / (sc_ms / 1e3) / 1e9 / hbm_peak, 4) if sc_ms > 0 else None,
                       "bound": "FP64 atomics (shared, then global)"},
           "spmv": spmv}
    del A, p

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "element pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": describe(w, mesh),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "working set > L2 and a 256 MB L2 flush between steps"},
        "quad_pt_pairs_per_s": round(world * n_pp / (ms_max / 1e3), 1),
        "assembly": {"ms": round(kern_ms, 3), "kernel_ms": roof["kernel_ms_per_assembly"],
                     "element_pairs_per_s": round(n_pairs / (kern_ms / 1e3), 1),
                     "quad_pt_pairs_per_s": round(n_pp / (kern_ms / 1e3), 1)},
        "counts": {"element_pairs": n_pairs, "quad_pt_pairs": n_pp, "items": st.n_items,
                   "fp64_rechecks": st.n_exact_checks,
                   "evaluated_point_pairs": stb.n_eval_point_pairs,
                   "band_point_pairs": stb.n_band_point_pairs,
                   "closed_form_items": stb.n_closed_items, "nnz": int(pinfo[1])},
        "fp64": fp64,
        "mixed": {"l2_err_omega": err_mixed, "precision_run": int(st.precision_run),
                  "A_rel_frobenius_vs_fp64": a_rel if fp64 else None,
                  "A_max_entry_rel_vs_fp64": a_max if fp64 else None,
                  "solve_iters": mx["last"]["it"],
                  "speedup_vs_fp64": round(ms64 / ms, 2) if fp64 else None},
        "solve_ms": {"p50": round(float(np.percentile(mx["solve_ms"], 50)), 3),
                     "p99": round(float(np.percentile(mx["solve_ms"], 99)), 3)},
        "roofline": roof,
        "hbm_kernels": hbm,
        "quad_rule": ("Algorithm 1 with the Euclidean approximate minimum distance of Sec. 5.1 "
                      "(NL_QUAD_MINDIST_L2; same matrix as eq. mindist)" if L2 else
                      "Algorithm 1 with eq. mindist"),
        "assembly_variants": variants,
        "gpu_launches": int(mx["launches"]),  # this library's kernels in the whole timed region
        "gpu_launches_per_step": int(mx["launches"] / max(1, args.steps)),
        "clocks": clocks,
    }
    del dmesh
    if not args.no_e2e:
        out["e2e"] = e2e_ours(args, mesh, w, stream, world)
    if args.c2_steps > 0:
        out["c2_2d"] = run_c2_block(args, nl, torch, stream, flush, world)
    if args.p2_steps > 0:
        out["p2"] = run_element_block(args, nl, torch, stream, flush, world, "c2_2d_p2",
                                      args.p2_steps, args.p2_fp64_steps)
    if args.quad_steps > 0:
        for key, name in (("q1", "c2_2d_q1"), ("q2", "c2_2d_q2"), ("hex", "c3_3d_hex"),
                          ("hex_q2", "c3_3d_hex_q2"), ("p2_tet", "c3_3d_p2")):
            out[key] = run_element_block(args, nl, torch, stream, flush, world, name,
                                         args.quad_steps, args.quad_fp64_steps)
    if args.eps_study:
        out["eps_study"] = run_eps_study(args)
    if args.batch_problems > 0:
        out["batching"] = run_batching(args)
    if args.serve_requests > 0:
        out["serving"] = run_serving(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(mesh, w, seconds=args.cpu_seconds)
    return out


def run_c2_block(args, nl, torch, stream, flush, world):
    """The 2D workload at h = 1/256 in its four (eps, kernel) combinations: mixed step and
    FP64 step with the L2 errors of both, and the FP32 kernel's roofline."""
    out = {}
    for name in C2_BLOCK:
        w, mesh = workload(name)
        rule = nl.nl_quad_rule(2)
        dm = nl.mesh_from(mesh)
        L2 = bool(args.mindist_l2)
        mx = _measure(nl, torch, stream, dm, mesh, w, nl.NL_PREC_FP32, args.c2_steps, 2, flush,
                      world, keep_last=args.c2_fp64_steps > 0, l2=L2)
        ms = statistics.mean(mx["times"])
        st = mx["stats"][-1]
        _, roof = _roofline(nl, dm, mesh, w, nl.NL_PREC_FP32, mx["stats"], l2=L2)
        tb = TRAFFIC_BYTES_PER_PAIR.get(2)
        roof["traffic"] = round(tb * st.n_pairs / roof["launches_per_assembly"]) if tb else None
        r = {"workload": describe(w, mesh), "element_pairs": st.n_pairs,
             "quad_pt_pairs": st.n_point_pairs, "ms_per_step": round(ms, 3),
             "element_pairs_per_s": round(st.n_pairs / (ms / 1e3), 1),
             "quad_pt_pairs_per_s": round(st.n_point_pairs / (ms / 1e3), 1),
             "assembly_ms": round(statistics.mean(s.ms_assemble for s in mx["stats"]), 3),
             "l2_err_omega": l2_err_omega(mesh, mx["last"]["u"], rule),
             "solve_ms_p50": round(float(np.percentile(mx["solve_ms"], 50)), 3),
             "roofline": roof}
        if args.c2_fp64_steps > 0:
            f64 = _measure(nl, torch, stream, dm, mesh, w, nl.NL_PREC_FP64, args.c2_fp64_steps, 0,
                           flush, world, keep_last=True, l2=L2)
            ms64 = statistics.mean(f64["times"])
            v32, v64 = mx["last"]["values"], f64["last"]["values"]
            r["fp64"] = {"ms_per_step": round(ms64, 3),
                         "element_pairs_per_s": round(st.n_pairs / (ms64 / 1e3), 1),
                         "l2_err_omega": l2_err_omega(mesh, f64["last"]["u"], rule),
                         "speedup_of_mixed": round(ms64 / ms, 2),
                         "A_rel_frobenius": float(np.linalg.norm(v32 - v64) / np.linalg.norm(v64))}
        out[name] = r
        del dm
    return out


def run_element_block(args, nl, torch, stream, flush, world, name, steps, fp64_steps):
    """Other element families: on the 2D workload's grid (h = 1/256) P2 triangles (c2_2d_p2:
    141,512 triangles, 284,089 nodes), Q1 and Q2 quadrilaterals (c2_2d_q1, c2_2d_q2: 70,756
    cells); on the 3D grid at h = 1/16 Q1 and Q2 hexahedra (c3_3d_hex, c3_3d_hex_q2: 10,648
    cells, the latter 91,125 nodes) and P2 tetrahedra (c3_3d_p2: 63,888 tetrahedra, 91,125
    nodes).  The FP32 step and the FP64 step (pairs, pattern, assembly, right-hand side,
    BiCGStab), their L2 errors, and the roofline of the assembly kernel in both
    precisions."""
    w, mesh = workload(name)
    rule = nl.nl_quad_rule(mesh.dim)
    dm = nl.mesh_from(mesh)
    mx = _measure(nl, torch, stream, dm, mesh, w, nl.NL_PREC_FP32, steps, 1, flush, world,
                  keep_last=fp64_steps > 0)
    ms = statistics.mean(mx["times"])
    st = mx["stats"][-1]
    stb, roof = _roofline(nl, dm, mesh, w, nl.NL_PREC_FP32, mx["stats"])
    roof["traffic"] = None
    r = {"workload": describe(w, mesh), "element_pairs": st.n_pairs,
         "quad_pt_pairs": st.n_point_pairs, "ms_per_step": round(ms, 3),
         "element_pairs_per_s": round(world * st.n_pairs / (ms / 1e3), 1),
         "quad_pt_pairs_per_s": round(world * st.n_point_pairs / (ms / 1e3), 1),
         "assembly_ms": round(statistics.mean(s.ms_assemble for s in mx["stats"]), 3),
         "scatter_ms": round(statistics.mean(s.ms_scatter for s in mx["stats"]), 3),
         "l2_err_omega": l2_err_omega(mesh, mx["last"]["u"], rule),
         "solve_ms_p50": round(float(np.percentile(mx["solve_ms"], 50)), 3),
         "solve_iters": mx["last"]["it"], "gpu_launches_per_step": int(mx["launches"] / max(1, steps)),
         "roofline": roof}
    if fp64_steps > 0:
        f64 = _measure(nl, torch, stream, dm, mesh, w, nl.NL_PREC_FP64, fp64_steps, 0,
                       flush, world, keep_last=True)
        ms64 = statistics.mean(f64["times"])
        _, roof64 = _roofline(nl, dm, mesh, w, nl.NL_PREC_FP64, f64["stats"], stb=stb)
        v32, v64 = mx["last"]["values"], f64["last"]["values"]
        r["fp64"] = {"ms_per_step": round(ms64, 3),
                     "element_pairs_per_s": round(world * st.n_pairs / (ms64 / 1e3), 1),
                     "assembly_ms": round(statistics.mean(s.ms_assemble for s in f64["stats"]), 3),
                     "l2_err_omega": l2_err_omega(mesh, f64["last"]["u"], rule),
                     "speedup_of_fp32": round(ms64 / ms, 2),
                     "A_rel_frobenius": float(np.linalg.norm(v32 - v64) / np.linalg.norm(v64)),
                     "roofline": roof64}
    del dm
    return r


def roofline_flops(dim, st, evaluated_only=False, nb=None):
    """Algorithmic flops of one assembly (FMA = 2), per quadrature point pair of the method's
    double sum as written (eqs. J21Nr, J22Nr): the distance and r^2 (2D 5, 3D 8), the weight
    w_x w_y C mu (2), the rank-one update of the local block over the nodes of m (2D 6, 3D 8)
    and the self-term sum (1): 14 (2D) / 19 (3D); per band point pair additionally r (1),
    s = (delta - r)/eps (2) and xi(s) by Horner (12): 15.  The units are the point pairs of
    Algorithm 1 (the method's quad-pt pairs: every (sub-element, m) item it integrates times
    the two rules' points), whether the kernel evaluates them one by one or sums a
    sub-element's point pairs in closed form (mu exactly 1 or 0); evaluated_only counts only
    the point pairs evaluated one by one.  (The kernel itself hoists the contraction with m's
    basis out of the loop over outer points and executes 11 (2D) / 16 (3D) flops per
    evaluated point pair for the same sums.)  With nb nodes per element (P2 triangles: 6) the
    rank-one update costs 2 nb: 20 flops per point pair."""
    pp = int(getattr(st, "n_eval_point_pairs" if evaluated_only else "n_point_pairs", 0) or 0)
    band = max(0, int(getattr(st, "n_band_point_pairs", 0) or 0))
    nb = nb or dim + 1
    per_pp = (5 if dim == 2 else 8) + 2 + 2 * nb + 1
    return float(max(0, pp) * per_pp + band * 15)


def e2e_ours(args, mesh, w, stream, world):
    """Public-API step from pinned host buffers: mesh upload, pairs, assembly, right-hand
    side, solve and the solution read back, all inside the timed region (one warm-up step,
    then up to three timed ones)."""
    import torch
    from paper_2101_08825_gb300 import nl

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    g = u_exact(mesh)
    f_const = -2.0 * mesh.dim
    coords, conn = pinned(mesh.coords), pinned(mesh.conn)
    eio, nf, gp = pinned(mesh.elem_in_omega), pinned(mesh.node_free), pinned(g)
    times = []
    steps = max(1, min(args.steps, 3))
    for k in range(1 + steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dm = nl.nl_mesh_create(mesh.dim, coords, conn, eio, nf)
        p = nl.nl_pairs_build(dm, w.delta, w.eps)
        A, st = nl.nl_assemble(dm, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel,
                               nl.NL_PREC_FP32, mindist_l2=bool(args.mindist_l2))
        b = nl.nl_rhs(dm, A, gp, f_const=f_const)
        u, it, rr, _ = nl.nl_solve(A, b, gp, solver=1, rtol=1e-10, max_iter=20000,
                                   precision=nl.NL_PREC_FP32)
        e1.record(stream)
        e1.synchronize()
        if k >= 1:
            times.append(e0.elapsed_time(e1))
        n_pairs = st.n_pairs
        del A, b, p, dm
    ms = allmax(world, statistics.mean(times))
    h2d = coords.nbytes + conn.nbytes + eio.nbytes + nf.nbytes + 2 * gp.nbytes
    d2h = u.nbytes
    return {"value": round(world * n_pairs / (ms / 1e3), 1), "unit": "element pairs/s",
            "ms_per_step": round(ms, 3), "steps": steps, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


def run_batching(args):
    """Batching leg: many small 2D problems (8-24 cells per side, delta in {2,3,4}h,
    eps = delta/10, L_max = 3, constant and Gaussian kernels alternating, jitter 0.1h), meshes
    and pair lists resident.  Sequential nl_assemble calls against one plan that assembles
    all of them in a single launch (autotuned launch shape, replayed CUDA graph); FP32."""
    import torch
    from paper_2101_08825_gb300 import nl
    probs = []
    for i in range(args.batch_problems):
        n = 8 + (i * 7) % 17
        h = 1.0 / n
        delta = (2 + i % 3) * h
        eps = delta / 10
        layer = int(math.ceil((delta + eps) / h - 1e-9))
        m = nl.nl_mesh_create_box(2, (n, n), h, (0.0, 0.0), layer, 0.1, i)
        p = nl.nl_pairs_build(m, delta, eps)
        probs.append((m, p, delta, eps, 3, 1, i % 2))
    pairs = sum(pr[1].info()[0] for pr in probs)

    def seq():
        for pr in probs:
            nl.nl_assemble(*pr[:2], pr[2], pr[3], pr[4], pr[5], pr[6], nl.NL_PREC_FP32)
        torch.cuda.synchronize()

    seq()
    t0 = time.perf_counter()
    for _ in range(3):
        seq()
    t_seq = (time.perf_counter() - t0) / 3
    plan = nl.Plan(probs, precision=nl.NL_PREC_FP32, flags=nl.NL_PLAN_AUTOTUNE | nl.NL_PLAN_GRAPH)
    plan.execute()
    plan.sync()
    t0 = time.perf_counter()
    for _ in range(10):
        plan.execute()
        st = plan.sync()
    t_plan = (time.perf_counter() - t0) / 10
    return {"problems": len(probs), "element_pairs": int(pairs),
            "sequential_pairs_per_s": round(pairs / t_seq, 1),
            "plan_pairs_per_s": round(pairs / t_plan, 1), "speedup": round(t_seq / t_plan, 2),
            "plan_gpu_ms": round(st[0].ms_assemble, 3), "shape": plan.shape()}


def l2_norm_p1(mesh, v, rule):
    """L2 norm over Omega of the P1 function with nodal values v (degree-5 rule)."""
    b, w = rule
    P = mesh.points()
    conn = mesh.conn[mesh.elem_in_omega.astype(bool)]
    V = P[conn]
    if mesh.dim == 2:
        vol = 0.5 * np.abs((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1]) -
                           (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    else:
        vol = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])) / 6.0
    vq = np.einsum("qv,ev->eq", b, v[conn])
    return float(math.sqrt(np.sum(vol[:, None] * w[None, :] * vq * vq)))


def run_eps_study(args):
    """eps-convergence study (the P1 analogue of the paper's Table 4): Omega = (0,1)^2,
    h = 1/32, delta = 0.1, u = x^4 + y^4 with the forcing of the sharp kernel
    (f = -12 (x^2 + y^2) - 2 delta^2, its P1 interpolant), the mollified kernel assembled for
    eps = delta/4 ... delta/64 at L_max = L0 - 1 ... L0 + 2, where L0 makes Algorithm 1's
    smallest sub-elements about eps (L0 = ceil(log2(h / eps)) + 1).  Reports per (eps, L_max)
    the FP32 and FP64 assembly times and the work, and two differences of the FP64 discrete
    solutions in L2(Omega) (FP64, so that no FP32 rounding of sums over up to 1e5 point pairs
    per element pair enters): to the same eps at L_max + 1 (quadrature error) and, at L0, to
    eps / 2 (the mollifier's contribution, expected to fall like eps^2)."""
    import torch
    from paper_2101_08825_gb300 import nl
    n, delta = 32, 0.1
    h = 1.0 / n
    divs = (4, 8, 16, 32, 64)
    layer = int(math.ceil((delta + delta / divs[0]) / h - 1e-9))
    from nl_inputs import structured_mesh
    mesh = structured_mesh(2, n, h, 0.0, layer)
    rule = nl.nl_quad_rule(2)
    X = mesh.coords
    g = (X ** 4).sum(axis=0)
    f = -12.0 * (X ** 2).sum(axis=0) - 2.0 * delta * delta
    dm = nl.mesh_from(mesh)
    rows, sol = [], {}
    for div in divs:
        eps = delta / div
        L0 = int(math.ceil(math.log2(h / eps))) + 1
        p = nl.nl_pairs_build(dm, delta, eps)
        for L in (L0 - 1, L0, L0 + 1, L0 + 2):
            if L < 1:
                continue
            nl.nl_assemble(dm, p, delta, eps, L, precision=nl.NL_PREC_FP32)  # warm
            _, st32 = nl.nl_assemble(dm, p, delta, eps, L, precision=nl.NL_PREC_FP32)
            A, st = nl.nl_assemble(dm, p, delta, eps, L, precision=nl.NL_PREC_FP64)
            b = nl.nl_rhs(dm, A, g, f_nodes=f)
            u, it, rr, _ = nl.nl_solve(A, b, g, solver=1, rtol=1e-12, max_iter=20000,
                                       precision=nl.NL_PREC_FP64)
            sol[(div, L)] = u
            rows.append({"eps": f"delta/{div}", "L_max": L, "L0": L0,
                         "assembly_ms_fp32": round(st32.ms_assemble, 3),
                         "assembly_ms_fp64": round(st.ms_assemble, 3),
                         "point_pairs": st.n_point_pairs, "element_pairs": st.n_pairs})
            del A, b
    for r in rows:
        div, L = int(r["eps"].split("/")[1]), r["L_max"]
        if (div, L + 1) in sol:
            r["quad_err_l2"] = l2_norm_p1(mesh, sol[(div, L)] - sol[(div, L + 1)], rule)
    conv = []
    for k in range(len(divs) - 1):
        a, c = divs[k], divs[k + 1]
        La = int(math.ceil(math.log2(h / (delta / a)))) + 1
        Lc = int(math.ceil(math.log2(h / (delta / c)))) + 1
        conv.append({"eps": f"delta/{a}", "diff_to_half_eps_l2":
                     l2_norm_p1(mesh, sol[(a, La)] - sol[(c, Lc)], rule)})
    for k in range(len(conv) - 1):
        conv[k]["p2"] = round(math.log2(conv[k]["diff_to_half_eps_l2"] /
                                        conv[k + 1]["diff_to_half_eps_l2"]), 3)
    return {"workload": "Omega=(0,1)^2, h=1/32, delta=0.1, u=x^4+y^4, sharp-kernel forcing; "
                        "FP64 assembly and BiCGStab to 1e-12 for the differences, FP32 "
                        "assembly timed beside",
            "runs": rows, "eps_convergence": conv}


def run_serving(args):
    """Serving leg: the first N requests of the seeded 512-request stream (mixed 2D/3D
    meshes, delta in [2h, 6h], constant or truncated-Gaussian kernel), each running mesh,
    pairs, FP32 assembly, right-hand side and BiCGStab in FP32 with FP64 refinement to 1e-10
    on the library's server.  Phase 1 submits all N at once (closed loop: throughput at
    saturation).  Phase 2 replays them with the stream's exponential inter-arrival gaps
    rescaled to 70% of that throughput (open loop at 70% load) and reports the latency
    percentiles (completion - submission, server clock)."""
    from nl_inputs.requests import serving_stream
    from paper_2101_08825_gb300 import nl
    reqs = serving_stream(512, seed=0)[: args.serve_requests]
    budget = 64 << 30

    def make(i, r):
        return nl.make_request(r.dim, (r.n,) * r.dim, 1.0 / r.n, (0.0,) * r.dim, r.layer,
                               r.delta, r.eps, r.L_max, kernel=r.kernel,
                               precision=nl.NL_PREC_FP32, ms=1, solver=1, rtol=1e-10,
                               jitter=0.1, seed=i, mindist_l2=args.serve_l2)

    def replay(times):
        with nl.Server(budget, args.serve_slots) as S:
            t0 = time.perf_counter()
            tickets = []
            for i, (r, ta) in enumerate(zip(reqs, times)):
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                tickets.append(S.submit(make(i, r)))
            results = [S.wait(t) for t in tickets]
            wall = time.perf_counter() - t0
            p50, p99, sps = S.stats()
        ok = [r for r in results if r.status == nl.NL_OK]
        lat = [r.t_done_ms - r.t_submit_ms for r in ok]
        queue = [r.t_start_ms - r.t_submit_ms for r in ok]
        run = [r.t_done_ms - r.t_start_ms for r in ok]
        per = [{"dim": rq.dim, "n_elem": rq.n_elem, "pairs": int(r.n_pairs),
                "queue_ms": round(r.t_start_ms - r.t_submit_ms, 1),
                "run_ms": round(r.t_done_ms - r.t_start_ms, 1), "group": int(r.group)}
               for rq, r in zip(reqs, results) if r.status == nl.NL_OK]
        return dict(p50=p50, p99=p99, sps=sps, wall=wall, failed=len(results) - len(ok),
                    pairs=sum(r.n_pairs for r in ok), lat=lat, queue=queue, run=run, per=per,
                    grouped=sum(1 for r in ok if r.group >= 0))

    sat = replay([0.0] * len(reqs))
    rate = 0.7 * sat["sps"]
    gaps = np.diff([0.0] + [r.arrival_s for r in reqs])
    scale = (1.0 / rate) / max(float(np.mean(gaps)), 1e-9) if rate > 0 else 0.0
    arrivals = np.cumsum(gaps * scale)
    ol = replay(list(arrivals)) if args.serve_open_loop else None

    def pct(v, q):
        return round(float(np.percentile(v, q)), 2) if v else None

    out = {"requests": len(reqs), "slots": args.serve_slots, "budget_bytes": budget,
           "quad_rule": "NL_QUAD_MINDIST_L2" if args.serve_l2 else "eq. mindist",
           "saturation": {"solves_per_s": round(sat["sps"], 3),
                          "element_pairs_per_s": round(sat["pairs"] / sat["wall"], 1),
                          "p50_ms": round(sat["p50"], 2), "p99_ms": round(sat["p99"], 2),
                          "grouped_requests": sat["grouped"], "failed": sat["failed"]}}
    if ol is not None:
        out["open_loop"] = {"arrival_rate_per_s": round(rate, 3), "p50_ms": round(ol["p50"], 2),
                            "p99_ms": round(ol["p99"], 2), "solves_per_s": round(ol["sps"], 3),
                            "max_latency_ms": round(max(ol["lat"]), 2) if ol["lat"] else None,
                            "queue_ms_p50": pct(ol["queue"], 50), "queue_ms_p99": pct(ol["queue"], 99),
                            "run_ms_p50": pct(ol["run"], 50), "run_ms_p99": pct(ol["run"], 99),
                            "grouped_requests": ol["grouped"], "failed": ol["failed"],
                            "per_request": ol["per"] if len(reqs) <= 64 else None}
    out.update({
            "sample": f"first {len(reqs)} of the 512-request seeded stream (seed 0); phase 2 "
                      f"arrivals = the stream's exponential gaps rescaled to 70% of phase 1's "
                      f"throughput"})
    return out


# ---- the oracle on a bounded sample, on all host cores ---------------------------------------

def _oracle_rows(args):
    """One process of the oracle sample: pairs (brute force), pattern and Algorithm-1
    assembly restricted to the inner elements `sel` of the workload; returns the pair and
    point-pair counts."""
    name, sel = args
    import oracle as O
    w, mesh = workload(name)
    mask = np.zeros(mesh.n_elem, np.uint8)
    mask[sel] = 1
    om = O.OMesh(mesh)
    off, pl = O.pairs(om, w.delta, w.eps, m_mask=mask)
    rp, col = O.csr(om, off, pl)
    _, st = O.assemble(om, off, pl, rp, col, w.delta, w.eps, w.L_max, w.L_min, w.kernel,
                       m_mask=mask)
    return len(pl), st.n_point_pairs


def _oracle_warm(name):
    import oracle as O
    O.build()
    O.lib()
    workload(name)
    return os.getpid()


class OraclePool:
    """Spawned worker processes (one per host core) that run the plain single-threaded oracle
    on disjoint seeded samples of inner elements.  Spawned, never forked: the parent may
    already hold a CUDA context."""

    def __init__(self, name, procs=None):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        import oracle as O
        O.build()
        self.name = name
        self.procs = procs or max(1, os.cpu_count() or 1)
        self.ex = ProcessPoolExecutor(max_workers=self.procs, mp_context=mp.get_context("spawn"))
        list(self.ex.map(_oracle_warm, [name] * self.procs))
        _, mesh = workload(name)
        self.n_elem = mesh.n_elem

    def run(self, n_m, seed):
        """Wall time of the oracle on n_m seeded inner elements split over the processes."""
        rng = np.random.default_rng(seed)
        sel = np.sort(rng.choice(self.n_elem, size=min(n_m, self.n_elem), replace=False))
        parts = [p for p in np.array_split(sel, self.procs) if len(p)]
        t0 = time.perf_counter()
        res = list(self.ex.map(_oracle_rows, [(self.name, p) for p in parts]))
        dt = time.perf_counter() - t0
        return sum(r[0] for r in res), sum(r[1] for r in res), dt, len(parts)

    def calibrate(self, seconds):
        """Inner elements per call that keep every process busy for about `seconds`."""
        n_p, n_pp, dt, used = self.run(2 * self.procs, seed=12345)
        per_m = dt / 2.0
        return int(max(self.procs, min(self.n_elem, self.procs * seconds / max(per_m, 1e-4))))

    def close(self):
        self.ex.shutdown()


def cpu_baseline(mesh, w, seconds=10.0):
    pool = OraclePool(w.name)
    try:
        n_m = pool.calibrate(seconds)
        n_p, n_pp, dt, used = pool.run(n_m, seed=1)
    finally:
        pool.close()
    return {"value": round(n_p / dt, 1), "unit": "element pairs/s", "cores": used,
            "kind": "oracle",
            "sample": f"pairs (brute force), pattern and Algorithm-1 assembly of the rows of "
                      f"{n_m} seeded inner elements of {w.name} ({n_p} element pairs, {n_pp} "
                      f"quad-pt pairs) in {dt:.1f} s wall on {used} processes of the plain "
                      f"single-threaded FP64 oracle (os.cpu_count() = {os.cpu_count()})",
            "quad_pt_pairs_per_s": round(n_pp / dt, 1)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w, mesh = workload(args.workload)
    pool = OraclePool(w.name)
    try:
        n_m = pool.calibrate(args.ref_step_seconds)
        for k in range(args.warmup):
            pool.run(max(pool.procs, n_m // 8), seed=99 + k)
        times, pairs, pps = [], [], []
        for k in range(args.steps):
            n_p, n_pp, dt, used = pool.run(n_m, seed=k)
            times.append(dt)
            pairs.append(n_p)
            pps.append(n_pp)
    finally:
        pool.close()
    value = sum(pairs) / sum(times)
    sample = (f"each step: pairs (brute force), pattern and Algorithm-1 assembly of the rows of "
              f"{n_m} seeded inner elements of {w.name}, split over {used} processes of the "
              f"plain single-threaded FP64 oracle")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1),
            "unit": "element pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": describe(w, mesh),
                       "parallelism": f"{used} host processes (oracle)",
                       "l2": "not applicable (CPU)"},
            "quad_pt_pairs_per_s": round(sum(pps) / sum(times), 1),
            "cpu_baseline": {"value": round(value, 1), "unit": "element pairs/s", "cores": used,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": "element pairs/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    import torch
    from paper_2101_08825_gb300 import nl
    from paper_2101_08825_gb300.build import build
    build()
    w, mesh = workload(args.profile_workload)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    names = {"fp64": nl.NL_PREC_FP64, "fp32": nl.NL_PREC_FP32, "tf32": nl.NL_PREC_MIXED_TF32,
             "bf16": nl.NL_PREC_MIXED_BF16}
    if args.profile_precs:
        precs = tuple(names[x] for x in args.profile_precs.split(","))
    else:
        precs = (nl.NL_PREC_FP32, nl.NL_PREC_FP64) if args.profile_fp64 else (nl.NL_PREC_FP32,)
    for prec in precs:
        A, st = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, prec,
                               mindist_l2=bool(args.mindist_l2))
        print(json.dumps({"profile_case": w.name, "precision": prec, "pairs": st.n_pairs,
                          "point_pairs": st.n_point_pairs, "kernel_ms": st.ms_quad,
                          "assembly_ms": st.ms_assemble}))
    torch.cuda.synchronize()


def main():
    args = parse()
    if args.profile:
        run_profile_case(args)
        return
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        import torch
        torch.cuda.set_device(local)
        # all work on one non-default stream (the library captures its Krylov batches into
        # CUDA graphs on streams that can be captured)
        with torch.cuda.stream(torch.cuda.Stream()):
            out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
