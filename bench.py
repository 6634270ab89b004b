#!/usr/bin/env python
"""Benchmark of the nonlocal assembly + solve hot path on one GB300 (or N replicas).

One step = the whole path on the 2D workload at scale (Omega = (0,1)^2, h = 1/256,
141,512 P1 triangles with the layer, delta = 4h, eps = delta/5, L_max = 4, constant kernel,
vertices jittered by up to 0.1h, seed 0): element-pair search and CSR pattern, Algorithm 1
assembly, right-hand side with lifting (u = x^2 + y^2, f = -4) and BiCGStab solve to 1e-10,
with the mesh resident on the device.  The headline runs the FP32 point-pair path with the
solve in FP32 inside FP64 iterative refinement ("mixed"); the same step in FP64 is measured
next to it with the solution error of both against the manufactured solution.

Beside the headline the JSON line carries: the FP64 step, the roofline of the assembly kernel,
the public-API end-to-end rate from host buffers (e2e), a batching leg (128 small problems:
sequential assembly against one plan), a serving leg (the first --serve-requests requests of
the seeded stream, closed loop and then open loop at 70% load) and the oracle timed on the host
cores (cpu_baseline).

Output: one JSON line (rank 0).  --impl reference times the plain CPU oracle on a bounded
sample of the same workload instead.  Under torchrun every rank runs its own replica.
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
WORKLOAD = "c2_2d"

# DRAM traffic of the FP32 assembly kernel per element pair: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the current kernel version on a small case of the
# same dimension (profiles/k_quad_2d_fp32_c2_h128.md) divided by its element pairs.  Almost all
# of it is the block buffer, written once per pair, so it scales with the pairs of a launch.
# None: no capture of the current version (3D: profiles/k_quad_3d_fp32_c3.md holds the counters
# of the version before the saturating mollifier).
TRAFFIC_BYTES_PER_PAIR = {2: 35.66, 3: None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed FP64 steps beside the mixed ones (0 = leave the FP64 path out)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="requests of the seeded 512-request serving stream replayed by the "
                         "serving leg (0 = skip; 512 = the whole stream)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--batch-problems", type=int, default=128,
                    help="small problems of the batching leg (0 = skip)")
    ap.add_argument("--profile", action="store_true",
                    help="one pair build and one FP32 and one FP64 assembly of a small workload "
                         "(--profile-workload, default the 2D workload at h=1/128) for ncu, "
                         "then exit")
    ap.add_argument("--profile-workload", default="c2_2d_h128")
    ap.add_argument("--profile-fp64", type=int, default=1,
                    help="with --profile: also run the FP64 assembly (0 = FP32 only)")
    return ap.parse_args()


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
    n_omega = int(mesh.elem_in_omega.sum())
    kern = "constant" if w.kernel == 0 else "truncated Gaussian"
    return (f"{w.name}: Omega=(0,1)^{mesh.dim}, h=1/{round(1 / w.h)}, {mesh.n_elem} P1 {shape} "
            f"({n_omega} in Omega), delta={w.delta / w.h:g}h, eps=delta/{w.delta / w.eps:g}, "
            f"L_max={w.L_max}, {kern} kernel, jitter {w.jitter:g}h seed {w.seed}; "
            f"u=sum x_k^2; BiCGStab to 1e-10")


def u_exact(mesh):
    return (mesh.coords ** 2).sum(axis=0)  # u = x^2 + y^2 (+ z^2)


def l2_err_omega(mesh, u_h, rule):
    """||u - u_h||_{L2(Omega)} with the degree-5 rule per element (u = sum x_k^2)."""
    b, w = rule
    P = mesh.points()
    conn = mesh.conn[mesh.elem_in_omega.astype(bool)]
    V = P[conn]  # (ne, nv, dim)
    if mesh.dim == 2:
        vol = 0.5 * np.abs((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1]) -
                           (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    else:
        vol = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])) / 6.0
    X = np.einsum("qv,evk->eqk", b, V)
    uh = np.einsum("qv,ev->eq", b, u_h[conn])
    d = (X ** 2).sum(-1) - uh
    return float(math.sqrt(np.sum(vol[:, None] * w[None, :] * d * d)))


# ---- our implementation ----------------------------------------------------------------------

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
    w, mesh = workload(args.workload)
    delta, eps, L_max = w.delta, w.eps, w.L_max
    g = u_exact(mesh)
    f_const = -2.0 * mesh.dim
    rule = nl.nl_quad_rule(mesh.dim)
    flush = torch.empty(int(256 * 2 ** 20) // 4, dtype=torch.float32, device="cuda")

    dmesh = nl.mesh_from(mesh)

    def step(prec, keep=False):
        p = nl.nl_pairs_build(dmesh, delta, eps)
        A, st = nl.nl_assemble(dmesh, p, delta, eps, L_max, precision=prec)
        b = nl.nl_rhs(dmesh, A, g, f_const=f_const)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        u, it, rr, _ = nl.nl_solve(A, b, g, solver=1, rtol=1e-10, max_iter=20000,
                                   precision=nl.NL_PREC_FP32 if prec != nl.NL_PREC_FP64 else nl.NL_PREC_FP64)
        t1.record(stream)
        t1.synchronize()
        res = dict(st=st, u=u, it=it, rr=rr, solve_ms=t0.elapsed_time(t1))
        if keep:
            res["A"] = A.export()
        return res

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize()
        times, solve_ms, kern_ms, last = [], [], [], None
        launches0 = nl.lib().nl_launch_count()
        for _ in range(steps):
            flush.zero_()  # L2 flush (256 MB > 129 MB L2) between steps, outside the timing
            barrier(world)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step(prec)
            e1.record(stream)
            e1.synchronize()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            solve_ms.append(last["solve_ms"])
            kern_ms.append(last["st"].ms_assemble)
        launches = nl.lib().nl_launch_count() - launches0
        return times, solve_ms, kern_ms, last, launches

    # mixed headline (timed with clock sampling)
    clk = ClockSampler(local)
    clk.start()
    times, solve_ms, kern_ms, last, launches = timed(nl.NL_PREC_FP32, args.steps, args.warmup)
    clocks = clk.stop()
    ms = statistics.mean(times)
    ms_max = allmax(world, ms)
    st = last["st"]
    n_pairs, n_pp = st.n_pairs, st.n_point_pairs
    value = world * n_pairs / (ms_max / 1e3)
    err_mixed = l2_err_omega(mesh, last["u"], rule)

    # FP64 path, same step (--fp64-steps 0 leaves it out, e.g. for the 3D h = 1/32 workload,
    # whose FP64 assembly takes minutes)
    fp64 = None
    if args.fp64_steps > 0:
        t64, s64, k64, last64, _ = timed(nl.NL_PREC_FP64, args.fp64_steps, 1)
        ms64 = statistics.mean(t64)
        err64 = l2_err_omega(mesh, last64["u"], rule)
        # matrix difference mixed vs FP64 (one extra untimed assembly each)
        r32 = step(nl.NL_PREC_FP32, keep=True)["A"]
        r64 = step(nl.NL_PREC_FP64, keep=True)["A"]
        a_rel = float(np.linalg.norm(r32 - r64) / np.linalg.norm(r64))
        fp64 = {"dtype": "f64", "ms_per_step": round(ms64, 3),
                "value": round(world * n_pairs / (ms64 / 1e3), 1),
                "assembly_kernel_ms": round(statistics.mean(k64), 3), "l2_err_omega": err64}

    # roofline of the dominant kernel (FP32 assembly kernel): algorithmic flops per launch;
    # the band count comes from one extra untimed launch with NL_QUAD_COUNT_BAND
    kern_avg = statistics.mean(kern_ms)
    pb = nl.nl_pairs_build(dmesh, delta, eps)
    _, stb = nl.nl_assemble(dmesh, pb, delta, eps, L_max, precision=nl.NL_PREC_FP32,
                            count_band=True)
    flops = roofline_flops(mesh.dim, stb)
    peak_tflops = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x 2 flops x max SM clock
    achieved = flops / (kern_avg / 1e3) / 1e12
    if fp64 is not None:
        # the FP64 assembly kernel against the FP64 pipe: same algorithmic count with the FP64
        # launch's own evaluated point pairs (its band pairs: those of the FP32 count launch,
        # identical up to the rounding of r at the band edges); peak = the measured FP64 FMA
        # chain of this GPU model, 1.19 TFLOP/s
        st64 = last64["st"]
        f64_flops = float(st64.n_eval_point_pairs * (14 if mesh.dim == 2 else 19)
                          + max(0, stb.n_band_point_pairs) * 15)
        k64_avg = statistics.mean(k64)
        fp64["roofline"] = {"bound": "fp64 pipe", "achieved": round(f64_flops / (k64_avg / 1e3) / 1e12, 4),
                            "peak": 1.19, "unit": "TFLOP/s",
                            "frac": round(f64_flops / (k64_avg / 1e3) / 1.19e12, 4),
                            "kernel": f"k_quad<{mesh.dim},double,{w.kernel}>"}
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 1),
            "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
            "traffic": (round(TRAFFIC_BYTES_PER_PAIR[mesh.dim] * n_pairs)
                        if TRAFFIC_BYTES_PER_PAIR.get(mesh.dim) else None),
            "kernel": f"k_quad<{mesh.dim},float,{w.kernel}>", "flops_per_launch": flops,
            "kernel_ms_avg": round(kern_avg, 3)}

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "element pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": describe(w, mesh),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "working set > L2 and a 256 MB L2 flush between steps"},
        "quad_pt_pairs_per_s": round(world * n_pp / (ms_max / 1e3), 1),
        "assembly_kernel": {"ms": round(kern_avg, 3),
                            "element_pairs_per_s": round(n_pairs / (kern_avg / 1e3), 1),
                            "quad_pt_pairs_per_s": round(n_pp / (kern_avg / 1e3), 1)},
        "counts": {"element_pairs": n_pairs, "quad_pt_pairs": n_pp, "items": st.n_items,
                   "fp64_rechecks": st.n_exact_checks,
                   "evaluated_point_pairs": stb.n_eval_point_pairs,
                   "band_point_pairs": stb.n_band_point_pairs,
                   "closed_form_items": stb.n_closed_items},
        "fp64": fp64,
        "mixed": {"l2_err_omega": err_mixed,
                  "A_rel_frobenius_vs_fp64": a_rel if fp64 else None,
                  "solve_iters": last["it"],
                  "speedup_vs_fp64": round(ms64 / ms, 2) if fp64 else None},
        "solve_ms": {"p50": round(float(np.percentile(solve_ms, 50)), 3),
                     "p99": round(float(np.percentile(solve_ms, 99)), 3)},
        "roofline": roof,
        "gpu_launches": int(launches),  # this library's kernels in the whole timed region
        "gpu_launches_per_step": int(launches / max(1, args.steps)),
        "clocks": clocks,
    }
    if not args.no_e2e:
        out["e2e"] = e2e_ours(args, mesh, w, g, f_const, stream, world)
    if args.batch_problems > 0:
        out["batching"] = run_batching(args)
    if args.serve_requests > 0:
        out["serving"] = run_serving(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(mesh, w, seconds=15.0)
    return out


def roofline_flops(dim, st):
    """Algorithmic flops of one assembly launch (FMA = 2), per point pair of the method's
    double sum as written (eqs. J21Nr, J22Nr): the distance and r^2 (2D 5, 3D 8), the weight
    w_x w_y C mu (2), the rank-one update of the local block over the nodes of m (2D 6, 3D 8)
    and the self-term sum (1): 14 (2D) / 19 (3D); per band point pair additionally r (1),
    s = (delta - r)/eps (2) and xi(s) by Horner (12): 15.  Counted over the point pairs the
    kernel evaluates one by one; sub-elements summed in closed form are not counted.  (The
    kernel itself hoists the contraction with m's basis out of the loop over outer points and
    executes 11 (2D) / 16 (3D) flops per point pair for the same sums.)"""
    ev = max(0, int(getattr(st, "n_eval_point_pairs", 0) or 0))
    band = max(0, int(getattr(st, "n_band_point_pairs", 0) or 0))
    per_pp = 14 if dim == 2 else 19
    return float(ev * per_pp + band * 15)


def e2e_ours(args, mesh, w, g, f_const, stream, world):
    """Public-API step from pinned host buffers: mesh upload, pairs, assembly, right-hand
    side, solve and the solution read back, all inside the timed region."""
    import torch
    from paper_2101_08825_gb300 import nl

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    coords, conn = pinned(mesh.coords), pinned(mesh.conn)
    eio, nf, gp = pinned(mesh.elem_in_omega), pinned(mesh.node_free), pinned(g)
    times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dm = nl.nl_mesh_create(mesh.dim, coords, conn, eio, nf)
        p = nl.nl_pairs_build(dm, w.delta, w.eps)
        A, st = nl.nl_assemble(dm, p, w.delta, w.eps, w.L_max, precision=nl.NL_PREC_FP32)
        b = nl.nl_rhs(dm, A, gp, f_const=f_const)
        u, it, rr, _ = nl.nl_solve(A, b, gp, solver=1, rtol=1e-10, max_iter=20000,
                                   precision=nl.NL_PREC_FP32)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
        n_pairs = st.n_pairs
    ms = allmax(world, statistics.mean(times))
    h2d = coords.nbytes + conn.nbytes + eio.nbytes + nf.nbytes + 2 * gp.nbytes
    d2h = u.nbytes
    return {"value": round(world * n_pairs / (ms / 1e3), 1), "unit": "element pairs/s",
            "ms_per_step": round(ms, 3), "h2d_bytes_per_step": int(h2d),
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
                               jitter=0.1, seed=i)

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
        return dict(p50=p50, p99=p99, sps=sps, wall=wall, failed=len(results) - len(ok),
                    pairs=sum(r.n_pairs for r in ok), lat=lat)

    sat = replay([0.0] * len(reqs))
    rate = 0.7 * sat["sps"]
    gaps = np.diff([0.0] + [r.arrival_s for r in reqs])
    scale = (1.0 / rate) / max(float(np.mean(gaps)), 1e-9) if rate > 0 else 0.0
    arrivals = np.cumsum(gaps * scale)
    ol = replay(list(arrivals))
    return {"requests": len(reqs), "slots": args.serve_slots, "budget_bytes": budget,
            "saturation": {"solves_per_s": round(sat["sps"], 3),
                           "element_pairs_per_s": round(sat["pairs"] / sat["wall"], 1),
                           "failed": sat["failed"]},
            "open_loop": {"arrival_rate_per_s": round(rate, 3), "p50_ms": round(ol["p50"], 2),
                          "p99_ms": round(ol["p99"], 2), "solves_per_s": round(ol["sps"], 3),
                          "max_latency_ms": round(max(ol["lat"]), 2) if ol["lat"] else None,
                          "failed": ol["failed"]},
            "sample": f"first {len(reqs)} of the 512-request seeded stream (seed 0); phase 2 "
                      f"arrivals = the stream's exponential gaps rescaled to 70% of phase 1's "
                      f"throughput"}


# ---- the oracle on a bounded sample ------------------------------------------------------------

def oracle_sample(mesh, w, n_m, seed=0):
    """Times the oracle's pair search, pattern and Algorithm 1 assembly for the rows of n_m
    seeded inner elements of the workload; returns (pairs, point pairs, seconds)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    mask = np.zeros(mesh.n_elem, np.uint8)
    mask[rng.choice(mesh.n_elem, size=n_m, replace=False)] = 1
    om = O.OMesh(mesh)
    t0 = time.perf_counter()
    off, pl = O.pairs(om, w.delta, w.eps, m_mask=mask)
    rp, col = O.csr(om, off, pl)
    vals, st = O.assemble(om, off, pl, rp, col, w.delta, w.eps, w.L_max, w.L_min, w.kernel,
                          m_mask=mask)
    dt = time.perf_counter() - t0
    return len(pl), st.n_point_pairs, dt


def cpu_baseline(mesh, w, seconds=15.0):
    import oracle as O
    O.build()
    n_p, n_pp, dt = oracle_sample(mesh, w, 8)
    n_m = int(max(8, min(mesh.n_elem, 8 * seconds / max(dt, 1e-3))))
    n_p, n_pp, dt = oracle_sample(mesh, w, n_m, seed=1)
    return {"value": round(n_p / dt, 1), "unit": "element pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"pairs, pattern and Algorithm-1 assembly of the rows of {n_m} seeded "
                      f"inner elements of the workload ({n_p} element pairs, {n_pp} quad-pt "
                      f"pairs, {dt:.1f} s single-threaded FP64)",
            "quad_pt_pairs_per_s": round(n_pp / dt, 1)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle as O
    O.build()
    w, mesh = workload(args.workload)
    n_p, n_pp, dt = oracle_sample(mesh, w, 4)
    n_m = int(max(4, min(mesh.n_elem, 4 * 6.0 / max(dt, 1e-3))))  # ~6 s per step
    for _ in range(args.warmup):
        oracle_sample(mesh, w, max(4, n_m // 8), seed=99)
    times, pairs = [], []
    for k in range(args.steps):
        n_p, n_pp, dt = oracle_sample(mesh, w, n_m, seed=k)
        times.append(dt)
        pairs.append(n_p)
    value = sum(pairs) / sum(times)
    sample = (f"each step: pairs, pattern and Algorithm-1 assembly of the rows of {n_m} seeded "
              f"inner elements of {w.name}")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1),
            "unit": "element pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": describe(w, mesh), "parallelism": "single CPU core (oracle)",
                       "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": round(value, 1), "unit": "element pairs/s", "cores": 1,
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
    precs = (nl.NL_PREC_FP32, nl.NL_PREC_FP64) if args.profile_fp64 else (nl.NL_PREC_FP32,)
    for prec in precs:
        A, st = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max, w.L_min, w.kernel, prec)
        print(json.dumps({"profile_case": w.name, "precision": prec, "pairs": st.n_pairs,
                          "point_pairs": st.n_point_pairs, "kernel_ms": st.ms_assemble}))
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
