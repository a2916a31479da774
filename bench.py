"""Benchmark of the walk-on-spheres / local-BIE DtN hot path on one GB300.

A step is one pass of the whole path over the unit-ball workload (2000 patches
on a Fibonacci sphere, a = 0.1, 128 panels and 512 hemisphere nodes per patch,
4096 walks per node, epsilon 1e-4, degree-8 random harmonic data): patch setup,
walks and their estimates, assembly, batched LU with refinement, the panel
gather of the patch cover and the potential at 1e5 targets.  Prints one JSON
line.  `--impl reference` times the FP64 CPU oracle instead, on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "WOS walk-steps/s & DtN patches/s vs plain FP64 path; p50/p99 query latency"
N_TARGETS = 100_000
# algorithmic thread-level ALU operations of the FP32 walk in the ball region.
# Per step: a third of a Philox4x32-10 block (10 rounds x (2 wide multiplies +
# 2 xor3 + 2 key adds) / 3 = 20) and of its split into six 21-bit fields
# (10 / 3 = 3), two uniforms (one integer add each) 2, direction (z, 1 - z^2,
# sqrt, azimuth and sincos) 8, distance to the sphere from the centre-relative
# position (|x|^2, sqrt, R - |x|) 6, shell test and step count 2, position
# update 4: 45.  Per walk: the score, projection onto the sphere 8 + degree-8
# harmonic data by the scaled solid-harmonic recurrence (36 off-diagonal (l, m)
# pairs x (3 recurrence + 2 accumulate) + 9 x 4 for the powers (x + iy)^m and
# the per-m sums) 216 + fixed-point terms 11: 235.
OPS_PER_STEP = 45
OPS_PER_WALK = 235
# The same count for the walk in the wire region (box minus 200 boxes), as a
# lower bound: the step without the ball distance (45 - 6 = 39), the outer box
# (6 differences, 5 minima) 11, the lookup-grid cell (3 x (difference, scale,
# floor, conversion, two clamps) + index) 20, the cell's cap 2, and 17 more per
# listed box (3 x (2 differences, 2 maxima), |e|^2, sqrt, minimum): 72 + 17 per
# listed box.  A counting build of the walk kernel on the wire workload (64 and
# 256 patches) saw 1.66 listed boxes per distance evaluation, so 72 + 28 = 100.
# Per walk: nearest point on the outer box 12, the grid cell 20, point-source
# data (3 differences, |r|^2, reciprocal square root, scale) 8, fixed-point
# terms 11, the listed boxes' nearest points counted as none: 51.
OPS_PER_STEP_WIRES = 100
OPS_PER_WALK_WIRES = 51
# DRAM bytes of the walk kernel per hemisphere node (node coordinates and the
# per-node sums): an ncu capture of the 64-patch unit-ball case read and wrote
# 1,768,704 bytes for its 32,768 nodes; scaled to the launch's nodes
DRAM_BYTES_PER_NODE = 1772800 / 32768   # ncu, 64-patch capture (32,768 nodes), read + write
# the same capture's issue-slot utilisation and active lanes per warp instruction
NCU_ISSUE_ACTIVE = 0.765        # ncu, same capture: issue slots busy
NCU_LANES_PER_INST = 30.65      # ncu, same capture: active lanes per warp instruction
SM_COUNT = 152
LANES_PER_SM = 128


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self):
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"dtn_bench_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(int(os.environ.get("LOCAL_RANK", "0"))) and parts[0] != "0":
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_patch_base(rank: int, n_patches: int) -> int:
    """RNG patch-id base of a replica: ranks solve independent copies with disjoint ids."""
    return rank * n_patches


def reduce_max(value: float, dist, device) -> float:
    """Max over ranks (the slowest replica sets the whole-job time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


ARGS = None


def make_workload():
    """The unit-ball workload (2000 patches, 4096 walks); --patches/--walks shrink it
    for profiler captures only."""
    n = ARGS.patches if ARGS is not None else 2000
    w = ARGS.walks if ARGS is not None else 4096
    wl = W.unit_ball(n_patches=n, walks=w)
    targets = W.targets_in_ball(N_TARGETS, 1.0, 0.05, seed=3)
    return wl, targets


# ------------------------------------------------------------------ reference arm: the oracle

def run_reference(args):
    import oracle as O
    wl, targets = make_workload()
    b = wl.batch
    o = O.wos_opts(eps=wl.epsilon, seed=wl.seed, stream=O.STREAM_F64)
    times = []
    sample = 1   # patches per step: a bounded sample of the same workload

    def one(k):
        i = k % b.n
        t0 = time.perf_counter()
        O.solve_patch(wl.geometry, wl.data, b.centers[i], float(b.radius[i]), int(b.n_theta[i]),
                      int(b.n_phi[i]), int(b.n_rings[i]), int(b.n_sectors[i]), int(b.walks[i]), i, o,
                      rtol=1e-12)
        return time.perf_counter() - t0

    for k in range(args.warmup):
        one(k)
    for k in range(args.steps):
        times.append(one(args.warmup + k))
    sec = sum(times) / len(times)
    value = sample / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "patches/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "patches_per_step": sample, "walks_per_node": int(b.walks[0]),
                   "nodes_per_patch": int(b.n_theta[0] * b.n_phi[0]), "panels_per_patch": int(b.n_rings[0] * b.n_sectors[0])},
        "cpu_baseline": {"value": value, "unit": "patches/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{sample} patch per step of the 2000-patch unit-ball workload, full walks"},
        "e2e": {"value": value, "unit": "patches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm

def cpu_baseline_sample(wl):
    """The oracle on a bounded sample on this host's cores: 2 patches with every
    core, then 1 patch on one core."""
    import oracle as O
    b = wl.batch
    o = O.wos_opts(eps=wl.epsilon, seed=wl.seed, stream=O.STREAM_F64)

    def run(n):
        t0 = time.perf_counter()
        steps = 0
        for i in range(n):
            r = O.solve_patch(wl.geometry, wl.data, b.centers[i], float(b.radius[i]), int(b.n_theta[i]),
                              int(b.n_phi[i]), int(b.n_rings[i]), int(b.n_sectors[i]), int(b.walks[i]), i, o,
                              rtol=1e-12)
            steps += r["steps"]
        dt = time.perf_counter() - t0
        return n / dt, steps / dt

    cores = O.num_threads()
    v, sps = run(2)
    O.set_num_threads(1)
    try:
        v1, sps1 = run(1)
    finally:
        O.set_num_threads(cores)
    return {"value": v, "unit": "patches/s", "cores": cores, "kind": "oracle",
            "sample": "first 2 patches of the workload, full walks, assembly and solve",
            "walk_steps_per_s": sps,
            "one_core": {"value": v1, "unit": "patches/s", "cores": 1, "walk_steps_per_s": sps1,
                         "sample": "first patch of the workload, full walks, assembly and solve"}}


def run_serving(dtn, n_queries=600, seed=7, loads=(0.5, 0.8), n_targets=100_000):
    """Continuous-batching server on the 200-wire geometry (resident on the device).

    Each query asks for the Neumann data at 1..4096 boundary points (log-uniform),
    served by wire-face patches taken in turn until their panels cover that many
    points, with 1024..16384 walks per hemisphere point (log-uniform).  The queries
    are submitted first all at once (saturated throughput), then as Poisson
    arrivals at each of `loads` x that rate (p50/p99 submit-to-result latency).
    Admission by device memory: the server's budget is the free device memory at
    its creation less a reserve.  Three slots; each batch's walk launch may fill
    the GPU (the lowest latency), and the saturated run is repeated with the
    slots sharing the SMs.  Then the potential at 10^5 targets outside the wires,
    by the integral representation over all served panels."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    wl = W.wires(n_patches=4096, walks=2048)
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=wl.epsilon, seed=wl.seed)
    panels = (b.n_rings * b.n_sectors).astype(np.int64)
    queries, start, points = [], 0, 0
    for _ in range(n_queries):
        want = int(np.exp(rng.uniform(0.0, np.log(4096.0))))
        idx = []
        got = 0
        while got < want:
            idx.append(start % b.n)
            got += int(panels[start % b.n])
            start += 1
        idx = np.asarray(idx)
        points += want
        walks = int(np.exp(rng.uniform(np.log(1024.0), np.log(16384.0))))
        queries.append(dict(centers=b.centers[idx], radius=b.radius[idx], n_theta=b.n_theta[idx],
                            n_phi=b.n_phi[idx], n_rings=b.n_rings[idx], n_sectors=b.n_sectors[idx],
                            walks=np.full(len(idx), walks, np.int64), patch_ids=idx.astype(np.uint32)))

    def saturated(srv):
        srv.submit(**queries[0])   # warm-up (first-use costs)
        srv.drain()
        t0 = time.perf_counter()
        for q in queries:
            srv.submit(**q)
        srv.drain()
        return time.perf_counter() - t0

    split = dtn.Server(g, opts, max_inflight=3, max_batch_patches=1024, split_sms=True)
    t_split = saturated(split)
    split_info = split.stats()
    split.close()
    srv = dtn.Server(g, opts, max_inflight=3, max_batch_patches=1024, split_sms=False)
    t_sat = saturated(srv)
    poisson = []
    served = []
    for load in loads:
        rate = load * n_queries / t_sat
        gaps = rng.exponential(1.0 / rate, n_queries)
        tickets = []
        t0 = time.perf_counter()
        for q, gap in zip(queries, gaps):
            time.sleep(gap)
            tickets.append(srv.submit(**q))
        srv.drain()
        t_poisson = time.perf_counter() - t0
        served = [srv.poll(t) for t in tickets]
        lat = np.array([r["latency_s"] for r in served]) * 1e3
        poisson.append({"offered_load": load, "offered_queries_per_s": rate, "queries_per_s": n_queries / t_poisson,
                        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                        "queries_not_ok": sum(1 for r in served if r["status"] != 0)})
    info = srv.stats()
    srv.close()
    # potential at targets outside the wires, over every served panel: the panel
    # geometry and data of the served patches (no walks), their served Neumann data
    allq = {k: np.concatenate([q[k] for q in queries]) for k in queries[0]}
    hb = dtn.HostBatch(allq["n_theta"], allq["n_phi"], allq["n_rings"], allq["n_sectors"], allq["walks"],
                       patch_ids=allq["patch_ids"])
    geo = dtn.alloc_result(hb)
    geo["u_gamma_mean"].zero_()
    dtn.solve_patches(g, allq["centers"], allq["radius"], hb, dtn.solve_opts(prec=dtn.PREC_MIXED, u_provided=True),
                      result=geo)
    q_served = torch.from_numpy(np.concatenate([r["neumann"] for r in served])).cuda()
    boxes = np.asarray(wl.geometry.boxes)
    tg = W.points_in_box(4 * n_targets, (0.0, 0.0, 0.0), (64.0, 64.0, 16.0), 0.05, seed=11)
    outside = np.ones(len(tg), bool)
    for bx in boxes:
        outside &= ~np.all((tg >= bx[:3] - 0.05) & (tg <= bx[3:] + 0.05), axis=1)
    tgt = torch.from_numpy(np.ascontiguousarray(tg[outside][:n_targets])).cuda()
    u_t = torch.empty(tgt.shape[0], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(3):
        if k == 2:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        dtn.eval_potential(g, geo["colloc_xyz"], geo["normals"], geo["areas"], q_served, geo["dirichlet"], tgt,
                           prec=dtn.PREC_MIXED, out=u_t)
    e1.record(stream)
    e1.synchronize()
    pot_ms = e0.elapsed_time(e1)
    n_pan = int(q_served.shape[0])
    return {"geometry": "box [0,64]^2x[0,16] minus 200 wires", "queries": n_queries, "points": points,
            "patches": int(len(allq["radius"])), "panels": n_pan,
            "walks_per_node": "1024..16384 log-uniform per query", "slots": 3,
            "saturated_queries_per_s": n_queries / t_sat, "saturated_patches_per_s": len(allq["radius"]) / t_sat,
            "poisson": poisson,
            "admission": {"rule": "free device memory at creation less max(1 GiB, 5%); slot workspaces plus "
                                  "each starting batch's workspace within it",
                          "budget_bytes": info["budget_bytes"], "peak_held_bytes": info["peak_held_bytes"],
                          "rejected": info["rejected"]},
            "device_overlap": {"batches": info["batches"], "max_concurrent": info["max_concurrent"],
                               "busy_ms": info["busy_ms"], "overlap_ms": info["overlap_ms"]},
            "split_sms": {"saturated_queries_per_s": n_queries / t_split, "batches": split_info["batches"],
                          "max_concurrent": split_info["max_concurrent"], "busy_ms": split_info["busy_ms"],
                          "overlap_ms": split_info["overlap_ms"]},
            "potential": {"targets": int(tgt.shape[0]), "panels": n_pan, "ms": pot_ms,
                          "targets_per_s": tgt.shape[0] / (pot_ms / 1e3),
                          "pair_terms_per_s": tgt.shape[0] * n_pan / (pot_ms / 1e3)}}


def run_single_point(dtn, n_points=256, ng=20, walks=1000):
    """The single-point method (Sec. 4.1) on the paper's two flat-boundary tests,
    20 x 20 hemisphere and ring rules, 1000 walks per node (4e5 paths per point,
    as in Tables 1 and 5), epsilon 1e-5, FP32 walks.  Test 1: the half space
    above z = 0 with a unit charge at depth 1, a = 0.5, exact q = 0.71554 on the
    circle of radius 0.5.  Test 4: outside the thin disk of radius 1 at potential
    1, a = 0.4, exact density 0.735105 on the circle of radius 0.5 (the paper
    times one point: 1218 s of CPU for 4e5 paths).  Device time of one call with
    CUDA events, for n_points points on that circle and for the single point."""
    import torch
    ang = 2 * np.pi * np.arange(n_points) / n_points
    circle = np.stack([0.5 * np.cos(ang), 0.5 * np.sin(ang), np.zeros(n_points)], 1)
    opts = dtn.solve_opts(prec=dtn.PREC_MIXED, epsilon=1e-5, seed=0)
    stream = torch.cuda.current_stream()
    out = {}
    for name, (geom, data), a, exact in (("test1_half_space", W.half_space_charge(), 0.5, 0.71554),
                                         ("test4_thin_disk", W.thin_disk(), 0.4, 0.735105)):
        g = dtn.Geometry.from_spec(geom).set_data_spec(data)
        res = {"a": a, "exact": exact}
        for tag, pts in (("points", circle), ("one_point", np.array([[-0.5, 0.0, 0.0]]))):
            xd = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
            for k in range(3):
                if k == 2:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                r = dtn.single_point_neumann(g, xd, a, ng, ng, 1e-6 * a, walks, opts)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            q = r["q"].cpu().numpy()
            se = r["se"].cpu().numpy()
            paths = len(pts) * ng * ng * walks
            res[tag] = {"n": len(pts), "ms": ms, "paths_per_s": paths / (ms / 1e3),
                        "q_mean": float(q.mean()), "rel_err_of_mean": float(q.mean() / exact - 1.0),
                        "mean_se": float(se.mean()), "max_abs_z": float(np.max(np.abs(q - exact) / se))}
        out[name] = res
    out["setup"] = f"{ng}x{ng} hemisphere and ring rules, {walks} walks per node, eps 1e-5, FP32 walks, delta 1e-6 a"
    return out


def run_potential_fmm(dtn, n_panels=1_000_000, n_targets=1_000_000, order=10, theta=0.6, direct=True):
    """Potential by the fast multipole method (Sec. 6) against the direct sum:
    n_panels equal-area panels of the unit sphere (Fibonacci lattice) with
    seeded N(0, 1) Neumann and Dirichlet values, n_targets uniform targets in
    the ball, all resident on the device.  Wall time of one call (the FMM
    synchronises: its trees and traversal are built level by level), best of 3
    after 2 warm-up calls; the direct FP32-pair sum is timed once with CUDA events."""
    import torch
    y, nrm, ar = W.sphere_panels(n_panels)
    q, g = W.panel_values(n_panels)
    t = W.targets_in_ball(n_targets, 1.0, 0.0, seed=4)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (y, nrm, ar, q, g, t)]
    geom = dtn.Geometry(dtn.GEOM_BALL_INTERIOR, radius=1.0).set_dirichlet(dtn.DATA_CONSTANT, constant=0.0)
    o = dtn.fmm_opts(order=order, theta=theta, leaf_sources=128, leaf_targets=64)
    times = []
    for k in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, st = dtn.eval_potential_fmm(geom, *dev, opts=o, want_stats=True)
        torch.cuda.synchronize()
        if k >= 2:
            times.append(time.perf_counter() - t0)
    fmm_s = min(times)
    out = {"panels": n_panels, "targets": n_targets, "order": order, "theta": theta,
           "leaf_sources": o.leaf_sources, "leaf_targets": o.leaf_targets, "fmm_ms": fmm_s * 1e3,
           "pair_terms_per_s_equivalent": n_panels * n_targets / fmm_s, "stats": st,
           "data": "synthetic: Fibonacci-sphere panels, N(0,1) values, uniform targets in the ball"}
    if direct:
        # FP64 direct sum at every 50th target: the accuracy of this setting
        samp = torch.arange(0, n_targets, 50, device="cuda")
        ref = dtn.eval_potential(geom, *dev[:5], dev[5][samp], prec=dtn.PREC_FP64)
        out["rel_l2_vs_fp64_direct_sample"] = float((u[samp] - ref).norm() / ref.norm())
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ud = dtn.eval_potential(geom, *dev, prec=dtn.PREC_MIXED)
        e1.record(stream)
        e1.synchronize()
        direct_s = e0.elapsed_time(e1) / 1e3
        out.update({"direct_ms": direct_s * 1e3, "speedup_vs_direct": direct_s / fmm_s,
                    "rel_l2_fp32_direct_vs_fp64_sample": float((ud[samp] - ref).norm() / ref.norm())})
    return out


def run_batch_leg(dtn, wl, ops_step, ops_walk, reps=2, n_plain=8, capture=False, exact_ops=True):
    """One workload solved in one mixed-precision call (captured as a CUDA graph
    and replayed when `capture`), walk launch autotuned: device time of the call
    (CUDA events, mean of `reps` after a warm-up), patches/s, walk-steps/s from
    a separate call with stage events, the walk kernel's ALU roofline, and the
    plain FP64 path (FP64 walks, assembly and LU, one patch per launch) on the
    first n_plain patches."""
    import torch
    b = wl.batch
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks)
    centers = torch.from_numpy(b.centers).cuda()
    radius = np.ascontiguousarray(b.radius)
    stream = torch.cuda.current_stream()
    base = dict(prec=dtn.PREC_MIXED, epsilon=wl.epsilon, seed=wl.seed)
    tuning = dtn.autotune_walks(g, centers, radius, hb, dtn.solve_opts(**base))
    res = dtn.alloc_result(hb)
    # walk time and walk-steps from one call with stage events (not captured)
    dtn.solve_patches(g, centers, radius, hb, dtn.solve_opts(record_stages=True, **base), result=res)
    torch.cuda.synchronize()
    walk_ms = g.stage_times()[1]
    steps = int(res["gamma_steps"].sum().item())
    status_ok = bool((res["patch_status"] == 0).all().item())
    o = dtn.solve_opts(graph_capture=capture, **base)
    times = []
    for k in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dtn.solve_patches(g, centers, radius, hb, o, result=res)
        e1.record(stream)
        e1.synchronize()
        if k:   # the first call captures (or warms up)
            times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    walks = int(np.sum(b.walks * (b.n_theta * b.n_phi)))
    peaks = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT * LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = (steps * ops_step + walks * ops_walk) / (walk_ms / 1e3) / 1e12
    # the plain FP64 path, one patch per launch
    o64 = dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=wl.epsilon, seed=wl.seed)
    hb1 = [dtn.HostBatch(b.n_theta[i:i + 1], b.n_phi[i:i + 1], b.n_rings[i:i + 1], b.n_sectors[i:i + 1],
                         b.walks[i:i + 1], patch_id_base=i) for i in range(n_plain)]
    r1 = [dtn.alloc_result(h) for h in hb1]
    dtn.solve_patches(g, centers[0:1], radius[0:1], hb1[0], o64, result=r1[0])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n_plain):
        dtn.solve_patches(g, centers[i:i + 1], radius[i:i + 1], hb1[i], o64, result=r1[i])
    e1.record(stream)
    e1.synchronize()
    plain = n_plain / (e0.elapsed_time(e1) / 1e3)
    value = b.n / (ms / 1e3)
    return {"workload": wl.name, "patches": b.n,
            "nodes_per_patch": sorted(set(int(v) for v in b.n_theta * b.n_phi)),
            "panels_per_patch": [int(np.min(b.n_rings * b.n_sectors)), int(np.max(b.n_rings * b.n_sectors))],
            "walks_per_node": int(b.walks[0]), "graph_capture": capture, "ms": ms, "patches_per_s": value,
            "walk_ms": walk_ms, "walk_steps": steps, "walk_steps_per_s": steps / (walk_ms / 1e3),
            "status_ok": status_ok, "walk_tuning": tuning,
            "roofline": {"bound": "alu", "kernel": "wos_kernel_f32", "achieved": achieved, "peak": alu_peak,
                         "unit": "Tops/s", "frac": achieved / alu_peak, "ops_per_walk_step": ops_step,
                         "ops_per_walk": ops_walk,
                         "ops_basis": "algorithmic count" if exact_ops else
                         "algorithmic count with the measured mean of 1.66 listed obstacle boxes per step"},
            "fp64_path": {"value": plain, "unit": "patches/s", "sample": f"first {n_plain} patches, one per launch",
                          "speedup": value / plain}}


def run_second_kind(dtn, g, centers, radius, hb, opts_kw):
    """The unit-ball workload solved with the second-kind local BIE (Eq. bw55-bw59,
    cap patches: (1/2 I - D) q = b, mixed precision): device time of the
    solve call (walks, assembly, solve) with CUDA events, best of 2 after one
    warm-up."""
    import torch
    stream = torch.cuda.current_stream()
    res = dtn.alloc_result(hb)
    opts = dtn.solve_opts(bie_kind=1, **opts_kw)
    best = None
    for k in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dtn.solve_patches(g, centers, radius, hb, opts, result=res)
        e1.record(stream)
        e1.synchronize()
        if k:
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
    n = int(centers.shape[0])
    return {"patches": n, "ms": best, "patches_per_s": n / (best / 1e3),
            "status_ok": bool((res["patch_status"] == 0).all().item()),
            "setup": "unit-ball workload, second-kind BIE on the caps, mixed precision"}


def run_ours(args):
    import torch
    import paper_1210_1491_gb300 as dtn

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl, targets = make_workload()
    b = wl.batch
    # replicas only: every rank solves its own copy with its own patch ids
    hb = dtn.HostBatch(b.n_theta, b.n_phi, b.n_rings, b.n_sectors, b.walks,
                       patch_id_base=replica_patch_base(rank, b.n))
    g = dtn.Geometry.from_spec(wl.geometry).set_data_spec(wl.data)
    prec = dtn.PREC_MIXED if args.prec == "mixed" else dtn.PREC_FP64
    opts = dtn.solve_opts(prec=prec, epsilon=wl.epsilon, seed=wl.seed, record_stages=True)
    dev = torch.device("cuda", local)
    centers = torch.from_numpy(b.centers).to(dev)
    radius = np.ascontiguousarray(b.radius)   # per-patch shape parameter (host)
    tgt = torch.from_numpy(targets).to(dev)
    res = dtn.alloc_result(hb)
    owner = torch.from_numpy(np.repeat(np.arange(b.n), int(b.n_rings[0] * b.n_sectors[0]))).to(dev)
    u_out = torch.empty(N_TARGETS, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    keep = torch.empty(res["neumann"].shape[0], dtype=torch.uint8, device=dev)

    def full_step():
        dtn.solve_patches(g, centers, radius, hb, opts, result=res)
        _, kept, nk = dtn.gather_owned(res["colloc_xyz"], owner, centers)
        dtn.eval_potential(g, res["colloc_xyz"], res["normals"], res["areas"], res["neumann"],
                           res["dirichlet"], tgt, prec=prec, out=u_out, index=kept, n_index=nk)

    # walk-kernel launch parameters picked by the library's autotuner (untimed),
    # or fixed on the command line (profiler captures)
    if args.walk_params:
        wc, wb, wr = (int(v) for v in args.walk_params.split(","))
        opts.walk_chunk, opts.wos_blocks_per_sm, opts.wos_refill = wc, wb, wr
        tuning = dict(walk_chunk=wc, wos_blocks_per_sm=wb, wos_refill=wr, source="command line")
    else:
        tuning = dtn.autotune_walks(g, centers, radius, hb, opts)
    for _ in range(args.warmup):
        full_step()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    step_ms, wos_ms, stage = [], [], []
    walk_steps = 0
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()   # write 256 MB between timed steps: L2 starts cold
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        full_step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = g.stage_times()
        stage.append(st)
        wos_ms.append(st[1])
        walk_steps = int(res["gamma_steps"].sum().item())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(step_ms) / len(step_ms)
    ms = reduce_max(ms, dist, dev)
    value = world * b.n / (ms / 1e3)
    wos = sum(wos_ms) / len(wos_ms)
    walk_steps_per_s = world * walk_steps / (wos / 1e3)

    # e2e: host buffers in, host results out, through the same C-ABI calls
    pin_c = torch.from_numpy(b.centers).pin_memory()
    pin_t = torch.from_numpy(targets).pin_memory()
    out_q = torch.empty(res["neumann"].shape, dtype=torch.float64).pin_memory()
    out_u = torch.empty(N_TARGETS, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        centers.copy_(pin_c, non_blocking=True)
        tgt.copy_(pin_t, non_blocking=True)
        full_step()
        out_q.copy_(res["neumann"], non_blocking=True)
        out_u.copy_(u_out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e = sum(e2e_ms) / len(e2e_ms)
    h2d = pin_c.numel() * 8 + pin_t.numel() * 8
    d2h = out_q.numel() * 8 + out_u.numel() * 8

    # the plain FP64 path, one patch per launch, on a sample of 20 patches
    o64 = dtn.solve_opts(prec=dtn.PREC_FP64, epsilon=wl.epsilon, seed=wl.seed)
    nplain = 20
    hb1 = [dtn.HostBatch(b.n_theta[i:i + 1], b.n_phi[i:i + 1], b.n_rings[i:i + 1], b.n_sectors[i:i + 1],
                         b.walks[i:i + 1], patch_id_base=i) for i in range(nplain)]
    r1 = [dtn.alloc_result(h) for h in hb1]
    dtn.solve_patches(g, centers[0:1], radius[0:1], hb1[0], o64, result=r1[0])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(nplain):
        dtn.solve_patches(g, centers[i:i + 1], radius[i:i + 1], hb1[i], o64, result=r1[i])
    e1.record(stream)
    e1.synchronize()
    plain = nplain / (e0.elapsed_time(e1) / 1e3)

    peaks = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT * LANES_PER_SM * sm_mhz * 1e6 / 1e12   # Tops/s
    n_walks = int(np.sum(b.walks * (b.n_theta * b.n_phi)))
    achieved = (walk_steps * OPS_PER_STEP + n_walks * OPS_PER_WALK) / (wos / 1e3) / 1e12
    # setup 3, walks + estimates + walk-cap statuses 3; mixed: group matrices 1, right-side weights 3
    # (far, near, walk term), samples 1, products 1, group factors + solves 2;
    # FP64: matrices and right sides 1, factor + solve 1; gather 4, potential 1
    # the potential adds a split-order reduction when the targets alone fill fewer than
    # 8 CTAs of 256 threads per SM (its panel list is then split across CTAs)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pot_reduce = 1 if sms * 8 // ((N_TARGETS + 255) // 256) > 1 else 0
    kernels_per_step = 3 + 3 + (1 + 3 + 1 + 1 + 2 if prec == dtn.PREC_MIXED else 1 + 1) + 4 + 1 + pot_reduce
    line = {
        "metric": METRIC, "value": value, "unit": "patches/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == dtn.PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "patches": b.n, "nodes_per_patch": int(b.n_theta[0] * b.n_phi[0]),
                   "panels_per_patch": int(b.n_rings[0] * b.n_sectors[0]), "walks_per_node": int(b.walks[0]),
                   "epsilon": wl.epsilon, "targets": N_TARGETS, "precision": args.prec,
                   "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{world}"},
        "walk_steps_per_s": walk_steps_per_s, "walk_steps_per_step": walk_steps,
        "stage_ms": {"setup": statistics.mean(s[0] for s in stage), "walks": wos,
                     "assembly": statistics.mean(s[2] for s in stage), "solve": statistics.mean(s[3] for s in stage),
                     "gather_and_potential": ms - sum(statistics.mean(s[k] for s in stage) for k in range(4))},
        "fp64_path": {"value": plain, "unit": "patches/s", "sample": f"{nplain} patches, one patch per launch",
                      "speedup": value / plain},
        "roofline": {"bound": "alu", "kernel": "wos_kernel_f32<ball>", "achieved": achieved,
                     "peak": alu_peak, "unit": "Tops/s", "frac": achieved / alu_peak,
                     "traffic": DRAM_BYTES_PER_NODE * int(np.sum(b.n_theta * b.n_phi)),
                     "traffic_basis": "ncu dram bytes of the 64-patch capture, scaled by hemisphere nodes",
                     "ncu_issue_slots_busy": NCU_ISSUE_ACTIVE, "ncu_active_lanes_per_inst": NCU_LANES_PER_INST,
                     "ops_per_walk_step": OPS_PER_STEP, "ops_per_walk": OPS_PER_WALK, "walks": n_walks,
                     "peak_basis": f"{SM_COUNT} SMs x {LANES_PER_SM} lanes x {sm_mhz:.0f} MHz (MEASURED_PEAKS sm_max_mhz)"},
        "e2e": {"value": b.n * world / (e2e / 1e3), "unit": "patches/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": kernels_per_step * args.steps,
        "walk_tuning": tuning,
        "clocks": clk,
    }
    if not args.no_serve:
        line["serving"] = run_serving(dtn)
        line["single_point"] = run_single_point(dtn)
        line["potential_fmm"] = run_potential_fmm(dtn)
        line["second_kind"] = run_second_kind(dtn, g, centers, radius, hb,
                                              dict(prec=prec, epsilon=wl.epsilon, seed=wl.seed))
        del res, keep, flush
        torch.cuda.empty_cache()
        # the batching workload (1e4 uneven wire patches, one captured launch) and
        # the precision study's size (2e4 patches x 1024 nodes x 8192 walks)
        line["wires_batch"] = run_batch_leg(dtn, W.wires(), OPS_PER_STEP_WIRES, OPS_PER_WALK_WIRES,
                                            capture=True, exact_ops=False)
        line["unit_ball_scaled"] = run_batch_leg(dtn, W.unit_ball_scaled(), OPS_PER_STEP, OPS_PER_WALK, reps=1,
                                                 n_plain=4)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_sample(wl)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--walk-params", default="", help="chunk,blocks_per_sm,refill (skips the autotuner)")
    ap.add_argument("--patches", type=int, default=2000, help="profiler captures only")
    ap.add_argument("--walks", type=int, default=4096, help="profiler captures only")
    ap.add_argument("--fmm-only", action="store_true", help="only the fast multipole leg (profiler captures)")
    ap.add_argument("--fmm-panels", type=int, default=1_000_000, help="panels = targets of --fmm-only")
    ap.add_argument("--no-direct", action="store_true", help="--fmm-only without the direct sum")
    args = ap.parse_args()
    global ARGS
    ARGS = args
    if args.fmm_only:
        import paper_1210_1491_gb300 as dtn
        print(json.dumps(run_potential_fmm(dtn, args.fmm_panels, args.fmm_panels, direct=not args.no_direct)))
        return
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
