#!/usr/bin/env python3
"""Benchmark of the ALI-FMM travel-time hot path on GB300.

Workload (N = 1): the batched weld workload -- 512 media samples (region
orientations drawn per sample) x 32 sources, grid sizes uniform in 128..320
(step 32), 10 x 10 weld regions, FP32.  One step is one pass of the whole hot
path over the batch: per-region constants, near-source initialisation, the
sweep to the fixed point (the schedule the autotuner picks), receiver times,
the FP64 convergence check, rays for 32 receivers per source and the adjoint
gradient of a receiver-time misfit with respect to the region orientations (the
last three, independent of one another, on three streams after the solve).

Metric: travel-time nodes/s = sum over fields of nx * ny / step time.  Also
reported: the plain single-medium form (256 x 256, 32 sources, FP32 and FP64)
and the gradient time of the 256-sample adjoint workload (200 x 200).
Inputs are synthetic and seeded; the packed fields (3.6 GB FP32) are larger
than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (launched by torchrun) every rank solves its own batch of the same shape
(its own seeded orientation draws; weak scaling, no collective on the data path), the
step time is the slowest rank's, and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "travel-time nodes/s (sources x models x nodes), batched FP32"
WORKLOAD = ("weld batch: 512 samples x 32 sources, n in 128..320 step 32, 10x10 regions, FP32; "
            "step = solve + FP64 check + 32 rays/source + adjoint gradient")
# Algorithmic work of one evaluation of the local operator per node (Secs. 4.2-4.3 with the recompute rule of
# Sec. 2): the FP64 oracle's operation count on converged fields of these workloads, stored by
# tests/golden/make_ops_per_node.py.  The sweep's roofline divides (this count x the launch's nodes) by the
# launch's CUDA-event time; the peak is SMs x 128 FP32 lanes x 2 (an FMA is two operations) x SM clock.
OPS_FILE = os.path.join(ROOT, "tests", "golden", "ops_per_node.txt")
# DRAM bytes per node of one solve's sweep launch (dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of an FP32 solve alone, divided by the launch's nodes; profiles/ holds the captures); None where
# the kernel has changed since its counters were taken
TRAFFIC_BYTES_PER_NODE = {"fim_warp_kernel": (2.619382e9 + 3.100162e9) / 147783680,
                          "fim_cta_kernel<64>": (0.749040896e9 + 1.390257152e9) / 147783680,
                          "fim_cta_kernel<128>": None, "fim_cta_kernel<256>": None,
                          # the plain 256 x 256 x 32 medium, the only workload the bench runs with 512 threads
                          "fim_cta_kernel<512>": (8.823296e6 + 0.104704e6) / 2097152}
FP32_LANES = 128
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (CUDA cores), nominal


def ops_per_node(workload: str) -> float:
    acc = [0, 0]
    for line in open(OPS_FILE):
        f = line.split()
        if line.startswith("#") or len(f) != 5 or f[0] != workload:
            continue
        acc[0] += int(f[3])
        acc[1] += int(f[4])
    return acc[0] / acc[1]


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=512)
    ap.add_argument("--quick", action="store_true", help="skip the plain and gradient side measurements")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: direct launches on the default stream, no autotune, one warm-up step and "
                         "one step, a short summary line (for ncu)")
    ap.add_argument("--profile-stages", default="all", choices=["all", "solve"],
                    help="profiling run: the whole step, or the travel-time solve alone")
    ap.add_argument("--sweep", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="profiling run: sweep schedule (0: the library's choice; 4: active tiles)")
    ap.add_argument("--band", type=float, default=1.5,
                    help="profiling run: front band of the sweep in cell-crossing times")
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 64, 128, 256, 512],
                    help="profiling run: threads of a field's CTA in sweep 3 (0: the library's choice)")
    ap.add_argument("--check", default="stream", choices=["fused", "stream"],
                    help="FP64 check of the step: inside the solve (alf_solve_check64) or on a stream of its own "
                         "after the solve (alf_check64 beside the rays and the adjoint)")
    ap.add_argument("--profile-workload", default="batch", choices=["batch", "plain"],
                    help="profiling run: the weld batch (--samples x 32 sources) or the plain single medium "
                         "(256 x 256 weld, 32 sources)")
    return ap.parse_args()


def _dist():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        ok = [r for r in self.rows if len(r) >= 9]
        sm = [float(r[1]) for r in ok if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in ok if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in ok for k, n in enumerate(names) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons}


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's step time (the whole job finishes when its last rank does)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(W, nsamples: int, rank: int):
    """Rank `rank`'s own batch: same shape and size as rank 0's, its own orientation draws."""
    return W.weld_batch(nsamples=nsamples, seed=W.rank_seed(2, rank))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(wl, seconds=12.0):
    """The FP64 oracle (heap FMM, as it stands) on a bounded sample of the workload's fields, timed on the host
    cores with one thread per field (ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    O.build()
    mats = [O.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    fields = [(b, s) for b in range(len(wl.samples)) for s in range(len(wl.samples[b].src))]
    order = np.random.default_rng(0).permutation(len(fields))
    cores = os.cpu_count() or 1

    def one(k):
        b, s = fields[order[k % len(fields)]]
        smp = wl.samples[b]
        M = O.OMedium.from_regions(smp.nx, smp.ny, smp.h, smp.region_map, smp.region_theta, wl.region_material, mats)
        fr, t0 = O.init_radius(M, *smp.src[s], 2)
        O.fmm(M, fr, t0)
        return smp.nx * smp.ny

    nodes, nf = 0, 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        while time.perf_counter() - t0 < seconds:
            nodes += sum(ex.map(one, range(nf, nf + cores)))
            nf += cores
    dt = time.perf_counter() - t0
    return {"value": nodes / dt, "unit": "nodes/s", "cores": cores, "kind": "oracle",
            "sample": f"{nf} of {len(fields)} fields, FP64 heap FMM (solve only), {dt:.1f} s on {cores} threads"}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    from paper_2302_10988_gb300 import workloads as W
    wl = W.weld_batch(nsamples=args.samples)
    for _ in range(args.warmup):
        cpu_baseline(wl, seconds=2.0)
    vals = [cpu_baseline(wl, seconds=6.0) for _ in range(args.steps)]
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "nodes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl.nodes() / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD}, "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_run(args, wl, api, local):
    """One warm-up step and one step of the hot path with direct launches (no CUDA graph) on the default stream."""
    import torch
    full = args.profile_stages == "all"
    P = api.Plan(wl, precision="fp32", device=local, keep_records=int(full), use_graph=0, band_cells=args.band,
                 sweep=args.sweep, cta_threads=args.cta_threads)
    th = P.theta_tensor()
    times, rect = P.new_times(), P.new_rec_times()
    rec = P.new_records() if full else None
    t0 = time.perf_counter()
    for _ in range(2):
        if full and args.check == "fused":
            P.solve_check64(th, times=times, rec_times=rect, records=rec)
        else:
            P.solve(th, times=times, rec_times=rect, records=rec)
        if full:
            if args.check != "fused":
                P.check64(th, times, rec)
            P.trace_rays(th, times)
            P.backward(th, times, rec, 2.0 * rect)
    torch.cuda.synchronize()
    st = P.stats()
    print(json.dumps({"profile_run": True, "fields": P.nfields, "nodes": P.total_nodes, "status": P.status(),
                      "evaluations_last_solve": st["evaluations"], "rounds_last_solve": st["rounds"],
                      "sweep": P.options.sweep, "cta_threads": P.options.cta_threads,
                      "cta_cluster": P.options.cta_cluster, "stages": args.profile_stages,
                      "seconds": time.perf_counter() - t0}), flush=True)


def _kernel_name(opts) -> str:
    kname = {1: "fim_eval_kernel", 2: "fim_warp_kernel", 3: "fim_cta_kernel", 4: "fim_tile_kernel"}[opts.sweep]
    if opts.sweep == 3:  # the CTA shape decides how many fields share the L2, hence the traffic
        kname += f"<{opts.cta_threads}>" + (f"x{opts.cta_cluster}" if opts.cta_cluster > 1 else "")
    return kname


def sweep_roofline(api, wl, theta, opts, steps, local, clock, nsm, ops_node, precision="fp32"):
    """Roofline of the sweep kernel of a solve with the tuned options: its launches timed with CUDA events on the
    solve's stream over `steps` solves (the library records them, option time_kernels)."""
    Pt = api.Plan(wl, precision=precision, device=local, time_kernels=1, band_cells=opts.band_cells,
                  sweep=opts.sweep, cta_threads=opts.cta_threads, cta_cluster=opts.cta_cluster)
    tt = Pt.new_times()
    Pt.solve(theta, times=tt)
    ev_ms, evals, launches = 0.0, 0, 0
    for _ in range(steps):
        Pt.solve(theta, times=tt)
        st = Pt.stats()
        ev_ms += st["eval_ms"]
        evals += st["evaluations"]
        launches += st["eval_launches"]
    if Pt.status() != 0:
        raise SystemExit("device status non-zero in the roofline solves")
    nodes = Pt.total_nodes
    if precision == "fp32":
        peak, peak_src = nsm * FP32_LANES * 2 * clock * 1e6 / 1e12, (
            f"{nsm} SMs x {FP32_LANES} FP32 lanes x 2 (FMA) x {clock:.0f} MHz (sampled SM clock)")
    else:
        peak, peak_src = FP64_NOMINAL_TFLOPS, "GB300 FP64 CUDA-core rate, nominal"
    achieved = ops_node * nodes * steps / (ev_ms * 1e-3) / 1e12
    kname = _kernel_name(opts)
    per_launch_nodes = nodes * steps / max(launches, 1)
    tb = TRAFFIC_BYTES_PER_NODE.get(kname) if precision == "fp32" else None  # the captures are FP32 solves
    out = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": tb * per_launch_nodes if tb else None,
           "peak_source": peak_src,
           "work": f"{ops_node:.1f} operations per node (FP64 oracle's count of one evaluation of F, "
                   f"tests/golden/ops_per_node.txt) x {per_launch_nodes:.4g} nodes per launch",
           "avg_launch_ms": ev_ms / max(launches, 1), "launches": launches // steps,
           "evaluations_per_node": evals / (steps * nodes)}
    del Pt, tt
    return out


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    # one build per node: local rank 0 compiles, the others load what it built
    if local == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    if local != 0:
        __graft_entry__.build()
    from paper_2302_10988_gb300 import api, workloads as W

    wl = rank_workload(W, args.samples, rank)
    if args.profile:
        return profile_run(args, W.weld_single() if args.profile_workload == "plain" else wl, api, local)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # rays: 256 points per ray is room for the longest (about 120 on a 320 x 320 grid); a ray that ran out of
    # room would set the plan's status, which is checked
    P = api.Plan(wl, precision="fp32", device=local, keep_records=1, max_ray_points=256)
    th = P.theta_tensor()
    times, rect, rec = P.new_times(), P.new_rec_times(), P.new_records()
    P.autotune(th, times, rec)
    # observed times: a solve at perturbed orientations plus 10 ns noise (inputs of the adjoint)
    th_obs = P.theta_tensor(np.stack([s.region_theta for s in wl.samples]) + 0.05)
    _, t_obs = P.solve(th_obs)
    t_obs = (t_obs + 1e-8 * torch.randn_like(t_obs)).contiguous()

    stage = {}
    side = [torch.cuda.Stream(), torch.cuda.Stream()]
    # the rays' points packed back to back for the host (alf_pack_rays), into buffers of the worst-case size
    nrays = P.nfields * P.nrec
    packed = torch.empty((nrays * P.options.max_ray_points, 2), dtype=torch.float32, device=th.device)
    offsets = torch.empty(nrays + 1, dtype=torch.int64, device=th.device)

    def step(theta, host=None):
        # the FP64 check (FP64 pipe) runs inside the solve, each field checked by the CTA that solved it
        # (--check fused), or after the solve on a stream of its own; the rays (FP32) and the adjoint (memory)
        # are independent of each other and of the check: they run on two more streams, and the step ends
        # when all have.  With `host` (the end-to-end leg), the rays' offsets, times and status leave for
        # pinned host memory on the rays' stream as soon as they are packed, beside the check and the adjoint
        cur = torch.cuda.current_stream()
        if args.check == "fused":
            _, _, mr, fl = P.solve_check64(theta, times=times, rec_times=rect, records=rec)
        else:
            P.solve(theta, times=times, rec_times=rect, records=rec)
        solved = torch.cuda.Event()
        solved.record(cur)
        for s in side:
            s.wait_event(solved)
        if args.check != "fused":
            with torch.cuda.stream(side[0]):
                mr, fl = P.check64(theta, times, rec)
        with torch.cuda.stream(side[1]):
            rays = P.trace_rays(theta, times)
            P.pack_rays(rays[0], rays[1], packed=packed, offsets=offsets)
            if host is not None:
                for h, o in zip(host["rays"], [offsets, rays[2], rays[3]]):
                    h.copy_(o, non_blocking=True)
                host["rays_out"].record(side[1])
        g = P.backward(theta, times, rec, 2.0 * (rect - t_obs))
        for s in side:
            cur.wait_stream(s)
        return {"max_rel": mr, "flips": fl, "grad": g, "rays": rays}

    def staged(theta):
        # stage timing: the same calls one after the other on one stream
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(stream)
        P.solve(theta, times=times, rec_times=rect, records=rec)
        ev[1].record(stream)
        P.check64(theta, times, rec)
        ev[2].record(stream)
        P.trace_rays(theta, times)
        ev[3].record(stream)
        P.backward(theta, times, rec, 2.0 * (rect - t_obs))
        ev[4].record(stream)
        P.solve_check64(theta, times=times, rec_times=rect, records=rec)
        ev[5].record(stream)
        torch.cuda.synchronize()
        for k, name in enumerate(["solve", "check64", "rays", "adjoint", "solve_check64"]):
            stage[name] = stage.get(name, 0.0) + ev[k].elapsed_time(ev[k + 1])

    for _ in range(max(args.warmup, 3)):
        step(th)
    torch.cuda.synchronize()
    if P.status() != 0:
        raise SystemExit("device status non-zero during warm-up")

    # the whole step captured once in a CUDA graph (the solve is one persistent launch for the field-resident
    # schedules, and nothing in the step waits on the host); replayed in the timed region
    graph, out = None, None
    launches0 = P.stats()["kernel_launches"]
    if P.options.sweep != 1:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
            out = step(th)
        torch.cuda.synchronize()
    launches = P.stats()["kernel_launches"] - launches0  # library kernels of one step

    def run():
        if graph is not None:
            graph.replay()
            return out
        return step(th)

    run()
    torch.cuda.synchronize()
    # ---- timed region (headline)
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = P.stats()["kernel_launches"]
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        res = run()
    end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if graph is None:
        launches = (P.stats()["kernel_launches"] - l0) // args.steps
    ms = max_over_ranks(start.elapsed_time(end) / args.steps, world)
    if P.status() != 0:
        raise SystemExit("device status non-zero in the timed region")
    mr, fl = res["max_rel"], res["flips"]
    nodes = P.total_nodes * world
    value = nodes / (ms * 1e-3)
    for _ in range(args.steps):
        staged(th)
    stage = {k: v / args.steps for k, v in stage.items()}

    # ---- roofline of the dominant kernel (the sweep of the local operator)
    peaks, peak_kind = _peaks()
    clock = ck["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    roof = sweep_roofline(api, wl, th, P.options, args.steps, local, clock, nsm, ops_per_node("weld_batch"))

    # ---- end to end through the public API: orientations from pinned host memory in, receiver times, the
    # gradient and every ray (points, point counts, times, status) back to pinned host memory
    # (the ray paths leave packed: the offsets, then the total's points; counts are the offsets' differences).
    # The rays' outputs leave while the check and the adjoint still run: the host waits for the offsets
    # alone, then queues the packed points on the rays' stream.
    pts, npts, rtime, rst = res["rays"]
    th_host = torch.from_numpy(np.stack([s.region_theta for s in wl.samples])).pin_memory()
    pinned = lambda o: torch.empty(o.shape, dtype=o.dtype).pin_memory()
    host = {"rays": [pinned(offsets), pinned(rtime), pinned(rst)], "rays_out": torch.cuda.Event()}
    rect_host, grad_host = pinned(rect), pinned(res["grad"])
    packed_host = torch.empty(packed.shape, dtype=packed.dtype).pin_memory()
    th_dev = torch.empty_like(th)
    d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        th_dev.copy_(th_host, non_blocking=True)
        r = step(th_dev, host)
        host["rays_out"].synchronize()
        total = int(host["rays"][0][-1])
        with torch.cuda.stream(side[1]):
            packed_host[:total].copy_(packed[:total], non_blocking=True)
        rect_host.copy_(rect, non_blocking=True)
        grad_host.copy_(r["grad"], non_blocking=True)
        torch.cuda.synchronize()
        d2h = (sum(h.numel() * h.element_size() for h in host["rays"] + [rect_host, grad_host]) +
               total * 2 * packed.element_size())
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    if P.status() != 0:
        raise SystemExit("device status non-zero in the end-to-end steps")

    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fields": P.nfields, "nodes_per_step": P.total_nodes,
                   "rays_per_step": P.nfields * P.nrec, "band_cells": P.options.band_cells,
                   "sweep": {1: "lockstep rounds over all fields", 2: "one warp per field",
                             3: "one CTA per field", 4: "active tiles"}[P.options.sweep],
                   "cuda_graph": graph is not None,
                   "fp64_check": {"fused": "inside the sweep kernel, per field after its sweep",
                                  "stream": "own kernel on a side stream after the solve"}[args.check],
                   "l2": "inputs larger than L2 (3.6 GB of fields), no flush"},
        "stage_ms": stage, "evaluations_per_node": roof["evaluations_per_node"],
        "fp64_check": {"max_rel_residual": float(mr.max().item()), "record_flips": int(fl.sum().item())},
        "e2e": {"value": nodes / (e2e_ms * 1e-3), "unit": "nodes/s",
                "h2d_bytes_per_step": int(th_host.numel() * th_host.element_size()),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": roof,
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
        "gpu_launches": int(launches),
    }
    if not args.quick:
        # plain single-medium form: 256 x 256 weld, 32 sources
        wl1 = W.weld_single()
        plain, plain_roof = {}, {}
        for prec in ("fp32", "fp64"):
            P1 = api.Plan(wl1, precision=prec, device=local)
            th1 = P1.theta_tensor()
            t1 = P1.new_times()
            P1.autotune(th1, t1)
            P1.solve(th1, times=t1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                P1.solve(th1, times=t1)
            e1.record(stream)
            torch.cuda.synchronize()
            plain[prec] = P1.total_nodes / (e0.elapsed_time(e1) / 3 * 1e-3)
            plain[prec + "_schedule"] = {"sweep": P1.options.sweep, "band_cells": P1.options.band_cells,
                                         "cta_threads": P1.options.cta_threads}
            plain_roof[prec] = sweep_roofline(api, wl1, th1, P1.options, 3, local, clock, nsm,
                                              ops_per_node("weld_single"), prec)
            del P1, t1
        line["plain_nodes_per_s"] = plain
        line["plain_roofline"] = plain_roof
        # large single medium: 2048 x 2048, 64 sources, 4096 receivers per source
        wlL = W.weld_large()
        PL = api.Plan(wlL, precision="fp32", device=local, max_ray_points=1024)
        thL = PL.theta_tensor()
        tL = PL.new_times()
        PL.solve(thL, times=tL)
        PL.trace_rays(thL, tL)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        PL.solve(thL, times=tL)
        e1.record(stream)
        PL.trace_rays(thL, tL)
        e2.record(stream)
        torch.cuda.synchronize()
        line["large_medium"] = {"config": "2048 x 2048, 0.1 mm, 100 x 100 regions, 64 sources x 4096 receivers, FP32",
                                "nodes_per_s": PL.total_nodes / (e0.elapsed_time(e1) * 1e-3),
                                "rays_per_s": PL.nfields * PL.nrec / (e1.elapsed_time(e2) * 1e-3),
                                "sweep": PL.options.sweep, "cta_threads": PL.options.cta_threads,
                                "cta_cluster": PL.options.cta_cluster,
                                "status": PL.status()}
        del PL, tL
        # gradient: 256 samples x 32 sources on 200 x 200, forward (records) + adjoint
        wl3, truth = W.weld_adjoint()
        P3 = api.Plan(wl3, precision="fp32", device=local, keep_records=1)
        th3 = P3.theta_tensor()
        Pt3 = api.Plan(truth, precision="fp32", device=local)
        _, tob = Pt3.solve(Pt3.theta_tensor())
        tob = (tob + torch.as_tensor(W.observation_noise(tuple(tob.shape)), device=tob.device).float())
        t3, r3, c3 = P3.new_times(), P3.new_rec_times(), P3.new_records()
        P3.autotune(th3, t3, c3)

        def grad_step():
            P3.solve(th3, times=t3, rec_times=r3, records=c3)
            return P3.backward(th3, t3, c3, 2.0 * (r3 - tob))
        grad_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            grad_step()
        e1.record(stream)
        torch.cuda.synchronize()
        line["grad_ms"] = e0.elapsed_time(e1) / 3
        line["grad_schedule"] = {"sweep": P3.options.sweep, "band_cells": P3.options.band_cells,
                                 "cta_threads": P3.options.cta_threads}
        line["grad_config"] = "256 samples x 32 sources x 32 receivers, 200 x 200, FP32 forward + adjoint"
        del P3, Pt3
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
