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
# algorithmic FP32-pipe operations of one evaluation of the local operator: 12 absolute values and masks,
# 66 rank compares, 48 feasibility compares, ~181 for the stencil times and metrics of 4.9 feasible pairs
# (37 each) and ~320 for the walk (2-3 change steps of ~100)
OPS_PER_EVAL = 627.0
# DRAM bytes (read + write) per evaluation of each sweep kernel, from one ncu capture of a 2,560-field
# solve (80 weld samples x 32 sources); scaled to a launch by its evaluations.  None for a kernel that
# changed since its capture.
TRAFFIC_BYTES_PER_EVAL = {"fim_warp_kernel": None, "fim_cta_kernel<64>": 5.90, "fim_cta_kernel<128>": 3.31,
                          "fim_cta_kernel<256>": None, "fim_cta_kernel<512>": None}
SMS, FP32_LANES = 152, 128


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
    ap.add_argument("--sweep", type=int, default=0, choices=[0, 1, 2, 3],
                    help="profiling run: sweep schedule (0: the library's choice)")
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 64, 128, 256, 512],
                    help="profiling run: threads of a field's CTA in sweep 3 (0: the library's choice)")
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
    P = api.Plan(wl, precision="fp32", device=local, keep_records=int(full), use_graph=0, band_cells=2.0,
                 sweep=args.sweep, cta_threads=args.cta_threads)
    th = P.theta_tensor()
    times, rect = P.new_times(), P.new_rec_times()
    rec = P.new_records() if full else None
    t0 = time.perf_counter()
    for _ in range(2):
        P.solve(th, times=times, rec_times=rect, records=rec)
        if full:
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
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    P = api.Plan(wl, precision="fp32", device=local, keep_records=1)
    th = P.theta_tensor()
    times, rect, rec = P.new_times(), P.new_rec_times(), P.new_records()
    P.autotune(th, times, rec)
    # observed times: a solve at perturbed orientations plus 10 ns noise (inputs of the adjoint)
    th_obs = P.theta_tensor(np.stack([s.region_theta for s in wl.samples]) + 0.05)
    _, t_obs = P.solve(th_obs)
    t_obs = (t_obs + 1e-8 * torch.randn_like(t_obs)).contiguous()

    stage = {}
    side = [torch.cuda.Stream(), torch.cuda.Stream()]

    def step(theta, timed_stages=False):
        if not timed_stages:
            # after the solve, the FP64 check (FP64 pipe), the rays (FP32) and the adjoint (memory) are
            # independent: they run on three streams and the step ends when all three have
            P.solve(theta, times=times, rec_times=rect, records=rec)
            solved = torch.cuda.Event()
            solved.record(stream)
            for s in side:
                s.wait_event(solved)
            with torch.cuda.stream(side[0]):
                mr, fl = P.check64(theta, times, rec)
            with torch.cuda.stream(side[1]):
                P.trace_rays(theta, times)
            g = P.backward(theta, times, rec, 2.0 * (rect - t_obs))
            for s in side:
                stream.wait_stream(s)
            return mr, fl, g
        # stage timing: the same calls one after the other on one stream
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        P.solve(theta, times=times, rec_times=rect, records=rec)
        ev[1].record(stream)
        mr, fl = P.check64(theta, times, rec)
        ev[2].record(stream)
        P.trace_rays(theta, times)
        ev[3].record(stream)
        g = P.backward(theta, times, rec, 2.0 * (rect - t_obs))
        ev[4].record(stream)
        torch.cuda.synchronize()
        for k, name in enumerate(["solve", "check64", "rays", "adjoint"]):
            stage[name] = stage.get(name, 0.0) + ev[k].elapsed_time(ev[k + 1])
        return mr, fl, g

    for _ in range(max(args.warmup, 3)):
        step(th)
    if P.status() != 0:
        raise SystemExit("device status non-zero during warm-up")

    # ---- timed region (headline): whole step, sweep rounds from CUDA graphs
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = P.stats()["kernel_launches"]
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        mr, fl, g = step(th)
    end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    launches = (P.stats()["kernel_launches"] - launches0) // args.steps
    ms = max_over_ranks(start.elapsed_time(end) / args.steps, world)
    if P.status() != 0:
        raise SystemExit("device status non-zero in the timed region")
    nodes = P.total_nodes * world
    value = nodes / (ms * 1e-3)
    for _ in range(args.steps):
        step(th, timed_stages=True)
    stage = {k: v / args.steps for k, v in stage.items()}

    # ---- roofline of the dominant kernel (the evaluation of the local operator): its launches timed with
    # CUDA events on the solve's stream, over a second run of the same solves
    Pt = api.Plan(wl, precision="fp32", device=local, time_kernels=1, band_cells=P.options.band_cells,
                  sweep=P.options.sweep, cta_threads=P.options.cta_threads, cta_cluster=P.options.cta_cluster)
    tt = Pt.new_times()
    Pt.solve(th, times=tt)
    ev_ms, evals, eval_launches = 0.0, 0, 0
    for _ in range(args.steps):
        Pt.solve(th, times=tt)
        s = Pt.stats()
        ev_ms += s["eval_ms"]
        evals += s["evaluations"]
        eval_launches += s["eval_launches"]
    peaks, peak_kind = _peaks()
    clock = ck["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    achieved = OPS_PER_EVAL * evals / (ev_ms * 1e-3) / 1e12
    peak = SMS * FP32_LANES * clock * 1e6 / 1e12
    evals_per_node = evals / (args.steps * P.total_nodes)
    kname = {1: "fim_eval_kernel", 2: "fim_warp_kernel", 3: "fim_cta_kernel"}[P.options.sweep]
    if P.options.sweep == 3:  # the CTA shape decides how many fields share the L2, hence the traffic
        kname += f"<{P.options.cta_threads}>" + (f"x{P.options.cta_cluster}" if P.options.cta_cluster > 1 else "")
    del Pt, tt

    # ---- end to end through the public API: orientations from pinned host memory, receiver times back
    th_host = torch.from_numpy(np.stack([s.region_theta for s in wl.samples])).pin_memory()
    rt_host = torch.empty(rect.shape, dtype=rect.dtype).pin_memory()
    g_host = torch.empty(th.shape, dtype=torch.float64).pin_memory()
    th_dev = torch.empty_like(th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        th_dev.copy_(th_host, non_blocking=True)
        _, _, g = step(th_dev)
        rt_host.copy_(rect, non_blocking=True)
        g_host.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fields": P.nfields, "nodes_per_step": P.total_nodes,
                   "rays_per_step": P.nfields * P.nrec, "band_cells": P.options.band_cells,
                   "sweep": {1: "lockstep rounds over all fields", 2: "one warp per field",
                             3: "one CTA per field"}[P.options.sweep],
                   "l2": "inputs larger than L2 (3.6 GB of fields), no flush"},
        "stage_ms": stage, "evaluations_per_node": evals_per_node,
        "fp64_check": {"max_rel_residual": float(mr.max().item()), "record_flips": int(fl.sum().item())},
        "e2e": {"value": nodes / (e2e_ms * 1e-3), "unit": "nodes/s",
                "h2d_bytes_per_step": int(th_host.numel() * th_host.element_size()),
                "d2h_bytes_per_step": int(rt_host.numel() * rt_host.element_size()
                                          + g_host.numel() * g_host.element_size())},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (TRAFFIC_BYTES_PER_EVAL[kname] * evals / args.steps / max(eval_launches // args.steps, 1)
                                 if TRAFFIC_BYTES_PER_EVAL.get(kname) else None),
                     "peak_source": f"152 SMs x 128 FP32 lanes x 1 op x {clock:.0f} MHz (sampled clock); "
                                    f"{OPS_PER_EVAL:.0f} FP32 ops per evaluation",
                     "avg_launch_ms": ev_ms / max(eval_launches, 1), "launches": eval_launches // args.steps},
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
        "gpu_launches": int(launches),
    }
    if not args.quick:
        # plain single-medium form: 256 x 256 weld, 32 sources
        wl1 = W.weld_single()
        plain = {}
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
            del P1, t1
        line["plain_nodes_per_s"] = plain
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
