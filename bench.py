#!/usr/bin/env python3
"""Benchmark of the ALI-FMM travel-time hot path on GB300.

Workload (N = 1): the batched weld workload -- 512 media samples (region
orientations drawn per sample) x 32 sources, grid sizes uniform in
128..320 (step 32), 10 x 10 weld regions, FP32 sweeps.  One step is one pass
of the hot path over the batch: per-region constants, near-source
initialisation, tile sweeps to the fixed point, FP64 convergence check,
receiver times and rays (32 receivers per source).

Metric: travel-time nodes/s = sum over fields of nx*ny / step time.
Inputs are synthetic and seeded; the packed fields (3.6 GB FP32) are larger
than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (launched by torchrun) every rank solves its own share of the
samples (no collective on the data path) and rank 0 prints the line.
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
WORKLOAD = "weld batch: 512 samples x 32 sources, n in 128..320 step 32, 10x10 regions, FP32"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=512)
    ap.add_argument("--no-rays", action="store_true")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for k, n in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 issue roofline of the ALU-bound sweep: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock
SMS, FP32_LANES = 152, 128


def cpu_baseline(wl, seconds=12.0):
    """The FP64 oracle (heap FMM, as it stands) on a bounded sample of the workload's fields, timed on the
    host cores with one thread per field (ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    O.build()
    mats = [O.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    fields = [(b, s) for b in range(len(wl.samples)) for s in range(len(wl.samples[b].src))]
    rng = np.random.default_rng(0)
    order = rng.permutation(len(fields))
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
            "sample": f"{nf} of {len(fields)} fields (FP64 heap FMM, radius-2 init), {dt:.1f} s"}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    from paper_2302_10988_gb300 import workloads as W
    wl = W.weld_batch(nsamples=args.samples)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(wl, seconds=2.0)
    for _ in range(args.steps):
        vals.append(cpu_baseline(wl, seconds=6.0))
    v = float(np.mean([x["value"] for x in vals]))
    total = wl.nodes()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "nodes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "fields larger than L2"},
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    __graft_entry__.build()
    from paper_2302_10988_gb300 import api, workloads as W

    wl_all = W.weld_batch(nsamples=args.samples)
    # weak scaling: every rank takes its own samples (the whole batch per rank)
    wl = wl_all
    P = api.Plan(wl, precision="fp32", device=local)
    th = P.theta_tensor()
    times = P.new_times()
    rect = P.new_rec_times()
    rec = P.new_records()
    max_rel = flips = None
    stream = torch.cuda.current_stream()

    def step():
        nonlocal max_rel, flips
        P.solve(th, times=times, rec_times=rect, records=rec)
        max_rel, flips = P.check64(th, times, rec)
        if not args.no_rays:
            P.trace_rays(th, times)

    for _ in range(max(args.warmup, 3)):
        step()
    code = P.status()
    if code != 0:
        raise SystemExit(f"device status {code} during warm-up")
    stats = P.stats()

    # sweep-kernel share of the step, timed on the launching stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(2):
        P.solve(th, times=times, rec_times=rect, records=rec)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1) / 2

    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step()
    end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = start.elapsed_time(end) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    code = P.status()
    if code != 0:
        raise SystemExit(f"device status {code} in the timed region")
    nodes = P.total_nodes * world
    value = nodes / (ms * 1e-3)

    # end to end: orientations from pinned host memory, receiver times back to the host
    th_host = torch.from_numpy(np.stack([s.region_theta for s in wl.samples])).pin_memory()
    rt_host = torch.empty(rect.shape, dtype=rect.dtype).pin_memory()
    th_dev = torch.empty_like(th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        th_dev.copy_(th_host, non_blocking=True)
        P.solve(th_dev, times=times, rec_times=rect, records=rec)
        P.check64(th_dev, times, rec)
        if not args.no_rays:
            P.trace_rays(th_dev, times)
        rt_host.copy_(rect, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    torch.cuda.synchronize()
    peaks, peak_kind = _peaks()
    clock = ck["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    # ALU roofline of the sweep: algorithmic FP32 flops per node x nodes / solve time
    flops_per_node = float(os.environ.get("ALF_FLOPS_PER_NODE", "0")) or None
    achieved = (flops_per_node * P.total_nodes / (solve_ms * 1e-3) / 1e12) if flops_per_node else None
    peak = SMS * FP32_LANES * 2 * clock * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fields": P.nfields, "nodes_per_step": P.total_nodes,
                   "rays_per_step": 0 if args.no_rays else P.nfields * P.nrec, "cta_threads": P.options.cta_threads,
                   "l2": "inputs larger than L2 (3.6 GB of fields), no flush"},
        "solve_ms": solve_ms, "evaluations_per_node": stats["evaluations"] / max(stats["nodes"], 1),
        "fp64_check": {"max_rel_residual": float(max_rel.max().item()), "record_flips": int(flips.sum().item())},
        "e2e": {"value": nodes / (e2e_ms * 1e-3), "unit": "nodes/s",
                "h2d_bytes_per_step": int(th_host.numel() * 8),
                "d2h_bytes_per_step": int(rt_host.numel() * rt_host.element_size())},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {clock:.0f} MHz (sampled clock)"},
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
        "gpu_launches": None,
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
