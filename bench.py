#!/usr/bin/env python3
"""Benchmark of the HASF library on its headline workload.

Workload (one step): a batch of 256 synthetic 512 x 512 binary images (12
discs/ellipses, 6 holes, 2-px jitter, 2-10 % salt-and-pepper noise), rmax = 5,
50 kept points C per image, smoothed by one hasf_smooth_batch launch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hasf|reference]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain single-threaded C restatement of the method) on the host cores, as the
reference arm.  Under torchrun every rank smooths its own batch (replicas, no
collective on the data path) and the value is all ranks' images over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HASF images/s at 512x512, rmax=5"
BATCH = 256
RMAX = 5
WORKLOAD = ("batch of 256 synthetic 512x512 binary images (discs/ellipses, holes, jitter, "
            "2-10% salt-and-pepper), rmax=5, 50 kept points C per image, one batched launch")
# Lane operations of one word test in the sweep kernel (32 pixels): 10 loads,
# 6 funnel shifts, 21 logic operations, 4 update operations.
OPS_PER_WORD_TEST = 41
# Lane operations of one ring-vector evaluation in a level update.
OPS_PER_RING_EVAL = 7


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_job(args):
    import numpy as np
    import oracle
    X, C, rmax = args
    t = time.perf_counter()
    oracle.hasf(X, rmax, C=C)
    return time.perf_counter() - t


def cpu_oracle_rate(jobs, cores):
    """Images/s of the oracle on `cores` host processes over `jobs`."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, [(jobs[0].X, jobs[0].C, jobs[0].rmax)] * cores)  # load in workers
        t0 = time.perf_counter()
        per = pool.map(_oracle_job, [(j.X, j.C, j.rmax) for j in jobs], chunksize=1)
        wall = time.perf_counter() - t0
    return len(jobs) / wall, wall, sum(per)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1603_09337_gb300 import synth
    cores = os.cpu_count() or 1
    per_step = cores
    jobs = synth.batch_512(per_step * (args.steps + args.warmup))
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        k = 0
        for _ in range(args.warmup):
            pool.map(_oracle_job, [(j.X, j.C, j.rmax) for j in jobs[k:k + per_step]], chunksize=1)
            k += per_step
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_job, [(j.X, j.C, j.rmax) for j in jobs[k:k + per_step]], chunksize=1)
            k += per_step
        wall = time.perf_counter() - t0
    value = per_step * args.steps / wall
    line = {
        "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORKLOAD + f"; reference arm: the CPU oracle, {per_step} images "
                   "per step (one per host core)", "images_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "images/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step * args.steps} images of the workload, "
                                   f"{per_step} per step, one oracle process per core"},
        "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_hasf(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1603_09337_gb300 import Context, Image, build, synth

    build.build()
    jobs = synth.batch_512(BATCH, first=rank * BATCH)
    ctx = Context(local)
    X = torch.from_numpy(np.stack([j.X for j in jobs])).to(dev)
    C = torch.from_numpy(np.stack([j.C for j in jobs])).to(dev)
    out = torch.empty_like(X)
    imgs = [Image(X[i], RMAX, C=C[i], out=out[i]) for i in range(BATCH)]
    arr = ctx.batch_descriptors(imgs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.smooth_batch_raw(arr, BATCH)
    ctx.status()

    # Work counters of one step (for the ALU roofline): a separate, untimed run.
    stats = ctx.stats_step(arr, BATCH) if hasattr(ctx, "stats_step") else None

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(torch.cuda.get_device_properties(dev).pci_bus_id if False else local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()                       # evict L2 (129 MB) between steps
            starts[i].record(stream)
            ctx.smooth_batch_raw(arr, BATCH)
            ends[i].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
    ctx.status()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = sum(step_ms)
    if ws > 1:
        tt = torch.tensor([t_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_ms = float(tt.item())
    total_images = BATCH * args.steps * ws
    value = total_images / (t_ms / 1e3)
    ms_per_step = t_ms / args.steps

    # End to end through the host-buffer entry point: H2D + compute + D2H.
    e2e = None
    if not args.no_e2e:
        hX = [np.ascontiguousarray(j.X) for j in jobs]
        hC = [np.ascontiguousarray(j.C) for j in jobs]
        hO = [np.empty_like(j.X) for j in jobs]
        host_jobs = [(hX[i], RMAX, hC[i], None, 8, hO[i]) for i in range(BATCH)]
        ctx.smooth_host(host_jobs)                     # warm-up (staging buffers)
        k = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            ctx.smooth_host(host_jobs)
        barrier()
        te = (time.perf_counter() - t0) / k
        e2e = {"value": BATCH * ws / te, "unit": "images/s",
               "h2d_bytes_per_step": int(sum(a.nbytes for a in hX) + sum(a.nbytes for a in hC)),
               "d2h_bytes_per_step": int(sum(a.nbytes for a in hO))}

    if rank != 0:
        ctx.close()
        return 0

    peaks, peak_src = _peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = 152 * 128 * sm_max * 1e6 / 1e12            # T lane-ops/s
    roof = None
    if stats is not None:
        ops = stats["word_tests"] * OPS_PER_WORD_TEST + stats["ring_evals"] * OPS_PER_RING_EVAL
        achieved = ops / (ms_per_step / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak, "traffic": None,
                "peak_source": "152 SMs x 128 int32 lanes x max SM clock (recipe units/clock)",
                "ops_per_step": ops, "counters": stats}
    alg_bytes = BATCH * 512 * 512 * 3
    hbm = {"achieved_gbs": alg_bytes / (ms_per_step / 1e3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
           "frac": alg_bytes / (ms_per_step / 1e3) / 1e9 / peaks["hbm_gbs"],
           "peak_source": peak_src}

    cpu = None
    if not args.no_cpu and ws == 1:
        cores = os.cpu_count() or 1
        sample = synth.batch_512(2 * cores, first=10_000)
        rate, cwall, cwork = cpu_oracle_rate(sample, cores)
        cpu = {"value": rate, "unit": "images/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(sample)} images of the workload (other seeds), one oracle "
                         f"process per core, {cwork:.1f} s of CPU work in {cwall:.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit planes (integer only)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "images_per_step": BATCH, "width": 512, "height": 512,
                   "rmax": RMAX, "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "mpixel_per_s": value * 512 * 512 / 1e6, "wall_s": wall},
        "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hasf", choices=["hasf", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_hasf(args)


if __name__ == "__main__":
    sys.exit(main())
