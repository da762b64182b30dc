#!/usr/bin/env python3
"""Benchmark of the HASF library on its headline workload.

Workload of one step: a batch of 256 synthetic 512 x 512 binary images (12
discs/ellipses of semi-axes 20-90, 6 holes, 2-px jitter, 2-10 % salt-and-
pepper noise), rmax = 5, 50 kept points C per image, smoothed by one
hasf_smooth_batch launch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hasf|reference]
                  [--workload batch512|ragged|large] [--serve-seconds S]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain single-threaded C restatement of the method) on the host cores, as the
reference arm.  Under torchrun every rank smooths its own batch (replicas, no
collective on the data path) and the value is all ranks' images over the
slowest rank's time.  The line also carries a serving measurement: Poisson
arrivals at 2,000 requests/s of images of mixed sizes through hasf_submit /
hasf_poll, p50/p99 latency against plain sequential hasf_smooth calls.
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
# Algorithmic lane operations (32 pixels per lane) of the bit-sliced method
# (RECIPE_MIX below): one word test = 6 funnel shifts aligning the 8
# neighbours, 8 logic operations for the four crossing terms, 4 to count
# exactly one, 2 to gate by the candidates and update the set; one ring read
# of a level update = 1 funnel shift + 1 OR.
# 3D: one voxel test = 27 lane-ops to assemble the 27-bit neighbourhood, then
# either the table read (index, shift, mask: 5) or at least two dilation steps
# of each of the two flood fills (about 18 each), counted as 100; one ring read
# of a word = funnel shift + AND/OR + address, 4.
OPS_PER_VOXEL_TEST = {"table": 32, "flood fill": 100}
OPS_PER_RING3_EVAL = 4
INT32_LANES_PER_SM = 128
# Lane-operations of the recipe by instruction class: per word test 6 funnel
# shifts and 14 logic operations, per ring read 1 funnel shift and 1 OR.
RECIPE_MIX = {"word_tests": {"shf": 6, "lop3": 14}, "ring_evals": {"shf": 1, "lop3": 1}}


TRAFFIC_SOURCES = ("hasf_reg.cu", "hasf_reg_kernel.cuh", "hasf_reg.cuh", "hasf_device.cuh",
                   "hasf_internal.h")


def _traffic_record(workload: str):
    """(record, stale): the headline kernel's last ncu capture (DRAM and L2
    bytes per launch) and whether the kernel sources have changed since it
    was taken (then the record is not used)."""
    import hashlib
    if workload != "batch512":
        return None, False
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "hasf_reg_kernel_traffic.json")))
    except Exception:
        return None, False
    src = b"".join(open(os.path.join(ROOT, "paper_1603_09337_gb300", "csrc", f), "rb").read()
                   for f in TRAFFIC_SOURCES)
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
        return None, True
    return rec, False


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU legs."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def measured_int_peaks(device: int):
    """Lane-operations per second of each integer instruction class on this
    GPU, from the probe kernels of libhasf_peak.so (CUDA events)."""
    import ctypes
    from paper_1603_09337_gb300 import build
    lib = ctypes.CDLL(build.PEAK_LIB)
    lib.hasf_peak_int.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_float)]
    out = {}
    for k, name in enumerate(("lop3", "shf", "iadd3", "shfl")):
        best = 0.0
        for _ in range(3):
            v, ms = ctypes.c_double(), ctypes.c_float()
            if lib.hasf_peak_int(k, device, ctypes.byref(v), ctypes.byref(ms)) == 0:
                best = max(best, v.value)
        out[name] = best / 1e12 if best else None
    return out


def alu_roofline(stats, ms_per_step, sms, sm_max_mhz, peaks_t):
    """The recipe's lane-operations per step over the step time, against the
    measured rate of its instruction mix (the time the recipe would take if
    every class ran at its measured rate, one after another)."""
    n = {"shf": 0, "lop3": 0}
    for key, mix in RECIPE_MIX.items():
        for cls, per in mix.items():
            n[cls] += stats[key] * per
    ops = sum(n.values())
    achieved = ops / (ms_per_step / 1e3) / 1e12
    nominal = sms * INT32_LANES_PER_SM * sm_max_mhz * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "unit": "Tops/s", "ops_per_step": ops,
            "counters": stats, "peak_nominal": nominal,
            "peak_nominal_source": f"{sms} SMs x 128 int32 lanes x {sm_max_mhz:.0f} MHz"}
    if peaks_t and all(peaks_t.get(c) for c in n):
        t_min = sum(n[c] / (peaks_t[c] * 1e12) for c in n)
        roof.update(peak=ops / t_min / 1e12, frac=achieved / (ops / t_min / 1e12),
                    peak_source="measured: per-class integer probe rates (hasf_peak_int) "
                                "weighted by the recipe's mix of funnel shifts and logic",
                    measured_class_peaks_tops=peaks_t)
    else:
        roof.update(peak=nominal, frac=achieved / nominal, peak_source="nominal (probe failed)")
    return roof


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
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
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
        for l in self.lines:
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
    import oracle
    X, C, rmax = args[:3]
    conn = args[3] if len(args) > 3 else 8
    st = oracle.Stats()
    t = time.perf_counter()
    oracle.hasf(X, rmax, C=C, conn=conn, stats=st)
    dt = time.perf_counter() - t
    # the sequential method's work: 9 simple tests per changed point plus
    # 4 * rmax EDTs of N points
    return dt, 9 * st.changes + 4 * rmax * X.size


def _pool(cores):
    import multiprocessing as mp
    import oracle
    oracle.build()
    return mp.get_context("spawn").Pool(cores)


def cpu_oracle_rate(jobs, cores):
    """Images/s of the oracle on `cores` host processes over `jobs`."""
    with _pool(cores) as pool:
        pool.map(_oracle_job, [(jobs[0].X, jobs[0].C, jobs[0].rmax, jobs[0].conn)] * cores)
        t0 = time.perf_counter()
        per = pool.map(_oracle_job, [(j.X, j.C, j.rmax, j.conn) for j in jobs], chunksize=1)
        wall = time.perf_counter() - t0
    cpu_oracle_rate.seq_ops_per_image = sum(p[1] for p in per) / max(1, len(per))
    return len(jobs) / wall, wall, sum(p[0] for p in per)


def run_reference(args):
    from paper_1603_09337_gb300 import replicas, synth
    ws, rank, _ = replicas.world()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    per_step = cores
    jobs = synth.batch_512(per_step * (args.steps + args.warmup))
    with _pool(cores) as pool:
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
        "cpu_baseline": {"value": value, "unit": "images/s", "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
                         "sample": f"{per_step * args.steps} images of the workload, "
                                   f"{per_step} per step, one oracle process per core"},
        "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --- serving: Poisson arrivals of mixed-size images -----------------------------------

def serving_pool(n: int = 48, seed: int = 4):
    """Images of the served stream: side lognormal (median 512, sigma 0.5), clipped
    to [128, 4096], aspect uniform in [0.5, 2], noise 2-10 %."""
    import math
    import numpy as np
    from paper_1603_09337_gb300 import synth
    rng = synth.SplitMix64(synth.image_seed(4, seed))
    out = []
    for i in range(n):
        u1 = (rng.next() >> 11) / float(1 << 53) or 1e-12
        u2 = (rng.next() >> 11) / float(1 << 53)
        z = math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
        s = min(4096.0, max(128.0, 512.0 * math.exp(0.5 * z)))
        a = 0.5 + 1.5 * (rng.next() >> 11) / float(1 << 53)
        w = int(min(4096, max(128, round(s * math.sqrt(a)))))
        h = int(min(4096, max(128, round(s / math.sqrt(a)))))
        area = w * h
        X = synth.shapes_image(synth.image_seed(4, 1000 + i), w, h,
                               max(1, (12 * area + 131072) // 262144), 20,
                               max(20, min(90, min(w, h) // 3)),
                               n_holes=(6 * area + 131072) // 262144, jitter=2,
                               noise_permille=rng.randint(20, 100))
        out.append(X)
    return out


def run_serving(ctx, dev, seconds: float, rate: float = 2000.0, seq_limit_s: float = 10.0):
    """Served stream vs plain sequential launches; latency = completion - arrival."""
    import numpy as np
    import torch
    from paper_1603_09337_gb300 import synth
    pool = serving_pool()
    ins = [torch.from_numpy(X).to(dev) for X in pool]
    slots = 8
    outs = [[torch.empty_like(t) for _ in range(slots)] for t in ins]
    free = [list(range(slots)) for _ in ins]
    rng = synth.SplitMix64(0xA77)
    n = int(rate * seconds)
    arrivals, picks, rmaxs = [], [], []
    t = 0.0
    import math
    for _ in range(n):
        u = ((rng.next() >> 11) + 1) / float(1 << 53)
        t += -math.log(u) / rate
        arrivals.append(t)
        picks.append(rng.randint(0, len(pool) - 1))
        rmaxs.append(rng.randint(1, 6))
    # warm-up: every image once
    for i, x in enumerate(ins):
        ctx.smooth(x, 3, out=outs[i][0])
    ctx.status()

    def served():
        lat = []
        pending = []           # (ticket, arrival, image, slot)
        waiting = []           # requests that arrived while their image had no free slot
        t0 = time.perf_counter()
        k = 0
        while k < n or pending or waiting:
            now = time.perf_counter() - t0
            while k < n and arrivals[k] <= now:
                waiting.append(k)
                k += 1
            still = []
            for q in waiting:
                i = picks[q]
                if free[i]:
                    sl = free[i].pop()
                    tk = ctx.submit(ins[i], rmaxs[q], outs[i][sl])
                    pending.append((tk, arrivals[q], i, sl))
                else:
                    still.append(q)
            waiting = still
            rest = []
            for tk, arr, i, sl in pending:
                done, st = ctx.poll(tk)
                if done:
                    lat.append(time.perf_counter() - t0 - arr)
                    free[i].append(sl)
                else:
                    rest.append((tk, arr, i, sl))
            pending = rest
        wall = time.perf_counter() - t0
        return lat, wall

    def sequential(limit_s: float):
        lat = []
        t0 = time.perf_counter()
        for q in range(n):
            now = time.perf_counter() - t0
            if now > limit_s:
                break
            if arrivals[q] > now:
                time.sleep(arrivals[q] - now)
            i = picks[q]
            ctx.smooth(ins[i], rmaxs[q], out=outs[i][0])
            ctx.status()
            lat.append(time.perf_counter() - t0 - arrivals[q])
        return lat, time.perf_counter() - t0

    s_lat, s_wall = served()
    q_lat, q_wall = sequential(seq_limit_s)
    pct = lambda a, p: float(np.percentile(np.array(a) * 1e3, p)) if a else None
    mpx = sum(pool[picks[q]].size for q in range(n)) / 1e6
    return {
        "arrival_rate_per_s": rate, "requests": n, "seconds": seconds,
        "images": f"pool of {len(pool)} images, sides lognormal(median 512, sigma 0.5) in "
                  "[128, 4096], aspect 0.5-2, noise 2-10%; rmax uniform 1-6 per request",
        "served": {"p50_ms": pct(s_lat, 50), "p99_ms": pct(s_lat, 99),
                   "images_per_s": len(s_lat) / s_wall, "mpixel_per_s": mpx / s_wall},
        "sequential_launches": {"p50_ms": pct(q_lat, 50), "p99_ms": pct(q_lat, 99),
                                "images_per_s": len(q_lat) / q_wall,
                                "completed": len(q_lat)},
    }


def single_image_latency(ctx, dev, flush, stream, reps: int = 50):
    """Latency of the single-image workload (512 x 512, 12 shapes, 6 holes,
    5 % noise, rmax 3, no C): CUDA events around each hasf_smooth call on
    `stream`, and around each hasf_smooth_noalloc call."""
    import ctypes
    import torch
    from paper_1603_09337_gb300 import _lib, synth
    job = synth.single_512()
    x = torch.from_numpy(job.X).to(dev)
    out = torch.empty_like(x)
    lib = _lib.load()
    d = _lib.HasfImage(x.data_ptr(), out.data_ptr(), None, None, 512, 512, 512, job.rmax, 8, 0)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    calls = {
        "hasf_smooth": lambda: ctx.smooth(x, job.rmax, out=out),
        "hasf_smooth_noalloc": lambda: _lib.check(
            lib.hasf_smooth_noalloc(ctypes.byref(d), ctypes.c_void_p(st.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream)), "noalloc"),
    }
    res = {"workload": "one 512x512 image (12 shapes, 6 holes, 2-px jitter, 5% noise), rmax=3, "
                       "no C, one call", "reps": reps,
           "l2": "flushed before each call (untimed)"}
    with ClockSampler(dev.index or 0) as clk:
        for name, call in calls.items():
            for _ in range(5):
                call()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                call()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            ctx.status()
            res[name] = {"best_ms": min(ts), "median_ms": statistics.median(ts),
                         "images_per_s": 1e3 / statistics.median(ts)}
    res["clocks"] = clk.summary()
    return res


def run_volume(args):
    """The 3D filter: a batch of 16 volumes of 128^3, rmax 4, through
    hasf_smooth3d."""
    import numpy as np
    import torch
    from paper_1603_09337_gb300 import Context, _lib, build, replicas, synth

    ws, rank, local = replicas.world()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    ctx = Context(local)
    simple_test = "flood fill" if args.simple3_flood else "table"
    ctx.set_option(_lib.OPT_SIMPLE3_TABLE, 0 if args.simple3_flood else 1)
    n = 16
    jobs = synth.volume_batch(n, 128, first=rank * n)
    Xs = [torch.from_numpy(j.X).to(dev) for j in jobs]
    vols = [(x, j.rmax, None, None) for x, j in zip(Xs, jobs)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.smooth3d(vols)
    ctx.status()
    ctx.read_stats()
    ctx.set_option(_lib.OPT_STATS, 1)
    ctx.smooth3d(vols)
    ctx.status()
    stats = ctx.read_stats()
    ctx.set_option(_lib.OPT_STATS, 0)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            ctx.smooth3d(vols)
            ends[i].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
    ctx.status()
    launches = ctx.read_stats()["launches"]
    t_ms = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, ends)), dev)
    ms_per_step = t_ms / args.steps
    value = n * args.steps * ws / (t_ms / 1e3)

    e2e = None
    if not args.no_e2e:
        hX = [torch.from_numpy(j.X).pin_memory() for j in jobs]
        hO = [torch.empty_like(h).pin_memory() for h in hX]
        k = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            dX = [h.to(dev, non_blocking=True) for h in hX]
            outs = ctx.smooth3d([(x, j.rmax, None, None) for x, j in zip(dX, jobs)])
            for o, h in zip(outs, hO):
                h.copy_(o, non_blocking=True)
            torch.cuda.synchronize()
        te = replicas.max_over_ranks((time.perf_counter() - t0) / k, dev)
        e2e = {"value": n * ws / te, "unit": "volumes/s",
               "h2d_bytes_per_step": int(sum(h.numel() for h in hX)),
               "d2h_bytes_per_step": int(sum(h.numel() for h in hO))}
    if rank != 0:
        ctx.close()
        return 0
    peaks, peak_src = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * INT32_LANES_PER_SM * sm_max * 1e6 / 1e12
    ops = (stats["word_tests"] * OPS_PER_VOXEL_TEST[simple_test]
           + stats["ring_evals"] * OPS_PER_RING3_EVAL)
    achieved = ops / (ms_per_step / 1e3) / 1e12
    vox = sum(x.numel() for x in Xs)
    cpu = None
    if not args.no_cpu and ws == 1:
        win = jobs[0].X[:32, :32, :32].copy()
        rate_w, cwall, cwork = cpu_oracle_rate3d(win, jobs[0].rmax)
        scale = win.size / jobs[0].X.size
        cpu = {"value": rate_w * scale, "unit": "volumes/s", "cores": 1, "kind": "oracle", "cpu": _cpu_model(),
               "sample": f"one 32^3 window of a volume, rmax {jobs[0].rmax}, one core, "
                         f"{cwork:.1f} s; volumes/s scaled by the voxel ratio {scale:.5f}"}
    line = {
        "metric": "HASF3D volumes/s at 128^3, rmax=4", "value": value, "unit": "volumes/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 bit planes (integer only)", "data": "synthetic",
        "config": {"workload": "batch of 16 synthetic 128^3 volumes (balls of radius 4-16, "
                               "3% noise), rmax=4, (26,6) adjacency, one hasf_smooth3d call",
                   "volumes_per_step": n, "mvoxel_per_s": vox * args.steps * ws / (t_ms / 1e3) / 1e6,
                   "simple_voxel_test": simple_test,
                   "l2": "flushed between timed steps (256 MB write, untimed)", "wall_s": wall},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                     "frac": achieved / alu_peak, "traffic": None,
                     "peak_source": f"{sms} SMs x 128 int32 lanes x max SM clock (nominal)",
                     "ops_per_step": ops, "counters": stats},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _oracle3d_job(args):
    import oracle
    X, rmax = args
    t = time.perf_counter()
    oracle.hasf3d(X, rmax)
    return time.perf_counter() - t


def cpu_oracle_rate3d(X, rmax):
    """Volumes/s of the 3D oracle on one host process over X."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(1) as pool:
        t0 = time.perf_counter()
        dt = pool.map(_oracle3d_job, [(X, rmax)])[0]
        wall = time.perf_counter() - t0
    return 1.0 / dt, wall, dt


def run_hasf(args):
    import numpy as np
    import torch
    from paper_1603_09337_gb300 import Context, Image, build, replicas, synth

    ws, rank, local = replicas.world()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    ctx = Context(local)

    if args.workload == "batch512":
        jobs = synth.batch_512(BATCH, first=rank * BATCH)
        workload, metric = WORKLOAD, METRIC
    elif args.workload == "ragged":
        jobs = synth.ragged_batch(args.ragged_n, first=rank * args.ragged_n)
        workload = (f"ragged batch of {args.ragged_n} images, sides uniform 128-2048, "
                    "rmax uniform 1-8, one batched launch")
        metric = "HASF images/s, ragged batch"
    else:
        jobs = [synth.large_image(args.side)]
        workload = f"one {args.side}x{args.side} image of 2,000 discs/ellipses, 3% noise, rmax=10"
        metric = f"HASF images/s at {args.side}x{args.side}, rmax=10"
    if args.conn == 4:
        for j in jobs:
            j.conn = 4
        workload += "; (4,8) adjacency"
        metric += ", (4,8)"
    n = len(jobs)
    Xs = [torch.from_numpy(j.X).to(dev) for j in jobs]
    Cs = [torch.from_numpy(j.C).to(dev) if j.C is not None else None for j in jobs]
    outs = [torch.empty_like(x) for x in Xs]
    imgs = [Image(Xs[i], jobs[i].rmax, C=Cs[i], out=outs[i], conn=jobs[i].conn)
            for i in range(n)]
    arr = ctx.batch_descriptors(imgs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    graph = ctx.graph_create(imgs) if args.graph else None

    def step():
        if graph is not None:
            ctx.graph_launch(graph)
        else:
            ctx.smooth_batch_raw(arr, n)

    for _ in range(args.warmup):
        step()
    ctx.status()
    stats = ctx.stats_step(arr, n)          # work counters of one step (untimed run)

    ctx.read_stats()                        # resets the launch counter
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()                       # evict L2 (129 MB) between steps, untimed
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
    ctx.status()
    launches = ctx.read_stats()["launches"]   # kernel launches inside the timed region
    if graph is not None:
        launches = stats["launches"] * args.steps  # the graph holds one step's launches
        ctx.graph_destroy(graph)
    t_ms = replicas.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), dev)
    value = n * args.steps * ws / (t_ms / 1e3)
    ms_per_step = t_ms / args.steps

    # The same step as plain per-image launches: one hasf_smooth per image on
    # the same stream (the alternative to the batched launch).
    per_image = None
    if args.workload != "large" and not args.no_per_image:
        for i in range(n):
            ctx.smooth(Xs[i], jobs[i].rmax, C=Cs[i], out=outs[i], conn=jobs[i].conn)
        ctx.status()
        k = 1 if args.workload == "ragged" else max(1, min(args.steps, 3))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(stream)
        for _ in range(k):
            for i in range(n):
                ctx.smooth(Xs[i], jobs[i].rmax, C=Cs[i], out=outs[i], conn=jobs[i].conn)
        b.record(stream)
        barrier()
        ctx.status()
        tp = replicas.max_over_ranks(a.elapsed_time(b) / k, dev)
        per_image = {"value": n * ws / (tp / 1e3), "unit": "images/s", "ms_per_step": tp,
                     "launches_per_step": n, "steps": k}

    # The single-image workload: one 512 x 512 image, rmax 3, one launch --
    # a latency figure (best and median of 50 launches after warm-up, L2
    # flushed before each), through hasf_smooth and through the
    # allocation-free entry point.
    single = None
    if args.workload == "batch512" and rank == 0:
        single = single_image_latency(ctx, dev, flush, stream)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    int_peaks = measured_int_peaks(local)

    # End to end through the host-buffer entry point with pinned host buffers:
    # H2D of X and C, the smoothing, D2H of the result, every step.
    e2e = None
    if not args.no_e2e:
        hX = [torch.from_numpy(j.X).pin_memory().numpy() for j in jobs]
        hC = [torch.from_numpy(j.C).pin_memory().numpy() if j.C is not None else None
              for j in jobs]
        hO = [torch.empty(j.X.shape, dtype=torch.uint8).pin_memory().numpy() for j in jobs]
        host_jobs = [(hX[i], jobs[i].rmax, hC[i], None, jobs[i].conn, hO[i]) for i in range(n)]
        # the buffers are described once, like the device batch's descriptors;
        # every step moves all inputs and results across the host link
        harr = ctx.host_descriptors(host_jobs)
        ctx.smooth_host_raw(harr, n)                   # warm-up
        k = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            ctx.smooth_host_raw(harr, n)
        barrier()
        te = replicas.max_over_ranks((time.perf_counter() - t0) / k, dev)
        e2e = {"value": n * ws / te, "unit": "images/s",
               "h2d_bytes_per_step": int(sum(a.nbytes for a in hX) +
                                         sum(a.nbytes for a in hC if a is not None)),
               "d2h_bytes_per_step": int(sum(a.nbytes for a in hO)),
               "api": "hasf_smooth_host on pinned host buffers described once "
                      "(Context.host_descriptors / smooth_host_raw), wall clock per call"}

    serving = None
    if rank == 0 and args.serve_seconds > 0 and args.workload == "batch512":
        serving = run_serving(ctx, dev, args.serve_seconds, seq_limit_s=args.sequential_seconds)

    if rank != 0:
        ctx.close()
        return 0

    peaks, peak_src = _peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    roof = alu_roofline(stats, ms_per_step, sms, sm_max, int_peaks)
    rec, stale = _traffic_record(args.workload)
    roof["traffic"] = None if rec is None else rec["dram_bytes_read"] + rec["dram_bytes_write"]
    if stale:
        roof["traffic_stale"] = True   # the ncu record predates the kernel sources timed here
    if rec is not None:
        # the same kernel's issue-slot and integer-pipe use (ncu): how much of
        # the issue peak it really occupies, algorithmic work or not
        roof["ncu_issue_active_pct"] = rec.get("issue_active_pct")
        roof["ncu_alu_pipe_pct"] = rec.get("alu_pipe_pct")
        roof["ncu_warps_active"] = rec.get("warps_active")
    in_bytes = sum(x.numel() for x in Xs) + sum(c.numel() for c in Cs if c is not None)
    alg_bytes = in_bytes + sum(o.numel() for o in outs)
    gbs = alg_bytes / (ms_per_step / 1e3) / 1e9
    hbm = {"achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
           "traffic_stale": stale,
           "ncu_dram_bytes_per_launch": None if rec is None else
           rec["dram_bytes_read"] + rec["dram_bytes_write"],
           "ncu_l2_bytes_per_launch": None if rec is None else rec.get("lts_bytes"),
           "l2_gbs": None if rec is None or not rec.get("lts_bytes") else
           rec["lts_bytes"] / (ms_per_step / 1e3) / 1e9,
           "peak_source": peak_src, "algorithmic_bytes_per_step": alg_bytes}

    cpu = None
    if not args.no_cpu and ws == 1 and args.workload != "large":
        cores = os.cpu_count() or 1
        if args.workload == "batch512":
            sample = synth.batch_512(2 * cores, first=10_000)
        else:
            sample = synth.ragged_batch(cores, first=100_000)
        for j in sample:
            j.conn = args.conn
        rate, cwall, cwork = cpu_oracle_rate(sample, cores)
        cpu = {"value": rate, "unit": "images/s", "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
               "sample": f"{len(sample)} images of the workload (other seeds), one oracle "
                         f"process per core, {cwork:.1f} s of CPU work in {cwall:.1f} s",
               "sequential_method_ops_per_image": cpu_oracle_rate.seq_ops_per_image}
    elif not args.no_cpu and ws == 1:
        # One full image takes the oracle minutes: time a 1024 x 1024 window of
        # it instead and scale by pixels (the work per pixel of a window is
        # that of the whole image up to border effects).
        cores = os.cpu_count() or 1
        win = jobs[0].X[:1024, :1024].copy()
        rate_w, cwall, cwork = cpu_oracle_rate([synth.Job(win, jobs[0].rmax, conn=args.conn)], 1)
        scale = win.size / jobs[0].X.size
        cpu = {"value": rate_w * scale, "unit": "images/s", "cores": 1, "kind": "oracle", "cpu": _cpu_model(),
               "sample": f"one 1024x1024 window of the image, rmax {jobs[0].rmax}, one core, "
                         f"{cwork:.1f} s; images/s scaled by the pixel ratio {scale:.4f}"}

    px = sum(x.numel() for x in Xs)
    line = {
        "metric": metric, "value": value, "unit": "images/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit planes (integer only)",
        "data": "synthetic",
        "config": {"workload": workload, "images_per_step": n,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "launch": "CUDA graph replay" if args.graph else "hasf_smooth_batch",
                   "mpixel_per_s": px * args.steps * ws / (t_ms / 1e3) / 1e6, "wall_s": wall},
        "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e,
        "per_image_launches": per_image, "single_image": single, "serving": serving,
        "gpu_launches": launches,
        "clocks": clocks,
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
    ap.add_argument("--workload", default="batch512",
                    choices=["batch512", "ragged", "large", "volume"])
    ap.add_argument("--ragged-n", type=int, default=1024)
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--sequential-seconds", type=float, default=10.0,
                    help="time limit of the plain sequential launches the served stream is "
                         "compared with")
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-per-image", action="store_true",
                    help="skip the one-launch-per-image comparison")
    ap.add_argument("--conn", type=int, default=8, choices=[8, 4],
                    help="adjacency of the object: 8 = (8,4), 4 = (4,8)")
    ap.add_argument("--simple3-flood", action="store_true",
                    help="volume workload: simple-voxel test by flood fill, not the table")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "volume":
        return run_volume(args)
    return run_hasf(args)


if __name__ == "__main__":
    sys.exit(main())
