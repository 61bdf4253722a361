#!/usr/bin/env python
"""Benchmark: multi-octave polynomial-noise heightmap generation on GB300.

Workload (one step = one pass of the whole generation path): a 2D heightmap of
8192 x 8192 samples, 12 octaves, base lattice 8 x 8 cells (1024 samples per
cell), C1 polynomial cells, persistence 0.5, lacunarity 2, FP32 output, seeds
cycling 0..3 (Thorimbert & Chopard, arXiv:1610.03525: cell polynomial of
Sec. 3, fractal sum of Sec. 4).  The output (268 MB) is larger than L2, so no
flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gsamples/s and % of roofline (8192² 12-oct C1) vs Perlin/OpenSimplex; p50/p99"
UNIT = "Gsamples/s"
SIZE, SPC, OCTAVES = (8192, 8192), 1024, 12
WORKLOAD = "2D heightmap 8192x8192, 12 octaves, base lattice 8x8 (spc 1024), C1, p=0.5, L=2, FP32 out, seeds 0..3"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard_seed(rank: int, step: int) -> int:
    """Seed of a step on a rank: each rank makes its own fields (weak scaling,
    no data exchange); seeds 0..3 cycle per step as in the workload."""
    return (rank * 4 + step % 4) % (1 << 24)


def aggregate_max(value: float, world: int):
    """Max of a per-rank value over all ranks (identity at world size 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples (200 ms period) in the background."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        inside = [p for (t, p) in self.samples if t0 - 0.05 <= t <= t1 + 0.05]
        src = "timed_region"
        if len(inside) < 3:
            inside = [p for (t, p) in self.samples]
            src = "timed_region_and_adjacent_window"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[2]) for p in inside if num(p[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in inside:
            for k, n in enumerate(names):
                if p[6 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(inside[0][3]),
                "power_w_max": max((num(p[4]) or 0.0) for p in inside), "reasons": sorted(reasons),
                "samples": len(inside), "source": src}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    """sha256 (first 16 hex digits) of the sources of the fused 2D generator."""
    import hashlib
    h = hashlib.sha256()
    for f in ("ptg_fbm2d.cu", "ptg_device.cuh", "ptg_eval.cuh"):
        with open(os.path.join(ROOT, "paper_1610_03525_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per launch of the timed kernel, from the machine-readable
    sidecar of its committed ncu capture (profiles/fbm2d_c1_8192_n12.json),
    if that capture was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "fbm2d_c1_8192_n12.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, TypeError, ValueError):
        return None


def oracle_sample_rate(rows: int, seed: int = 0, threads: int = 0):
    """Oracle throughput on `rows` distinct full rows of the workload, evenly
    spread over the field, on `threads` host threads (0 = all).  Returns
    (samples/s, samples, seconds, threads)."""
    import numpy as np
    import oracle as O
    ys = np.unique(np.linspace(0, SIZE[1] - 1, max(1, rows)).astype(np.int64))
    idx = np.concatenate([np.stack([np.arange(SIZE[0]), np.full(SIZE[0], y)], 1) for y in ys]).astype(np.int64)
    O.lib()
    t0 = time.perf_counter()
    O.field_samples(2, (SPC, SPC), (1, 1), idx, octaves=OCTAVES, method=O.C1, seed=seed, persistence=0.5,
                    nthreads=threads)
    dt = time.perf_counter() - t0
    return idx.shape[0] / dt, idx.shape[0], dt, threads if threads > 0 else O.num_threads()


def oracle_small_fields():
    """The oracle on the whole 256^2, 6-octave, spc-64 field (C1, Perlin S5,
    OpenSimplex), all host threads: seconds and samples/s of each."""
    import oracle as O
    res = {}
    for name, method in [("c1", O.C1), ("perlin_s5", O.PERLIN_S5), ("opensimplex", O.OPENSIMPLEX)]:
        t0 = time.perf_counter()
        O.field_grid(2, (256, 256), (4, 4), octaves=6, method=method, seed=0, persistence=0.5)
        dt = time.perf_counter() - t0
        res[name] = {"seconds": round(dt, 4), "gsamples_s": 256 * 256 / dt / 1e9}
    return res


def bench_3d(P, R, ctx, stream, torch, reps=10):
    """512^3, 8 octaves, spc 128, C1, FP16 output, origin (2^20, 2^20, 0); and
    Perlin S5 and OpenSimplex on the same volume as the 3D baselines."""
    size = (512, 512, 512)
    out = torch.empty((512, 512, 512), dtype=torch.float16, device="cuda")
    peak = R.alu_peak(torch.cuda.get_device_properties(0).multi_processor_count, 2070.0)
    res = {"workload": "3D 512^3, 8 octaves, spc 128 (4^3 base cells), FP16 out, origin (2^20, 2^20, 0)"}
    for name, fn, kw in [("c1", P.ptg_field, dict(smoothness=P.PTG_C1)),
                         ("perlin_s5", P.ptg_perlin, dict(variant=P.PTG_PERLIN_S5)),
                         ("opensimplex", P.ptg_opensimplex, dict())]:
        d = P.make_desc(dims=3, size=size, spc=128, origin=(1 << 20, 1 << 20, 0), octaves=8, seed=0,
                        dtype=P.PTG_F16, **kw)
        for _ in range(3):
            fn(ctx, d, out, stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = 2 if name == "opensimplex" else reps
        for _ in range(n):
            fn(ctx, d, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        ops = R.lane_ops_3d(name, size, 128, 8)
        res[name] = {"gsamples_s": 512 ** 3 / ms / 1e6, "ms": ms, "ops_per_sample": ops["per_sample"],
                     "alu_frac": ops["total"] / (ms / 1e3) / peak}
        if name != "opensimplex":
            res[name]["frac_vs_bound"] = R.bound_ops(name, size, 128, 8)["total"] / (ms / 1e3) / peak
    # ridged noise on the same volume: the fused ridged kernel, and the per-sample generator
    # on the same volume one sample off the cell grid (where the fused kernel does not apply)
    ridged = {}
    for name, fn, kw, off in [("c1", P.ptg_field, dict(smoothness=P.PTG_C1), 0),
                              ("perlin_s5", P.ptg_perlin, dict(variant=P.PTG_PERLIN_S5), 0),
                              ("c1_per_sample", P.ptg_field, dict(smoothness=P.PTG_C1), 1)]:
        kw = dict(kw)
        kw["variant"] = kw.get("variant", 0) | P.PTG_RIDGED
        d = P.make_desc(dims=3, size=size, spc=128, origin=(1 << 20, 1 << 20, 0), offset=(off, 0, 0), octaves=8,
                        seed=0, dtype=P.PTG_F16, **kw)
        for _ in range(2):
            fn(ctx, d, out, stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 2 if off else reps
        a.record(stream)
        for _ in range(n):
            fn(ctx, d, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        ridged[name] = {"gsamples_s": 512 ** 3 / ms / 1e6, "ms": ms}
    res["ridged"] = ridged
    del out
    return res


def bench_small_field(P, ctx, stream, torch, reps=500):
    """The 256^2, 6-octave, spc-64 field (FP32): device time per field over
    back-to-back launches, and the host time of one ptg_* call (argument
    checks, plan, launch)."""
    out = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    res = {"workload": "2D 256^2, 6 octaves, spc 64 (4x4 base cells), FP32, %d launches back to back" % reps}
    for name, fn, kw in [("c1", P.ptg_field, dict(smoothness=P.PTG_C1)),
                         ("perlin_s5", P.ptg_perlin, dict()),
                         ("opensimplex", P.ptg_opensimplex, dict())]:
        d = P.make_desc(dims=2, size=(256, 256), spc=64, octaves=6, seed=0, **kw)
        for _ in range(10):
            fn(ctx, d, out, stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        for _ in range(reps):
            fn(ctx, d, out, stream)
        b.record(stream)
        host_us = (time.perf_counter() - t0) / reps * 1e6
        torch.cuda.synchronize()
        us = a.elapsed_time(b) / reps * 1e3
        res[name] = {"us_per_field": round(us, 2), "host_us_per_call": round(host_us, 2),
                     "gsamples_s": 256 * 256 / us / 1e3}
    del out
    return res


def bench_octave_sweep(P, ctx, stream, torch, octaves=(1, 2, 4, 6, 8, 10, 12), reps=5):
    """Time per 8192^2 field against the octave count N (spc 1024: octaves
    10 and 11 sit on lattice points), per method -- the GPU counterpart of the
    paper's execution time against N at fixed resolution (Sec. 5.2)."""
    out = torch.empty((SIZE[1], SIZE[0]), dtype=torch.float32, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, fn, kw in [("c1", P.ptg_field, dict(smoothness=P.PTG_C1)),
                         ("zero_gradient", P.ptg_field, dict(smoothness=P.PTG_ZERO_GRADIENT)),
                         ("perlin_s5", P.ptg_perlin, dict()),
                         ("opensimplex", P.ptg_opensimplex, dict())]:
        row = {}
        for n in octaves:
            d = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=n, seed=0, **kw)
            fn(ctx, d, out, stream)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(reps):
                fn(ctx, d, out, stream)
            b.record(stream)
            torch.cuda.synchronize()
            row[str(n)] = round(a.elapsed_time(b) / reps, 4)
        res[name + "_ms"] = row
    del out
    return res


def bench_batched(P, ctx, stream, torch, n_chunks=4096, reps=5):
    """4096 2D chunks (side 64..1024, octaves 4..12, C1/C2) in one persistent
    launch replayed from a CUDA graph, against one ptg_field launch per chunk."""
    from paper_1610_03525_gb300 import workloads as Wl
    chunks = Wl.chunk_batch(n_chunks)
    descs, outs = [], []
    for c in chunks:
        descs.append(P.make_desc(dims=2, size=c["size"], spc=c["spc"], origin=c["origin"], octaves=c["octaves"],
                                 smoothness=c["smoothness"], seed=c["seed"]))
        outs.append(torch.empty((c["size"][1], c["size"][0]), dtype=torch.float32, device="cuda"))
    n_samples = sum(c["size"][0] * c["size"][1] for c in chunks)
    shapes = {}
    for d in descs:
        rw, nt = P.ptg_launch_config(ctx, d)
        key = "%dx%d%s" % (rw, 32 // rw, " tile" if nt else "")
        shapes[key] = shapes.get(key, 0) + 1
    plan = P.ptg_batch_prepare(ctx, descs, outs)
    for _ in range(2):
        P.ptg_batch_launch(plan, stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        P.ptg_batch_launch(plan, stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_batch = a.elapsed_time(b) / reps
    P.ptg_batch_free(plan)

    def per_chunk():
        for d, o in zip(descs, outs):
            P.ptg_field(ctx, d, o, stream)
    per_chunk()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a.record(stream)
    for _ in range(reps):
        per_chunk()
    b.record(stream)
    torch.cuda.synchronize()
    wall_single = (time.perf_counter() - t0) * 1e3 / reps
    ms_single = a.elapsed_time(b) / reps
    del outs
    return {"workload": "%d 2D chunks, side log-uniform 64..1024, octaves 4..12, C1/C2 50/50, spc 1024, "
                        "seeds = chunk id, origins uniform in +-2^20 cells, FP32 out" % n_chunks,
            "samples": n_samples, "launch_configs": shapes,
            "batched_graph_ms": ms_batch, "batched_gsamples_s": n_samples / ms_batch / 1e6,
            "per_chunk_launches_ms": ms_single, "per_chunk_gsamples_s": n_samples / ms_single / 1e6,
            "per_chunk_host_wall_ms": wall_single,
            "speedup": ms_single / ms_batch}


def bench_quality(P, ctx, stream, torch):
    """The paper's map statistics on the device (Sec. 5.3, 5.1): coastline
    fractal dimension D (level 0, box sides 2..64 samples) against the octave
    count N for R = 1024 maps with base frequency 2 (spc 512), p = 0.5, four
    seeds; and the height / slope-norm distributions of 100 maps of 512^2
    (N = 8, spc 256), with the statistics kernels' times."""
    import numpy as np
    res = {"workload": "D: 1024^2, spc 512, p 0.5, seeds 0..3, boxes 2..64; distributions: 100 maps 512^2, N 8"}
    m = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    kinds = [("c1", P.ptg_field, dict(smoothness=P.PTG_C1)),
             ("zero_gradient", P.ptg_field, dict(smoothness=P.PTG_ZERO_GRADIENT)),
             ("perlin_s5", P.ptg_perlin, dict(variant=P.PTG_PERLIN_S5))]
    for name, fn, kw in kinds:
        ds = {}
        for N in (1, 2, 3, 4, 6, 8, 10):
            vals = []
            for seed in range(4):
                d = P.make_desc(dims=2, size=(1024, 1024), spc=512, octaves=N, seed=seed, **kw)
                fn(ctx, d, m, stream)
                vals.append(P.box_dimension(P.ptg_box_counts(ctx, m, 0.0, 7, stream), 1, 6))
            ds[str(N)] = round(float(np.mean(vals)), 4)
        res[name + "_D_vs_N"] = ds
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    for _ in range(10):
        P.ptg_box_counts(ctx, m, 0.0, 7, stream)
    res["box_counts_ms_1024"] = (time.perf_counter() - t0) * 100.0
    del m
    maps = torch.empty((100, 512, 512), dtype=torch.float32, device="cuda")
    for name, fn, kw in kinds:
        for k in range(100):
            d = P.make_desc(dims=2, size=(512, 512), spc=256, octaves=8, seed=k, **kw)
            fn(ctx, d, maps[k], stream)
        out = {}
        for what, lo, hi, bins in [(0, -2.0, 2.0, 80), (1, 0.0, 0.1, 100)]:
            P.ptg_histogram(ctx, maps, lo, hi, bins, what, stream=stream)  # warm-up
            a.record(stream)
            hist = P.ptg_histogram(ctx, maps, lo, hi, bins, what, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            h = hist.cpu().numpy().astype(np.float64)[1:-1]
            centres = lo + (np.arange(bins) + 0.5) * (hi - lo) / bins
            mean = float((h * centres).sum() / h.sum())
            std = float(np.sqrt((h * (centres - mean) ** 2).sum() / h.sum()))
            key = "height" if what == 0 else "slope"
            out[key] = {"mean": round(mean, 5), "std": round(std, 5), "ms": round(a.elapsed_time(b), 4)}
        res[name + "_distributions"] = out
    del maps
    return res


def bench_serving(P, torch, duration_s=10.0, warmup_s=1.0, rate_hz=20000.0, budget=40 << 30, slots=256):
    """Poisson request stream through ptg_submit / ptg_poll (80% 2D 128..2048,
    20% 3D 32..256, octaves 4..12, C1/C2) under a 40 GB budget."""
    from paper_1610_03525_gb300 import workloads as Wl
    ctx = P.ptg_create(torch.cuda.current_device(), budget)
    reqs = Wl.request_stream(rate_hz=rate_hz, duration_s=duration_s + warmup_s)
    slot_bytes = 256 ** 3 * 4
    pool = torch.empty((slots, slot_bytes // 4), dtype=torch.float32, device="cuda")
    descs = [P.make_desc(dims=r["dims"], size=r["size"], spc=r["spc"], origin=r["origin"], octaves=r["octaves"],
                         smoothness=r["smoothness"], seed=r["seed"]) for r in reqs]
    # warm the kernels
    for d in descs[:64]:
        P.ptg_field(ctx, d, pool[0].data_ptr(), 0)
    torch.cuda.synchronize()
    free = list(range(slots))
    inflight = {}
    lat = []
    samples_done = 0
    stalls = 0
    t0 = time.perf_counter()
    k = 0
    first_measured = None
    last_end_ns = 0
    first_submit_ns = None
    while k < len(reqs) or inflight:
        now = time.perf_counter() - t0
        while k < len(reqs) and reqs[k]["t"] <= now:
            if not free:
                stalls += 1
                break
            sl = free.pop()
            rid = P.ptg_submit(ctx, descs[k], pool[sl].data_ptr())
            inflight[rid] = (sl, k)
            k += 1
        for rid in list(inflight.keys()):
            st, ts = P.ptg_poll(ctx, rid)
            if st == P.PTG_PENDING:
                continue
            sl, kk = inflight.pop(rid)
            free.append(sl)
            if reqs[kk]["t"] >= warmup_s:
                lat.append((ts[3] - ts[0]) / 1e6)
                n = 1
                for v in reqs[kk]["size"]:
                    n *= v
                samples_done += n
                if first_submit_ns is None:
                    first_submit_ns = ts[0]
                last_end_ns = max(last_end_ns, ts[3])
    ctx.close()
    del pool
    lat.sort()
    span_s = (last_end_ns - first_submit_ns) / 1e9 if first_submit_ns else float("nan")
    return {"workload": "Poisson %g req/s for %.1f s after %.1f s warm-up; 80%% 2D side 128..2048 (spc 1024), "
                        "20%% 3D side 32..256 (spc 128); octaves 4..12; C1/C2 50/50; 40 GB budget" % (
                            rate_hz, duration_s, warmup_s),
            "requests": len(lat), "p50_ms": lat[len(lat) // 2], "p99_ms": lat[int(0.99 * (len(lat) - 1))],
            "sustained_gsamples_s": samples_done / span_s / 1e9, "client_slot_stalls": stalls}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    rows = max(1, args.ref_rows)
    for _ in range(args.warmup):
        oracle_sample_rate(1)
    per = []
    tot_samples = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        rate, n, dt, threads = oracle_sample_rate(rows, seed=k % 4)
        per.append(dt)
        tot_samples += n
    elapsed = time.perf_counter() - t0
    value = tot_samples / elapsed / 1e9
    sample = "%d full rows (%d samples) of the 8192^2 field per step, oracle FP64, %d threads" % (
        rows, rows * SIZE[0], threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=32)
    ap.add_argument("--cpu-rows", type=int, default=1536, help="oracle rows for the cpu_baseline sample")
    ap.add_argument("--no-extras", action="store_true", help="skip baselines, e2e and the oracle leg")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="measured seconds of the serving stream")
    ap.add_argument("--tune-cache", default=None,
                    help="thread-shape table: loaded if present (and written for this GPU), else timed and written")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1610_03525_gb300 import build as _build
    _build.build()
    import paper_1610_03525_gb300 as P
    from paper_1610_03525_gb300 import roofline as R

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ctx = P.ptg_create(local)
    t_tune = time.perf_counter()
    P.ptg_autotune(ctx, 0, args.tune_cache)  # 2D thread shape per octave structure, timed on this GPU
    t_tune = time.perf_counter() - t_tune
    stream = torch.cuda.current_stream()
    n_samples = SIZE[0] * SIZE[1]
    out = torch.empty((SIZE[1], SIZE[0]), dtype=torch.float32, device="cuda")
    descs = [P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, smoothness=P.PTG_C1, persistence=0.5,
                         seed=shard_seed(rank, k)) for k in range(4)]

    def step(k):
        P.ptg_field(ctx, descs[k % 4], out, stream)

    for k in range(args.warmup):
        step(k)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)  # let the sampler take its first readings
    barrier()
    # The timed region holds the steps alone (an event pair around every step
    # would add about 4.5 us a step between the launches); each step is one
    # generator launch, so the region's mean is the mean launch duration.
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    t_start.record(stream)
    for k in range(args.steps):
        step(k)
    t_end.record(stream)
    barrier()
    wall1 = time.time()
    # adjacent window of identical work for clock readings when the timed
    # region is shorter than the sampling period
    while time.time() - wall1 < 1.0:
        for k in range(8):
            step(k)
        torch.cuda.synchronize()
    sampler.stop()
    clocks = sampler.summary(wall0, wall1)
    local_ms = t_start.elapsed_time(t_end)
    max_ms = aggregate_max(local_ms, world)
    value = world * n_samples * args.steps / (max_ms / 1e3) / 1e9
    avg_launch_s = local_ms / args.steps / 1e3
    # per-launch spread (p50 / p99): a second pass of the same steps, an event
    # pair around each launch, outside the timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    per = sorted(a.elapsed_time(b) for a, b in ev)

    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = R.alu_peak(props.multi_processor_count, sm_max)
    rw, nt = P.ptg_launch_config(ctx, descs[0])
    ops = R.lane_ops_2d("c1", SIZE, SPC, OCTAVES, rw, nt)
    achieved = ops["total"] / avg_launch_s
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tlane-ops/s",
            "frac": achieved / peak, "traffic": profile_traffic(),
            "ops_per_launch": ops["total"], "ops_per_sample": ops["per_sample"],
            "peak_source": "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)" % (
                props.multi_processor_count, sm_max, peak_src),
            "hbm_write_gbs": n_samples * 4 / avg_launch_s / 1e9,
            "hbm_frac": n_samples * 4 / avg_launch_s / 1e9 / float(peaks.get("hbm_gbs", 6800.0))}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / R.alu_peak(props.multi_processor_count, clocks["sm_mhz"])
    # kernel-independent lower bound of the work (each distinct corner and
    # lattice sample hashed once, the octave sum combined per sample)
    bnd = R.bound_ops("c1", SIZE, SPC, OCTAVES)
    roof["bound_ops_per_sample"] = bnd["per_sample"]
    roof["frac_vs_bound"] = bnd["total"] / avg_launch_s / peak
    roof["frac_note"] = ("frac: the kernel's counted arithmetic over the issue peak (the 0.70 target); "
                         "frac_vs_bound: the method's irreducible work over the same peak")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": world, "samples_per_step": world * n_samples,
                   "parallelism": "replicas (independent fields per rank)" if world > 1 else "single GPU",
                   "l2": "output 268 MB > 129 MB L2 each step; no flush",
                   "launch_config": "thread shape %dx%d, %d octaves at the tile nodes (autotuned in %.2f s)" % (
                       rw, 32 // rw, nt, t_tune)},
        "p50_ms": per[len(per) // 2], "p99_ms": per[min(len(per) - 1, int(0.99 * len(per)))],
        "p50_p99_note": "per-launch spread from a second pass of the same steps with an event pair around each "
                        "launch, outside the timed region",
        "gpu_launches": args.steps,
        "roofline": roof,
        "clocks": clocks,
    }

    if not args.no_extras:
        # same-GPU baselines and variants at the same size and octave count
        extras = {}
        n_ex = max(5, min(args.steps, 50))

        def time_fn(fn, dtype=torch.float32, reps=n_ex):
            o = torch.empty((SIZE[1], SIZE[0]), dtype=dtype, device="cuda")
            for _ in range(3):
                fn(o)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn(o)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            del o
            return {"gsamples_s": n_samples / ms / 1e6, "ms": ms}
        dC2 = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, smoothness=P.PTG_C2, seed=0)
        d16 = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, smoothness=P.PTG_C1, seed=0,
                          dtype=P.PTG_F16)
        dP = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, seed=0, variant=P.PTG_PERLIN_S5)
        dZ = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, smoothness=P.PTG_ZERO_GRADIENT, seed=0)
        dG = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, smoothness=P.PTG_PAPER_D2M1N3, seed=0)
        extras["c2_f32"] = time_fn(lambda o: P.ptg_field(ctx, dC2, o, stream))
        extras["c1_f16"] = time_fn(lambda o: P.ptg_field(ctx, d16, o, stream), torch.float16)
        extras["perlin_s5_f32"] = time_fn(lambda o: P.ptg_perlin(ctx, dP, o, stream))
        extras["zero_gradient_f32"] = time_fn(lambda o: P.ptg_field(ctx, dZ, o, stream))
        extras["paper_d2m1n3_f32"] = time_fn(lambda o: P.ptg_field(ctx, dG, o, stream))
        extras["opensimplex_f32"] = time_fn(lambda o: P.ptg_opensimplex(ctx, dP, o, stream), reps=5)
        ex_desc = {"c2_f32": (dC2, P.METHOD_FIELD), "c1_f16": (d16, P.METHOD_FIELD),
                   "perlin_s5_f32": (dP, P.METHOD_PERLIN), "zero_gradient_f32": (dZ, P.METHOD_FIELD),
                   "paper_d2m1n3_f32": (dG, P.METHOD_FIELD), "opensimplex_f32": (None, None)}
        for k, v in extras.items():
            d_k, m_k = ex_desc[k]
            rw_k, nt_k = P.ptg_launch_config(ctx, d_k, m_k) if d_k is not None else (8, 0)
            if d_k is not None:
                v["launch_config"] = "%dx%d, %d tile octaves" % (rw_k, 32 // rw_k, nt_k)
            v["ops_per_sample"] = R.lane_ops_2d({"c2_f32": "c2", "c1_f16": "c1", "perlin_s5_f32": "perlin_s5",
                                                 "zero_gradient_f32": "zero_grad",
                                                 "paper_d2m1n3_f32": "paper_gauge",
                                                 "opensimplex_f32": "opensimplex"}[k], SIZE, SPC,
                                                OCTAVES, rw_k, nt_k)["per_sample"]
            v["alu_frac"] = v["ops_per_sample"] * n_samples / (v["ms"] / 1e3) / peak
            bk = {"c2_f32": "c2", "c1_f16": "c1", "perlin_s5_f32": "perlin_s5", "zero_gradient_f32": "zero_grad",
                  "paper_d2m1n3_f32": "paper_gauge"}.get(k)
            if bk:
                v["frac_vs_bound"] = R.bound_ops(bk, SIZE, SPC, OCTAVES)["total"] / (v["ms"] / 1e3) / peak
        line["baselines"] = extras
        # any frequency ratio between octaves (per-sample generator), same size and octave count
        general = {}
        for name, fn, kw in [("c1", P.ptg_field, dict(smoothness=P.PTG_C1)),
                             ("zero_gradient", P.ptg_field, dict(smoothness=P.PTG_ZERO_GRADIENT)),
                             ("perlin_s5", P.ptg_perlin, dict(variant=P.PTG_PERLIN_S5)),
                             ("opensimplex", P.ptg_opensimplex, dict())]:
            dL = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, seed=0, lacunarity=1.9, **kw)
            general[name + "_f32"] = time_fn(lambda o, fn=fn, dL=dL: fn(ctx, dL, o, stream), reps=3)
        line["lacunarity_1.9"] = general
        # ridged noise (the paper's ridged mountains), same size and octave count: the fused ridged
        # kernel (tiles aligned to cells); "per_sample" times the per-sample generator on the same
        # field one sample off the cell grid (offset 1), where the fused kernel does not apply
        ridged = {}
        for name, fn, kw in [("zero_gradient", P.ptg_field, dict(smoothness=P.PTG_ZERO_GRADIENT)),
                             ("c1", P.ptg_field, dict(smoothness=P.PTG_C1)),
                             ("perlin_s5", P.ptg_perlin, dict())]:
            kw = dict(kw)
            kw["variant"] = kw.get("variant", 0) | P.PTG_RIDGED
            dR = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, seed=0, **kw)
            ridged[name + "_f32"] = time_fn(lambda o, fn=fn, dR=dR: fn(ctx, dR, o, stream), reps=3)
            if name == "c1":
                dU = P.make_desc(dims=2, size=SIZE, spc=SPC, octaves=OCTAVES, seed=0, offset=(1, 0, 0), **kw)
                ridged["c1_f32_per_sample"] = time_fn(lambda o, fn=fn, dU=dU: fn(ctx, dU, o, stream), reps=3)
        line["ridged"] = ridged
        if rank == 0:
            line["volume3d_512_n8"] = bench_3d(P, R, ctx, stream, torch)
            line["field_256_n6"] = bench_small_field(P, ctx, stream, torch)
            line["octave_sweep"] = bench_octave_sweep(P, ctx, stream, torch)
            line["batched"] = bench_batched(P, ctx, stream, torch)
            line["serving"] = bench_serving(P, torch, duration_s=args.serve_seconds)
            line["quality"] = bench_quality(P, ctx, stream, torch)

        # end to end through the C ABI into pinned host memory
        host = torch.empty((SIZE[1], SIZE[0]), dtype=torch.float32).pin_memory()
        P.ptg_generate_host(ctx, descs[0], P.METHOD_FIELD, host)
        n_e2e = max(3, min(args.steps, 20))
        barrier()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            P.ptg_generate_host(ctx, descs[k % 4], P.METHOD_FIELD, host)
        dt = aggregate_max(time.perf_counter() - t0, world)
        line["e2e"] = {"value": world * n_samples * n_e2e / dt / 1e9, "unit": UNIT,
                       "h2d_bytes_per_step": P.ctypes.sizeof(P.ptg_field_desc),
                       "d2h_bytes_per_step": n_samples * 4, "steps": n_e2e,
                       "note": "descriptor in, whole FP32 field out to pinned host memory; banded D2H overlapped "
                               "with generation"}
        if rank == 0 and world == 1:
            rate, n, dtc, threads = oracle_sample_rate(args.cpu_rows)
            line["cpu_baseline"] = {"value": rate / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                                    "sample": "%d full rows (%d samples) of the 8192^2 field, %.1f s on %d "
                                              "threads (%.0f core-seconds)" % (args.cpu_rows, n, dtc, threads,
                                                                               dtc * threads)}
            rate1, n1, dt1, _ = oracle_sample_rate(max(1, args.cpu_rows // 16), threads=1)
            line["cpu_baseline"]["single_core"] = {"value": rate1 / 1e9, "unit": UNIT,
                                                   "sample": "%d samples, %.1f s" % (n1, dt1)}
            line["cpu_baseline"]["field_256_n6"] = oracle_small_fields()
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
