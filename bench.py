#!/usr/bin/env python
"""Benchmark of the funnel-transform hot path on GB300.

Workload: 64 synthetic 1024 x 1024 FP32 images per GPU (1-20 ridge/step lines,
occluders, noise), map 1024 x 1024 (n_slope = W, n_intercept = H), top-32
peaks per image.  One step = detection over the resident batch: Sec. 3.1
steps 1-4 (step 4 also writes the maximum of |P| per tile) and the peak
detection of Sec. 4.4, which reads only the tiles that can hold a top-32 peak.
The timed steps go through ft_detect_batches, PIPE_RUN steps per run (step 1
of one step runs beside the peak pass of the step before); the first step of
every run is a separate one-batch call whose launches are bracketed by CUDA
events (per-kernel durations).  The same step through one ft_detect call each
is timed too ("per_call").  Metric: megapixels (input pixels) per second, whole
job.  Inputs (268 MB) and maps (268 MB) exceed the 129 MB L2.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own 64 images (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the max over ranks is reported by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BATCH = 64
SIDE = 1024
TOP_K = 32
PROF_EVERY = 10     # per-launch CUDA events on every 10th step of a timed region (extra legs)
PIPE_RUN = 50       # main step: steps per ft_detect_batches run; the first of each run is instrumented
METRIC = "megapixels/s funnel fwd(+bwd) at 1024² FP32 vs plain form; % of HBM roofline"
UNIT = "Mpx/s"
WORKLOAD = "64 x 1024x1024 FP32 synthetic line images, map 1024x1024, top-32 peaks per image"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-varlen", action="store_true", help="skip the mixed-size batch measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the 8 x 4096^2 split-precision leg")
    ap.add_argument("--precision-only", action="store_true",
                    help="run only the 4096^2 precision leg on --images images (8 = its workload; fewer for ncu)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the main step (no e2e, forward+backward or mixed-size legs), for ncu captures")
    ap.add_argument("--images", type=int, default=64,
                    help="images per GPU (64 = the benchmark workload; smaller only for ncu captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_info():
    from paper_1904_09409_gb300 import replicas
    return replicas.env_world()


def make_batch(rank: int, world: int = 1, with_lines: bool = False):
    """This rank's images: replicas.shard gives every rank its own BATCH images."""
    from paper_1904_09409_gb300 import replicas, synth
    idx = replicas.shard(rank, world, BATCH)
    if not with_lines:
        return synth.batch_1024(len(idx), start=idx.start, side=SIDE)
    imgs = np.empty((len(idx), SIDE, SIDE), dtype=np.float32)
    lines = []
    for j, i in enumerate(idx):
        si = synth.mixed_image(synth.WL_BATCH_1024, i, SIDE, SIDE)
        imgs[j] = si.img
        lines.append(si.lines)
    return imgs, lines


def line_cells(lines, H, W, n_slope, n_intercept):
    """Map cells (t, s) of drawn lines (corner coordinates row = k col + b_c):
    centred intercept b = b_c + k W/2 - H'/2 + (H'-H)/2, then eqs. (22)-(23)."""
    top = (n_intercept - H) // 2
    out = []
    for ln in lines:
        b = ln.b_c + ln.k * W / 2.0 - n_intercept / 2.0 + top
        out.append(((b + n_intercept / 2.0) % n_intercept, (ln.k * n_slope / 2.0 + n_slope / 2.0) % n_slope))
    return out


def blob_targets(lines_list, side):
    from paper_1904_09409_gb300 import synth
    return np.stack([synth.blob_target(side, side, line_cells(ls, side, side, side, side)) for ls in lines_list])


def time_fwd_bwd(f, plan, x, target, steps, stream, dev):
    """Forward, loss mean((|P|/(W/2) - T)^2) with its gradient, adjoint: CUDA-event
    time per step (ms) and per-kernel timing of the timed region."""
    import torch
    P = torch.empty((x.shape[0], plan.Hp, plan.S), dtype=torch.float32, device=dev)
    loss = torch.empty(x.shape[0], dtype=torch.float32, device=dev)
    gx = torch.empty_like(x)

    def step():
        f.ft_forward(plan, x, P, stream=stream)
        f.ft_abs_mse_backward(plan, P, target, 2.0 / plan.W, loss=loss, grad_img=gx, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    f.ft_profile_read(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        f.ft_profile_enable(plan, i % PROF_EVERY == 0)
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    prof = f.ft_profile_read(plan)
    f.ft_profile_enable(plan, False)
    return e0.elapsed_time(e1) / steps, {k: v[0] / v[1] * 1e3 for k, v in prof.items()}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_bytes(name: str, H: int, W: int, S: int, Hp: int, K: int) -> float:
    """Algorithmic DRAM bytes per image of each kernel (compulsory reads and
    writes of its own inputs and outputs).  The peak pass from tile maxima reads
    the tile maxima and the cells of the tiles it tests, at least the 32 it
    starts with (more when its bound needs them)."""
    L = Hp // 2 + 1
    ntiles = ((Hp + 31) // 32) * ((S + 63) // 64)
    kt = min(K, 512)
    # tiles of step 4's maxima at H' = 1024: 16 rows x 16 columns; the first 32
    # (one per warp) are read with their one-cell halo (18 x 18 cells)
    c2r_tiles = (Hp // 16) * ((S + 15) // 16)
    R = min(c2r_tiles, 32)
    return {
        "k_col_r2c": 4.0 * H * W + 8.0 * L * W,          # image in, half spectrum out
        "k_nvmt_rows": 8.0 * L * W + 8.0 * L * S,        # spectrum rows in, G rows out
        "k_col_c2r": 8.0 * L * S + 4.0 * Hp * S + 4.0 * c2r_tiles,   # G in, map and tile maxima out
        "k_peak_sparse": 4.0 * c2r_tiles + 4.0 * R * 18 * 18 + 20.0 * K + 4.0,
        "k_tile_max": 4.0 * Hp * S + 4.0 * ((Hp + 15) // 16) * ((S + 15) // 16),
        "k_peak_tiles": 4.0 * Hp * S + 8.0 * ntiles * kt,  # map in, tile keys out
        "k_peak_select": 8.0 * ntiles * kt + 20.0 * K + 4.0,
    }.get(name, 0.0)


def sources_digest(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, batch: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to `batch` images, or None when absent or when the kernel's sources have
    changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        k = json.load(f).get("kernels", {}).get(kernel)
    if not k or sources_digest(k["sources"]) != k["digest"]:
        return None
    return float(k["dram_bytes_per_image"]) * batch


class ClockSampler:
    """nvidia-smi clocks / throttle reasons of one GPU, sampled every 200 ms."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- oracle (CPU) legs
def _oracle_one(img):
    import oracle
    t = time.perf_counter()
    P = oracle.funnel_ref(img, SIDE, SIDE)
    oracle.peaks_ref(np.abs(P), TOP_K)
    return time.perf_counter() - t


def oracle_pool(cores: int):
    return mp.get_context("spawn").Pool(cores)


def time_oracle_sample(pool, imgs):
    """Wall time of the oracle (map + peak list) on the given images, one image
    per task, run by the pool in parallel."""
    t = time.perf_counter()
    per = pool.map(_oracle_one, list(imgs), chunksize=1)
    return time.perf_counter() - t, per


def _varlen_img(args):
    from paper_1904_09409_gb300 import synth
    idx, h, w = args
    return synth.varlen_image(idx, h, w).img


def _large_img(i):
    from paper_1904_09409_gb300 import synth
    return synth.large_4096(1, start=i)[0].img


def large_images(pool, count=8):
    return pool.map(_large_img, list(range(count)), chunksize=1)


# Relative L2 error of the 4096^2 precision workload's map (image 0) against the
# FP64 oracle, per variant, as tests/test_gpu_tensorcore.py measures it on GB300
# (the bench runs no oracle outside its CPU-baseline leg); the split-precision
# target is 1e-5, which BF16 hi + lo misses once steps 1 and 4 run on the tensor
# cores as well (six GEMMs in sequence).
PRECISION_ORACLE_ERR = {"fp32": 9.7e-7, "bf16x3": 3.0e-5, "fp16x3": 2.2e-6, "bf16x6": 3.5e-6}


def time_precision(f, imgs, steps, stream, dev):
    """8 x 4096^2 (100 lines each): forward + top-100 peaks per step-3 precision.
    The split variants are compared with the FP32 path's maps and peaks on the
    device (their error against the FP64 oracle is what the GPU tests check)."""
    import torch
    x = torch.from_numpy(np.stack(imgs)).to(dev)
    B = x.shape[0]
    K = 100
    maps, peaks, out = {}, {}, {}
    for prec in ("fp32", "bf16x3", "fp16x3", "bf16x6"):
        plan = f.Plan(4096, 4096, 4096, 4096, "linear")
        f.ft_plan_set_precision(plan, prec)
        m = torch.empty((B, 4096, 4096), dtype=torch.float32, device=dev)
        pk = torch.empty(B * K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        cn = torch.empty(B, dtype=torch.int32, device=dev)

        def step():
            f.ft_detect(plan, x, m, K, out=pk, count=cn, stream=stream)

        for _ in range(3):
            step()
        torch.cuda.synchronize(dev)
        f.ft_profile_read(plan)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for i in range(steps):
            f.ft_profile_enable(plan, i % PROF_EVERY == 0)
            step()
        q1.record(stream)
        torch.cuda.synchronize(dev)
        ms = q0.elapsed_time(q1) / steps
        prof = f.ft_profile_read(plan)
        errs = f.ft_plan_tc_errors(plan)
        res = f.peaks_to_numpy(pk, cn, K)
        peaks[prec] = [{(int(p["t"]), int(p["s"])) for p in r} for r in res]
        out[prec] = {"value": B * 4096 * 4096 / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                     "steps": steps, "tc_error_flags": errs,
                     "kernels_us_per_launch": {k: v[0] / v[1] * 1e3 for k, v in prof.items()},
                     "rel_l2_vs_fp64_oracle_in_gpu_tests": PRECISION_ORACLE_ERR[prec],
                     "meets_1e-5_target": PRECISION_ORACLE_ERR[prec] <= 1e-5}
        if prec == "fp32":
            maps[prec] = m
        else:
            ref = maps["fp32"]
            num = sum(float(torch.linalg.vector_norm((m[i].double() - ref[i].double()))) ** 2 for i in range(B))
            den = sum(float(torch.linalg.vector_norm(ref[i].double())) ** 2 for i in range(B))
            out[prec]["rel_l2_vs_fp32_path"] = (num / den) ** 0.5
            out[prec]["top100_agreement_vs_fp32_path"] = sum(
                len(a & b) for a, b in zip(peaks[prec], peaks["fp32"])) / (B * K)
            del m
        plan.close()
    del maps, x
    torch.cuda.empty_cache()
    return {"workload": "8 x 4096^2 images, 100 lines each (mixed edge types, noise 0.2), n_slope = "
                        "n_intercept = 4096, linear NVMT: ft_detect with top-100 peaks; the three length-4096 "
                        "transforms (steps 1, 3, 4) in FP32 (FFT) or as split-precision four-step DFTs on "
                        "the tensor cores",
            "variants": out}


def varlen_images(pool, shapes):
    return pool.map(_varlen_img, [(i, h, w) for i, (h, w) in enumerate(shapes)], chunksize=4)


def time_varlen(f, imgs, shapes, steps, dev):
    """512 mixed-size images (H, W from {128 ... 2048}), forward + top-32 peaks:
    the grouped kernels (one launch per stage over every image, work queues)
    after autotuning, in one captured graph; returns the JSON record with the
    tuner's table and per-size throughput (each shape alone, as a batch of its
    own with the chosen configuration)."""
    import torch
    cache = os.path.join(ROOT, "paper_1904_09409_gb300", "tune_cache.json")
    b = f.Batch(shapes, tune_cache=cache)
    x = torch.from_numpy(b.pack(imgs)).to(dev)
    m = torch.empty(b.map_total, dtype=torch.float32, device=dev)
    out = torch.empty(b.n * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cnt = torch.empty(b.n, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)

    def timed(batch, xb, mb, ob, cb, n):
        with torch.cuda.stream(s):
            for _ in range(3):
                batch.run(xb, mb, TOP_K, out=ob, count=cb, stream=s, graph=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(n):
                batch.run(xb, mb, TOP_K, out=ob, count=cb, stream=s, graph=True)
            e1.record(s)
            s.synchronize()
        return e0.elapsed_time(e1) / n

    with torch.cuda.stream(s):
        t0 = time.perf_counter()
        b.run(x, m, TOP_K, out=out, count=cnt, stream=s, tune=True)
        s.synchronize()
        tune_s = time.perf_counter() - t0
    ms = timed(b, x, m, out, cnt, steps)
    cfg = b.config()
    chosen = (cfg["r2c_threads"], cfg["rows_threads"], cfg["c2r_threads"])
    tune_table = {f"{a}/{r}/{c}": round(v, 4) for (a, r, c), v in b.tune_ms().items()}
    px = sum(h * w for h, w in shapes)
    # per size: the workload's images of one shape, repeated to at least 16
    # megapixels, as a batch of their own with the same configuration (a launch
    # of a shape's few images alone would measure launch latency, not the kernels)
    per = {}
    groups = b.groups()
    for g in groups:
        h, w, start, count = g["H"], g["W"], g["start"], g["count"]
        idx = [int(i) for i in b.order[start:start + count]]
        reps = max(count, -(-16 * 2 ** 20 // (h * w)))
        sel = [imgs[idx[r % count]] for r in range(reps)]
        with f.Batch([(h, w)] * reps) as bg:
            bg.set_config(*chosen)
            xg = torch.from_numpy(bg.pack(sel)).to(dev)
            mg = torch.empty(bg.map_total, dtype=torch.float32, device=dev)
            og = torch.empty(reps * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            cg = torch.empty(reps, dtype=torch.int32, device=dev)
            tg = timed(bg, xg, mg, og, cg, 10)
        per[f"{h}x{w}"] = round(reps * h * w / (tg / 1e3) / 1e6, 1)
    b.close()
    return {"images_per_s": len(shapes) / (ms / 1e3), "value": px / (ms / 1e3) / 1e6, "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "images": len(shapes), "megapixels": px / 1e6,
            "shape_groups": len(groups), "launches_per_step": cfg["launches"],
            "grouped_images": cfg["grouped_images"], "tune_s": tune_s,
            "threads_chosen": {"r2c": chosen[0], "rows": chosen[1], "c2r": chosen[2]},
            "default_threads": "512/128/256", "tune_ms": tune_table,
            "per_size_mpx_s": per,
            "workload": "512 images, H and W i.i.d. from {128,192,256,384,512,768,1024,1536,2048}, content as "
                        "the 1024^2 batch, maps H x W, top-32; forward + peaks of every image in the grouped "
                        "kernels (one persistent launch per stage, device work queues), one CUDA graph launch, "
                        "threads per block chosen by the autotuner (tune_ms: r2c/rows/c2r -> ms); per-size "
                        "figures are each shape's images, repeated to >= 16 Mpx, as a batch of their own"}


def fourier_rows_flops(H, W, S, Hp):
    """FP32 FLOPs of steps 2-3 with the band-limited interpolator per image: per
    kept row (l >= 1) complex FFTs of lengths W, M (twice) and S at 5 N log2 N,
    the pre-chirp and its weights on W + 1 entries (8 each), the chirp spectrum
    product on M (6) and the post-chirp with its weights on S (8)."""
    import math
    M = W + S
    while True:                                    # the smallest 2^a 3^b >= W + S
        m = M
        for p in (2, 3):
            while m % p == 0:
                m //= p
        if m == 1:
            break
        M += 1
    per_row = (5 * W * math.log2(W) + 2 * 5 * M * math.log2(M) + 5 * S * math.log2(S)
               + 8 * (W + 1) + 6 * M + 8 * S)
    return per_row * (Hp // 2)


def fma_peak(f, stream, dev):
    """Measured FP32 FMA throughput of this GPU (ft_fma_probe, 8 blocks of 256
    threads per multiprocessor, best of 5) next to the nominal figure
    SMs x 128 lanes x 2 x max SM clock."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    blocks, iters = sms * 8, 8192
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    f.ft_fma_probe(out, blocks, iters, stream=stream)
    best = None
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        flops = f.ft_fma_probe(out, blocks, iters, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        t = flops / (a.elapsed_time(b) / 1e3) / 1e12
        best = t if best is None or t > best else best
    try:
        max_mhz = float(subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                                        "-i", str(dev.index or 0)], capture_output=True, text=True,
                                       timeout=20).stdout.split()[0])
    except Exception:
        max_mhz = 2070.0
    return {"measured_tflops": best, "nominal_tflops": sms * 128 * 2 * max_mhz * 1e6 / 1e12, "sms": sms,
            "sm_max_mhz": max_mhz, "probe": f"{blocks} blocks x 256 threads x {iters} rounds x 8 FMA chains"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(imgs):
    n_images = len(imgs)
    cores = min(host_cores(), n_images)
    with oracle_pool(cores) as pool:
        time_oracle_sample(pool, imgs[:cores])                      # warm-up (imports)
        wall, per = time_oracle_sample(pool, imgs)
    px = n_images * SIDE * SIDE
    single = statistics.median(per)                                 # one image on one core
    return {"value": px / wall / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_s_per_image": single, "single_core_value": SIDE * SIDE / single / 1e6,
            "sample": f"{n_images} of the 64 images (FP64 NumPy map + Sec. 4.4 peak list), "
                      f"one image per task, {cores} processes; {sum(per):.1f} CPU-s"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    cores = host_cores()
    imgs = make_batch(0)
    with oracle_pool(cores) as pool:
        _, per0 = time_oracle_sample(pool, imgs[:cores])            # calibration (also warm-up)
        t_img = statistics.median(per0)
        budget = 150.0                                             # seconds for the whole run
        n = int(budget * cores / max(t_img, 1e-3) / (args.steps + args.warmup))
        n = max(1, min(BATCH, n))
        for _ in range(args.warmup):
            time_oracle_sample(pool, imgs[:n])
        walls = [time_oracle_sample(pool, imgs[:n])[0] for _ in range(args.steps)]
    total = sum(walls)
    value = args.steps * n * SIDE * SIDE / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": BATCH, "images_per_step_sampled": n,
                   "parallelism": f"{cores} host processes"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} of the 64 images per step, one image per process"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
def run_ours(args):
    global BATCH
    BATCH = args.images
    import torch
    from paper_1904_09409_gb300 import funnel as f

    from paper_1904_09409_gb300 import replicas
    ws, rank, local = dist_info()
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    if ws > 1:
        replicas.init("nccl", dev)

    # CPU baseline first (spawned pool, before any kernel of ours runs)
    from paper_1904_09409_gb300 import synth
    imgs, lines = make_batch(rank, ws, with_lines=True)
    cpu = None
    vl_shapes = synth.varlen_shapes(512)
    vl_imgs = None
    big_imgs = None
    if not args.no_extras:
        with oracle_pool(min(host_cores(), 32)) as pool:
            if not args.no_varlen:
                vl_imgs = varlen_images(pool, vl_shapes)
            if not args.no_precision:
                big_imgs = large_images(pool, 8)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(imgs)

    plan = f.Plan(SIDE, SIDE, SIDE, SIDE)
    x = torch.from_numpy(imgs).to(dev)
    m = torch.empty((BATCH, SIDE, SIDE), dtype=torch.float32, device=dev)
    pk = torch.empty(BATCH * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cnt = torch.empty(BATCH, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        f.ft_detect(plan, x, m, TOP_K, out=pk, count=cnt, stream=stream)

    # PIPE_RUN pipelined steps per ft_detect_batches call, over the same resident images
    xs = [x] * PIPE_RUN
    pk_n = torch.empty(PIPE_RUN * BATCH * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cnt_n = torch.empty(PIPE_RUN * BATCH, dtype=torch.int32, device=dev)

    def steps(n):
        f.ft_detect_batches(plan, xs[:n], m, TOP_K, out=pk_n, count=cnt_n, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    steps(PIPE_RUN)
    torch.cuda.synchronize(dev)
    # the same step, one ft_detect call each (uninstrumented)
    n_pc = min(args.steps, 300)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(n_pc):
        step()
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    per_call_ms = pe0.elapsed_time(pe1) / n_pc

    uuid = str(getattr(torch.cuda.get_device_properties(dev), "uuid", "") or "")
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.5)
    f.ft_profile_read(plan)
    replicas.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # every PIPE_RUN-th step's launches are bracketed by CUDA events (per-kernel
    # durations inside the timed region); the others run uninstrumented and pipelined
    for c0 in range(0, args.steps, PIPE_RUN):
        n = min(PIPE_RUN, args.steps - c0)
        f.ft_profile_enable(plan, True)
        steps(1)
        f.ft_profile_enable(plan, False)
        if n > 1:
            steps(n - 1)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    replicas.barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    prof = f.ft_profile_read(plan)
    f.ft_profile_enable(plan, False)

    ms = replicas.max_over_ranks(ms, dev)

    extra = {} if args.no_extras else run_extras(f, args, plan, imgs, lines, x, stream, dev, rank, ws,
                                                  vl_imgs, vl_shapes, big_imgs)

    px_step = ws * BATCH * SIDE * SIDE
    value = args.steps * px_step / (ms / 1e3) / 1e6

    # roofline of the dominant kernel
    kernels = {}
    total_kernel_ms = sum(v[0] for v in prof.values()) or 1.0
    prof_steps = (args.steps + PIPE_RUN - 1) // PIPE_RUN
    for name, (kms, n) in prof.items():
        per = kms / n
        imgs_per_launch = BATCH * prof_steps / n          # the plan may split a batch over streams
        b = kernel_bytes(name, SIDE, SIDE, SIDE, SIDE, TOP_K) * imgs_per_launch
        kernels[name] = {"ms_per_launch": per, "launches": n, "images_per_launch": imgs_per_launch,
                         "share": kms / total_kernel_ms,
                         "algorithmic_bytes_per_launch": b, "achieved_gbs": b / (per / 1e3) / 1e9}
    hbm, src = measured_peaks()
    dom = max(kernels, key=lambda k: kernels[k]["share"]) if kernels else None
    roof = None
    if dom:
        k = kernels[dom]
        roof = {"kernel": dom, "bound": "hbm", "achieved": k["achieved_gbs"], "peak": hbm,
                "unit": "GB/s", "frac": k["achieved_gbs"] / hbm, "peak_source": src,
                "traffic": ncu_traffic(dom, k["images_per_launch"]),
                "algorithmic_bytes_per_launch": k["algorithmic_bytes_per_launch"]}
    # the whole step against the same peak: compulsory bytes (image in, map out: 8 B/px),
    # algorithmic bytes (every kernel's inputs and outputs) and the ncu DRAM bytes
    step_s = ms / args.steps / 1e3
    alg = sum(kernel_bytes(n, SIDE, SIDE, SIDE, SIDE, TOP_K) for n in prof) * BATCH
    traf = [ncu_traffic(n, BATCH) for n in prof]
    step_roof = {"compulsory_gbs": 8.0 * BATCH * SIDE * SIDE / step_s / 1e9,
                 "algorithmic_gbs": alg / step_s / 1e9,
                 "dram_gbs": (sum(traf) / step_s / 1e9) if all(t is not None for t in traf) else None,
                 "peak": hbm, "unit": "GB/s"}
    step_roof["compulsory_frac"] = step_roof["compulsory_gbs"] / hbm
    step_roof["algorithmic_frac"] = step_roof["algorithmic_gbs"] / hbm
    step_roof["dram_frac"] = step_roof["dram_gbs"] / hbm if step_roof["dram_gbs"] else None
    # our kernels launched in the timed region (the profiled steps give the count per step)
    launches = sum(n for _, n in prof.values()) * args.steps // prof_steps
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": ws * BATCH, "images_per_gpu": BATCH,
                       "H": SIDE, "W": SIDE, "n_slope": SIDE, "n_intercept": SIDE, "interp": "linear",
                       "top_k": TOP_K, "l2": "inputs larger than L2 (268 MB images + 268 MB maps per GPU)",
                       "parallelism": f"replicas x{ws}, no collective on the data path"},
            "roofline": roof,
            "kernel_timing": f"CUDA events around every launch of every {PIPE_RUN}th timed step",
            "pipelining": f"ft_detect_batches, {PIPE_RUN - 1} pipelined steps per call after one instrumented "
                          "step (step 1 of a step beside the peak pass of the one before)",
            "per_call": {"call": "ft_detect", "steps": n_pc, "ms_per_step": per_call_ms,
                         "value": px_step / (per_call_ms / 1e3) / 1e6, "unit": UNIT},
            "step_roofline": step_roof,
            "kernels": kernels,
            "cpu_baseline": cpu,
            **extra,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    replicas.finish()
    return 0


def run_extras(f, args, plan, imgs, lines, x, stream, dev, rank, ws, vl_imgs, vl_shapes, big_imgs):
    """e2e through ft_detect_host, forward+backward legs, the mixed-size batch and
    the host-to-device copy rate; returns the extra JSON keys."""
    import torch
    from paper_1904_09409_gb300 import replicas, synth
    px_step = ws * BATCH * SIDE * SIDE
    # end to end through the public host-buffer call: H2D of the step's images
    # from pinned memory, forward + peaks, D2H of the peaks and counts
    h_img = torch.from_numpy(imgs).pin_memory()
    h_pk = torch.empty(BATCH * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    h_cnt = torch.empty(BATCH, dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 30))
    for _ in range(2):
        f.ft_detect_host(plan, h_img, TOP_K, out_host=h_pk, count_host=h_cnt, stream=stream)
    replicas.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        f.ft_detect_host(plan, h_img, TOP_K, out_host=h_pk, count_host=h_cnt, stream=stream)
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, dev)

    # forward + loss + adjoint on the same resident batch, and on 32 x 512^2
    tgt = torch.from_numpy(blob_targets(lines, SIDE)).to(dev)
    fb_steps = max(3, min(args.steps, 100))
    fb_ms, fb_kernels = time_fwd_bwd(f, plan, x, tgt, fb_steps, stream, dev)
    fb_ms = replicas.max_over_ranks(fb_ms, dev)
    del tgt
    g_imgs = synth.grad_batch_512(32, start=rank * 32)
    plan512 = f.Plan(512, 512, 512, 512)
    x512 = torch.from_numpy(np.stack([g.img for g in g_imgs])).to(dev)
    t512 = torch.from_numpy(np.stack([synth.blob_target(512, 512, line_cells(g.lines, 512, 512, 512, 512))
                                      for g in g_imgs])).to(dev)
    fb512_ms, _ = time_fwd_bwd(f, plan512, x512, t512, fb_steps, stream, dev)
    fb512_ms = replicas.max_over_ranks(fb512_ms, dev)
    plan512.close()

    varlen = None
    if vl_imgs is not None:
        varlen = time_varlen(f, vl_imgs, vl_shapes, max(3, min(args.steps, 50)), dev)

    # the paper's band-limited (chirp-z) interpolator on the same batch
    fplan = f.Plan(SIDE, SIDE, SIDE, SIDE, "fourier")
    mf = torch.empty((BATCH, SIDE, SIDE), dtype=torch.float32, device=dev)
    pk = torch.empty(BATCH * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cn = torch.empty(BATCH, dtype=torch.int32, device=dev)
    for _ in range(3):
        f.ft_detect(fplan, x, mf, TOP_K, out=pk, count=cn, stream=stream)
    fo_steps = max(3, min(args.steps, 50))
    f.ft_profile_read(fplan)
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for i in range(fo_steps):
        f.ft_profile_enable(fplan, i % PROF_EVERY == 0)
        f.ft_detect(fplan, x, mf, TOP_K, out=pk, count=cn, stream=stream)
    q1.record(stream)
    torch.cuda.synchronize(dev)
    fo_ms = replicas.max_over_ranks(q0.elapsed_time(q1) / fo_steps, dev)
    fo_prof = {k: 1e3 * v[0] / v[1] for k, v in f.ft_profile_read(fplan).items()}
    fplan.close()
    del mf
    fma = fma_peak(f, stream, dev)
    fo_flops = fourier_rows_flops(SIDE, SIDE, SIDE, SIDE) * BATCH
    fo_rows_us = fo_prof.get("k_nvmt_rows")
    fo_alu = None
    if fo_rows_us:
        t = fo_flops / (fo_rows_us / 1e6) / 1e12
        fo_alu = {"kernel": "k_nvmt_rows (chirp-z)", "bound": "alu", "flops_per_launch": fo_flops,
                  "achieved": t, "peak": fma["measured_tflops"], "unit": "TFLOP/s",
                  "frac": t / fma["measured_tflops"], "peak_source": "measured (FMA probe in this run)"}

    # Sec. 4.5 line verification of the step's top-32 peaks (band of 5 pixels)
    pk_b = torch.empty(BATCH * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    cn_b = torch.empty(BATCH, dtype=torch.int32, device=dev)
    mv = torch.empty((BATCH, SIDE, SIDE), dtype=torch.float32, device=dev)
    f.ft_detect(plan, x, mv, TOP_K, out=pk_b, count=cn_b, stream=stream)
    for _ in range(3):
        f.ft_verify(plan, x, pk_b, cn_b, TOP_K, 2, 0.05, 64, stream=stream)
    v_steps = max(3, min(args.steps, 50))
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record(stream)
    for _ in range(v_steps):
        _, _, verdict = f.ft_verify(plan, x, pk_b, cn_b, TOP_K, 2, 0.05, 64, stream=stream)
    v1.record(stream)
    torch.cuda.synchronize(dev)
    v_ms = v0.elapsed_time(v1) / v_steps
    verified = int((verdict == 1).sum().item())
    del mv
    verify = {"ms_per_call": v_ms, "peaks_per_s": BATCH * TOP_K / (v_ms / 1e3), "steps": v_steps,
              "verified": verified, "peaks": int(cn_b.sum().item()),
              "workload": f"ft_verify of the top-{TOP_K} peaks of the same {BATCH} x 1024^2 maps: band of 5 pixels, "
                          "contrast >= 0.05, centre line >= 64 samples"}

    precision = None
    if big_imgs is not None:
        precision = time_precision(f, big_imgs, max(3, min(args.steps, 20)), stream, dev)

    # host -> device copy rate of the pinned image buffer (context for e2e)
    hd = torch.empty_like(x)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hd.copy_(h_img, non_blocking=True)
    c0.record(stream)
    for _ in range(5):
        hd.copy_(h_img, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize(dev)
    h2d_gbs = 5 * h_img.numel() * 4 / (c0.elapsed_time(c1) / 1e3) / 1e9
    return {
        "e2e": {"value": e2e_steps * px_step / e2e_s / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": ws * BATCH * SIDE * SIDE * 4,
                "d2h_bytes_per_step": ws * (BATCH * TOP_K * f.PEAK_DTYPE.itemsize + BATCH * 4),
                "call": "ft_detect_host", "steps": e2e_steps, "h2d_copy_gbs": h2d_gbs},
        "varlen": varlen,
        "verify": verify,
        "precision_4096": precision,
        "fp32_fma_peak": fma,
        "fourier_interp": {"value": px_step / (fo_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": fo_ms,
                           "steps": fo_steps, "kernels_us": fo_prof, "roofline": fo_alu,
                           "workload": "the same 64 x 1024^2 step (ft_detect, top-32 peaks) with the band-limited "
                                       "(chirp-z, Sec. IV) interpolator instead of the linear one"},
        "fwd_bwd": {"value": px_step / (fb_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": fb_ms,
                    "steps": fb_steps, "kernels_us": fb_kernels,
                    "workload": "the same 64 x 1024^2 batch: ft_forward + ft_abs_mse_backward (loss "
                                "mean((|P|/(W/2) - T)^2), T Gaussian blobs of 2 cells at the drawn "
                                "lines, and its gradient with respect to the images through the exact "
                                "adjoint; the map gradient is formed inside the first adjoint kernel)"},
        "fwd_bwd_512": {"value": ws * 32 * 512 * 512 / (fb512_ms / 1e3) / 1e6, "unit": UNIT,
                        "ms_per_step": fb512_ms, "steps": fb_steps,
                        "workload": "32 x 512^2 gradient workload, same step"},
    }


def run_precision_only(args):
    import torch
    from paper_1904_09409_gb300 import funnel as f
    n = args.images if args.images != 64 else 8
    with oracle_pool(min(host_cores(), 32)) as pool:
        imgs = large_images(pool, n)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    res = time_precision(f, imgs, max(1, args.steps), torch.cuda.current_stream(dev), dev)
    print(json.dumps({"precision_4096": res}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.precision_only:
        return run_precision_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
