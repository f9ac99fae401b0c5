#!/usr/bin/env python3
"""Benchmark of the GB300 particle-filter registration path.

One step = one whole registration of the image-based workload -- 224x208x176
uint8 speckle volumes, N = 2048 particles, 50 iterations, +-30 deg / +-25
voxel limits, trilinear NCC^2 -- followed by the warp of the 20-frame source
sequence with the estimate (context creation, all iterations, estimate and
warp inside the step).  Inputs are seeded synthetic stand-ins (pfsynth).

Metric: particle-voxel evaluations per second, counted densely
(N x iterations x target voxels per registration), and ms per registration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank registers its own pair (independent
problems, weak scaling); rank 0 prints one JSON line.  ``--impl reference``
times the CPU oracle (the only reference this method has) on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pfsynth  # noqa: E402

WORKLOADS = {
    "image224": dict(pfsynth.IMAGE224, kind="image_ncc", dims=(224, 208, 176)),
    "mask64": dict(pfsynth.MASK64, kind="mask_dice", dims=(64, 64, 64), n_frames=0, default_steps=1500),
    "batch64": dict(name="batch64_mixed_96to256_n512to8192_k20to60", kind="batch", n_regs=64),
    "batch64_small": dict(name="batch64_mixed_40to80_n128to1024_k8to16", kind="batch", n_regs=64, small=True),
    "combined256": dict(pfsynth.COMBINED256, kind="combined", dims=(256, 256, 256)),
    "conv32": dict(name="conv3d_b32_32x32x32x32_to_16x16x16x32_bf16", kind="conv"),
    "proposal": dict(name="proposal_speckle224x208x176_learned_n512_vs_plain_n2048_k50", kind="proposal",
                     n_particles=512, plain_particles=2048, n_iters=50, rot_limit_deg=30.0, trans_limit=25.0,
                     seed=0, train_steps=3125, train_batch=32, lr=1e-3, std_inflate=1.5),
}
METRIC = "particle-voxel evals/s (dense N*iters*target voxels per registration) and ms per registration"
UNIT = "particle-voxel evals/s"

# FP32 operations the arithmetic definition fixes per visited voxel of the
# trilinear measurement: 3 mul + 3 add (coordinates), 3 floor, 3 subtract
# (fractions), 7 lerps x (1 subtract + 1 fused multiply-add), 1 rounding to
# 15 fractional bits; each counts one lane operation against the FP32 lane
# rate (152 SMs x 128 lanes x clock).
OPS_PER_EVAL = 27
# nearest-neighbour mask sample: 3 mul + 3 add (coordinates), 3 add (+0.5),
# 3 floor; the combined score does both on one coordinate.
OPS_PER_EVAL_MODE = {"image_ncc": OPS_PER_EVAL, "mask_dice": 12, "combined": OPS_PER_EVAL + 6}
FP32_LANES_PER_SM = 128

# Counters of one measurement launch from an ncu capture of each workload
# (summarised under profiles/), keyed by workload and tied to the hash of the
# kernel source they were taken on: DRAM bytes (read + write) per launch and
# L2 -> L1 bytes per visited evaluation.  A workload without its own capture,
# or whose kernel changed since, reports null.
NCU_COUNTERS = {
    # profiles/measure_counters_image224_mask64_combined256.md
    "image224": {"measure_code_sha1": "1d26970369b009c4d4885828ca94135a828b8568",
                 "dram_bytes_per_launch": 36136704, "l2_to_l1_bytes_per_eval": 139410378752 / 9388958565.74},
    "mask64": {"measure_code_sha1": "1d26970369b009c4d4885828ca94135a828b8568",
               "dram_bytes_per_launch": 278016, "l2_to_l1_bytes_per_eval": 43771840 / 41168147.2},
    "combined256": {"measure_code_sha1": "42c6fb5ada11cf158665be670855a77ffecc4fe2",
                    "dram_bytes_per_launch": 140074539520, "l2_to_l1_bytes_per_eval": 2002563646368 / 152465706355.25},
}


# the measurement kernel's translation unit (its source and the headers it includes)
MEASURE_SOURCES = [os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", f)
                   for f in ("measure.cu", "kernels.h", "device.cuh")]


def kernel_code_hash(paths):
    """sha1 of CUDA sources with their comments and whitespace removed, so that
    it names the kernel's code (a comment edit leaves it unchanged)."""
    h = hashlib.sha1()
    for path in paths:
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode() + b"\0")
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 3; 1500 for the 64^3 mask workload, whose registration takes "
                         "~2 ms, so that the clock sampler sees the timed region)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="image224")
    ap.add_argument("--batch-regs", type=int, default=64)
    ap.add_argument("--proposal-eval-pairs", type=int, default=200,
                    help="held-out pairs of the learned-proposal comparison (seeds 5000 + 1000 rank + i)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-particles", type=int, default=None,
                    help="oracle sample: particles (default: 64, or the whole cloud of the 64^3 mask workload)")
    ap.add_argument("--cpu-sample-iters", type=int, default=None,
                    help="oracle sample: iterations (default: 2, or all of the 64^3 mask workload's)")
    ap.add_argument("--cpu-all-cores-particles", type=int, default=512)
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the short 64^3 mask and convolution lines the default run attaches")
    args = ap.parse_args()
    if args.steps is None:   # the oracle arm's steps are bounded samples: 3 by default everywhere
        args.steps = WORKLOADS[args.workload].get("default_steps", 3) if args.impl == "ours" else 3
    return args


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    def __init__(self, world):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, v):
        if self.world == 1:
            return v
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v):
        if self.world == 1:
            return v
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def l2_read_peak(pk, torch, dev, stream):
    """L2 -> SM read bandwidth (GB/s) measured with the library's probe: a
    48 MiB buffer (resident in the 129 MB L2) read 20 times with 16-byte loads
    that bypass L1, timed with CUDA events on the launching stream."""
    buf = torch.ones(48 << 20, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    reps = 20
    pk.pf_probe_read(buf, 2, sink, stream=stream)            # warm-up: brings the buffer into L2
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pk.pf_probe_read(buf, reps, sink, stream=stream)
        e1.record(stream)
        e1.synchronize()
        gbs = buf.numel() * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
        best = gbs if best is None else max(best, gbs)
    return best


def load_workload(name, rank):
    w = WORKLOADS[name]
    if w["kind"] == "combined":
        pair = pfsynth.cached(pfsynth.speckle_pair, rank, src_dims=w["dims"], with_masks=True,
                              max_rot_deg=20.0, max_trans=15.0)
        frames = pfsynth.cached(pfsynth.frame_sequence, pair, w["n_frames"])
    elif w["kind"] == "image_ncc":
        pair = pfsynth.cached(pfsynth.speckle_pair, rank, with_masks=True)
        frames = pfsynth.cached(pfsynth.frame_sequence, pair, w["n_frames"]) if w["n_frames"] else None
    else:
        pair = pfsynth.ellipsoid_pair(rank)
        frames = None
    return w, pair, frames


def settled_iteration(dice, target):
    """1-based first iteration from which the estimate's Dice stays >= target
    for the rest of the run, or None when the last one is below it."""
    dice = np.asarray(dice, np.float64)
    if len(dice) == 0 or dice[-1] < target:
        return None
    below = np.nonzero(dice < target)[0]
    return int(below[-1] + 2) if len(below) else 1


def dense_units(w, pair):
    return w["n_particles"] * w["n_iters"] * int(np.prod(pair.tgt.shape))


# --------------------------------------------------------------- CPU oracle

def oracle_sample(w, pair, n_particles, n_iters):
    """Time the oracle on a bounded sample of the workload: the same pair,
    n_particles particles, n_iters iterations.  Returns (seconds, dense units)."""
    import oracle
    oracle.build()
    if w["kind"] == "image_ncc":
        kw = dict(src=pair.src, tgt=pair.tgt)
    elif w["kind"] == "combined":
        kw = dict(src=pair.src, tgt=pair.tgt, src_mask=pair.src_mask, tgt_mask=pair.tgt_mask)
    else:
        kw = dict(src_mask=pair.src, tgt_mask=pair.tgt)
    t0 = time.perf_counter()
    oracle.register(w["kind"], pair.src_dims, pair.src_origin, pair.tgt_dims, pair.tgt_origin, n_particles,
                    n_iters, np.deg2rad(w["rot_limit_deg"]), w["trans_limit"], seed=w["seed"], trace=False, **kw)
    dt = time.perf_counter() - t0
    return dt, n_particles * n_iters * int(np.prod(pair.tgt.shape))


def _measure_chunk(task):
    """Pool worker: the oracle's measurement of a chunk of matrices."""
    kind, src, tgt, smask, tmask, mats, a = task
    import oracle
    if kind in ("image_ncc", "combined"):
        oracle.measure_image(src, tgt, mats, a)
    if kind != "image_ncc":
        oracle.measure_mask(smask, tmask, mats, a)
    return len(mats)


def oracle_measure_all_cores(w, pair, n_particles, cores):
    """The oracle's measurement (the > 99 % part of an iteration) of
    n_particles initial-cloud matrices, split over ``cores`` spawned
    processes.  Returns (seconds, dense units, cores)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    lim = np.array([np.deg2rad(w["rot_limit_deg"])] * 3 + [w["trans_limit"]] * 3, np.float32)
    x = oracle.init_particles(n_particles, w["seed"], lim)
    mats, a = oracle.pose_matrices(x, pair.src_dims, pair.src_origin, pair.tgt_origin)
    if w["kind"] == "mask_dice":
        vols = (None, None, pair.src, pair.tgt)
    else:
        vols = (pair.src, pair.tgt, pair.src_mask, pair.tgt_mask)
    chunks = [c for c in np.array_split(mats, cores) if len(c)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_measure_chunk, [(w["kind"], *vols, mats[:1], a)] * cores)   # start-up, untimed
        t0 = time.perf_counter()
        pool.map(_measure_chunk, [(w["kind"], *vols, c, a) for c in chunks])
        dt = time.perf_counter() - t0
    return dt, n_particles * int(np.prod(pair.tgt.shape)), cores


def run_reference(args, rank, world):
    if rank != 0:
        return
    if WORKLOADS[args.workload]["kind"] == "batch":      # a bounded sample of one image-based member
        m = batch_members(2, 7, small=WORKLOADS[args.workload].get("small", False))[1]
        w = dict(name=WORKLOADS[args.workload]["name"], kind=m["mode"], rot_limit_deg=30.0, trans_limit=25.0,
                 seed=1)
        pair = m["pair"]
    elif WORKLOADS[args.workload]["kind"] in ("proposal", "conv"):
        w, pair, _ = load_workload("image224", 0)   # the filter the proposal seeds: the image workload's pair
    else:
        w, pair, _ = load_workload(args.workload, 0)
    n, k = cpu_sample_size(args, w)[0], 1
    times, units = [], 0
    for i in range(args.warmup + args.steps):
        dt, u = oracle_sample(w, pair, n, k)
        if i >= args.warmup:
            times.append(dt)
            units = u
    tot = sum(times)
    value = units * len(times) / tot
    sample = (f"oracle (single-threaded C) on the same pair: {n} particles x {k} iteration "
              f"({units:.3g} dense evals) per step; warp excluded")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": w["name"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our path

def run_ours(args, rank, world, local):
    import torch

    import paper_2504_19930_gb300 as pk

    torch.cuda.set_device(local)
    pk.build()
    pk.load()
    dist = Dist(world)
    w, pair, frames = load_workload(args.workload, rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    src_d = torch.from_numpy(pair.src).to(dev)
    tgt_d = torch.from_numpy(pair.tgt).to(dev)
    fr_d = [torch.from_numpy(f).to(dev) for f in frames] if frames is not None else []
    out_d = [torch.empty(pair.tgt.shape, dtype=torch.uint8, device=dev) for _ in fr_d]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lr, lt = np.deg2rad(w["rot_limit_deg"]), w["trans_limit"]
    kind = w["kind"]

    if kind == "combined":
        smask_d = torch.from_numpy(pair.src_mask).to(dev)
        tmask_d = torch.from_numpy(pair.tgt_mask).to(dev)

    def make_reg():
        vols = dict(src=src_d, tgt=tgt_d) if kind != "mask_dice" else dict(src_mask=src_d, tgt_mask=tgt_d)
        if kind == "combined":
            vols.update(src_mask=smask_d, tgt_mask=tmask_d)
        return pk.Registration(kind, src_origin=pair.src_origin, tgt_origin=pair.tgt_origin,
                               n_particles=w["n_particles"], rot_limit=lr, trans_limit=lt, seed=w["seed"],
                               autotune=True, **vols)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps + args.warmup)]
    rec = {"measure_ms": 0.0, "measure_launches": 0, "evals": 0, "warp_ms": 0.0, "tile": None}

    def step(i, timed):
        flush.fill_(i & 0xFF)                      # L2 flush (outside the timed events)
        e0, e1, e2 = ev[i]
        e0.record(stream)
        reg = make_reg()
        rec["tile"] = reg.tile_shape()
        if timed:
            pk.pf_profile_begin(reg.ctx, w["n_iters"])
        reg.step(w["n_iters"])
        pose, _ = reg.estimate(with_score=False)
        e1.record(stream)
        if fr_d:
            pk.warp_sequence(fr_d, pair.src_dims, pair.src_origin, out_d, pair.tgt_dims, pair.tgt_origin,
                             pose, 1, stream=stream)
        e2.record(stream)
        if timed:
            ms, n = pk.pf_profile_end(reg.ctx)
            rec["measure_ms"] += ms
            rec["measure_launches"] += n
            _, _, _, evals, _ = pk.pf_get_log(reg.ctx, capacity=w["n_iters"])
            rec["evals"] += int(evals.sum())
        reg.close()
        return pose

    for i in range(args.warmup):
        step(i, False)
    torch.cuda.synchronize()
    l2_peak = l2_read_peak(pk, torch, dev, stream)
    torch.cuda.synchronize()
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    launches0 = pk.pf_kernel_launches()
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clocks:
        t0 = time.perf_counter()
        for i in range(args.warmup, args.warmup + args.steps):
            pose = step(i, True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    dist.barrier()
    launches = pk.pf_kernel_launches() - launches0
    step_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(args.warmup, args.warmup + args.steps)]
    warp_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(args.warmup, args.warmup + args.steps)]
    local_s = sum(step_ms) / 1e3
    t_max = dist.max(local_s)
    units = dense_units(w, pair) * args.steps
    total_units = dist.sum(units)
    value = total_units / t_max
    clk = clocks.summary()

    # roofline of the dominant kernel (the measurement)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk["sm_mhz"] or peaks.get("sm_max_mhz") or 2070.0
    peak_ops = sm_count * FP32_LANES_PER_SM * mhz * 1e6
    meas_s = rec["measure_ms"] / 1e3
    ops = OPS_PER_EVAL_MODE[kind]
    achieved = rec["evals"] * ops / meas_s if meas_s > 0 else 0.0
    sha = kernel_code_hash(MEASURE_SOURCES)
    ncu = NCU_COUNTERS.get(args.workload)
    ncu = ncu if ncu and ncu["measure_code_sha1"] == sha else None
    traffic = ncu["dram_bytes_per_launch"] if ncu else None
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "TOP/s",
                "frac": achieved / peak_ops if peak_ops else None, "traffic": traffic,
                "kernel": {"image_ncc": "k_measure<image>", "mask_dice": "k_measure<mask>",
                           "combined": "k_measure<image+mask>"}[kind], "ops_per_eval": ops,
                "evals_per_launch": rec["evals"] / max(rec["measure_launches"], 1),
                "avg_launch_ms": rec["measure_ms"] / max(rec["measure_launches"], 1),
                "share_of_step": rec["measure_ms"] / sum(step_ms),
                "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM} fp32 lanes x {mhz:.0f} MHz (median SM clock sampled during the timed steps)"}
    # the L2 roof of the same kernel: L2 -> L1 bytes per visited evaluation
    # (ncu capture of this workload and kernel) x the live evaluation rate,
    # against the L2 read bandwidth the probe measured on this GPU
    l2_bpe = ncu["l2_to_l1_bytes_per_eval"] if ncu else None
    l2_ach = l2_bpe * rec["evals"] / meas_s / 1e9 if (l2_bpe and meas_s > 0) else None
    roofline["l2"] = {"achieved": l2_ach, "peak": l2_peak, "unit": "GB/s",
                      "frac": l2_ach / l2_peak if (l2_ach and l2_peak) else None,
                      "bytes_per_eval": l2_bpe,
                      "peak_basis": "pf_probe_read: 48 MiB L2-resident buffer, 16-byte loads bypassing L1, "
                                    "best of 3 x 20 passes (CUDA events)",
                      "bytes_basis": "ncu l1tex__m_xbar2l1tex_read_bytes.sum / visited evaluations of one launch "
                                     "of this workload (null without a capture of the current kernel)"}

    # the sequence warp: algorithmic bytes (each frame read once, each output
    # written once) against the measured HBM copy rate
    roofline_warp = None
    if fr_d:
        wbytes = sum(f.nbytes for f in frames) + sum(o.numel() for o in out_d)
        wsec = statistics.mean(warp_ms) / 1e3
        hbm = peaks.get("hbm_gbs")
        roofline_warp = {"bound": "hbm", "kernel": "k_warp", "achieved": wbytes / wsec / 1e9 if wsec > 0 else None,
                         "peak": hbm, "unit": "GB/s",
                         "frac": (wbytes / wsec / 1e9 / hbm) if (hbm and wsec > 0) else None,
                         "bytes_per_launch": int(wbytes), "ms": 1e3 * wsec,
                         "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy)"}

    # end to end through the public API from pinned host buffers
    # Time-to-Dice: one traced registration (untimed) warps the LV-cavity
    # masks with the estimate after every iteration (Sec. 3.2 validation);
    # the first iteration whose Dice is within 0.005 of the final one, at the
    # measured time per iteration.
    trace = None
    if pair.src_mask is not None:
        vols = dict(src=src_d, tgt=tgt_d) if kind != "mask_dice" else dict(src_mask=src_d, tgt_mask=tgt_d)
        if kind != "mask_dice":
            vols.update(src_mask=torch.from_numpy(pair.src_mask).to(dev),
                        tgt_mask=torch.from_numpy(pair.tgt_mask).to(dev))
        with pk.Registration(kind, src_origin=pair.src_origin, tgt_origin=pair.tgt_origin,
                             n_particles=w["n_particles"], rot_limit=lr, trans_limit=lt, seed=w["seed"],
                             trace_estimate=True, **vols) as treg:
            treg.step(w["n_iters"])
            _, _, _, _, dice = treg.log()
        final = float(dice[-1])
        hit = settled_iteration(dice, final - 0.005) - 1
        ms_iter = statistics.mean(step_ms) / w["n_iters"]
        # Dice before registration (identity pose)
        with pk.Registration("mask_dice", src_mask=torch.from_numpy(pair.src_mask).to(dev),
                             tgt_mask=torch.from_numpy(pair.tgt_mask).to(dev),
                             src_origin=pair.src_origin, tgt_origin=pair.tgt_origin, n_particles=1) as z:
            M0, a0 = pk.pf_pose_matrix(np.zeros(6, np.float32), pair.src_dims, pair.src_origin,
                                       pair.tgt_origin)
            mom = z.measure(M0, a0)[0]
        bfull = int((pair.tgt_mask != 0).sum())
        before = 2.0 * int(mom[11]) / (int(mom[9]) + bfull) if int(mom[9]) + bfull else 0.0
        trace = {"dice_before": before, "final_dice": final, "iters_to_dice": hit + 1,
                 "time_to_dice_ms": (hit + 1) * ms_iter,
                 "criterion": "estimate Dice within 0.005 of final from this iteration on"}

    e2e = None
    if args.e2e_steps > 0:
        src_h = torch.from_numpy(pair.src).pin_memory()
        tgt_h = torch.from_numpy(pair.tgt).pin_memory()
        fr_h = [torch.from_numpy(f).pin_memory() for f in frames] if frames is not None else []
        out_h = [torch.empty(pair.tgt.shape, dtype=torch.uint8).pin_memory() for _ in fr_h]
        mode_kw = dict(src=src_h, tgt=tgt_h) if kind != "mask_dice" else dict(src_mask=src_h, tgt_mask=tgt_h)
        if kind == "combined":
            mode_kw.update(src_mask=torch.from_numpy(pair.src_mask).pin_memory(),
                           tgt_mask=torch.from_numpy(pair.tgt_mask).pin_memory())

        def e2e_step():
            return pk.register_sequence(kind, frames=fr_h, n_iters=w["n_iters"], src_origin=pair.src_origin,
                                        tgt_origin=pair.tgt_origin, out=out_h, n_particles=w["n_particles"],
                                        rot_limit=lr, trans_limit=lt, seed=w["seed"], **mode_kw)

        e2e_step()                                 # warm-up of the host path
        torch.cuda.synchronize()
        dist.barrier()
        times = []                                 # host wall time per call, L2 flush excluded
        for _ in range(args.e2e_steps):
            flush.fill_(2)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        e2e_s = dist.max(sum(times))
        h2d = pair.src.nbytes + pair.tgt.nbytes + sum(f.nbytes for f in (frames if frames is not None else []))
        d2h = sum(o.numel() for o in out_h) + 6 * 4
        e2e = {"value": dist.sum(units / args.steps * args.e2e_steps) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * e2e_s / args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, k = cpu_sample_size(args, w)
        dt, u = oracle_sample(w, pair, n, k)
        ncpu = os.cpu_count() or 1
        cpu = {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} particles x {k} iterations of the same pair ({u:.3g} dense evals, "
                         f"{dt:.1f} s single-threaded); warp excluded",
               "host": f"{ncpu} cores, {platform.machine()}"}
        if args.cpu_all_cores_particles > 0 and ncpu > 1:
            dt2, u2, c2 = oracle_measure_all_cores(w, pair, args.cpu_all_cores_particles, ncpu)
            cpu["all_cores"] = {
                "value": u2 / dt2, "unit": UNIT, "cores": c2,
                "sample": f"measurement only: {args.cpu_all_cores_particles} particles of the initial cloud "
                          f"split over {c2} spawned processes ({dt2:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "volume": "x".join(map(str, pair.src_dims)),
                       "n_particles": w["n_particles"], "n_iters": w["n_iters"],
                       "frames_warped": len(fr_d), "mode": kind,
                       "l2": "flushed before every step (256 MiB write, outside the timed events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "warp_ms_per_step": statistics.mean(warp_ms),
                       "tile": {"rows_per_item": rec["tile"][0], "items_per_warp": rec["tile"][1],
                                "autotuned": True},
                       "overlap_evals_per_step": rec["evals"] / args.steps,
                       "overlap_evals_per_s": rec["evals"] / local_s,
                       "time_to_dice": trace},
            "roofline": roofline, "roofline_warp": roofline_warp, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
            "wall_s_timed": wall, "final_pose": [float(v) for v in pose],
            "true_pose": [float(v) for v in pair.true_pose],
        }
        if world == 1 and args.workload == "image224" and not args.no_secondary:
            line["secondary"] = run_secondary()
        print(json.dumps(line), flush=True)
    dist.close()


def run_secondary():
    """The default run's short companions, each its own bench.py process on
    the same GPU after the main line's timed work: the 64^3 mask workload
    (1500 timed registrations) and the proposal network's largest
    convolution.  A summary of each line (or the reason it is missing)."""
    out = {}
    cmds = {"mask64": ["--workload", "mask64", "--no-cpu-baseline", "--e2e-steps", "2"],
            "conv32": ["--workload", "conv32", "--steps", "20"]}
    for name, extra in cmds.items():
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), *extra], capture_output=True, text=True,
                               timeout=600)
            lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
            if r.returncode != 0 or not lines:
                out[name] = {"missing": f"exit {r.returncode}: {r.stderr.strip().splitlines()[-1:]}"}
                continue
            d = json.loads(lines[-1])
            rf = d.get("roofline") or {}
            out[name] = {"workload": d["config"]["workload"], "metric": d["metric"], "value": d["value"],
                         "unit": d["unit"], "steps": d["steps"], "ms_per_step": d.get("ms_per_step"),
                         "roofline": {k: rf.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit", "frac",
                                                              "traffic")},
                         "l2_frac": (rf.get("l2") or {}).get("frac"), "e2e": d.get("e2e"),
                         "clocks": d.get("clocks"), "gradients": d.get("gradients")}
        except Exception as e:   # a companion's failure never costs the main line
            out[name] = {"missing": repr(e)}
    return out


def _member_pair(spec):
    """Pool worker: the synthetic pair of one batch member."""
    kind, pseed, dims = spec
    if kind == "mask_dice":
        return pfsynth.ellipsoid_pair(pseed, src_dims=dims, tgt_dims=dims,
                                      tgt_origin=(0.0, 0.0, float(int(0.2 * dims[2]))),
                                      semi_axes=(0.31 * dims[0], 0.22 * dims[1], 0.22 * dims[2]),
                                      max_trans=0.06 * min(dims))
    return pfsynth.speckle_pair(pseed, src_dims=dims, with_masks=True)


def batch_members(n_regs, seed, small=False):
    """The batched workload: registration r draws its grid (each axis 96..256),
    particle count {512, 1024, 4096, 8192}, iteration count 20..60 and mode
    (even r: mask Dice on an ellipsoid mask pair, odd r: image NCC on a speckle
    pair with its LV-cavity masks, which only the Dice trace reads), all from
    one seeded generator.  small: grids 40..80, particle counts {128, 256, 512,
    1024}, 8..16 iterations -- registrations too small to fill the GPU on
    their own.  The pairs are generated by spawned processes on the host
    cores."""
    rng = np.random.default_rng(seed)
    specs, out = [], []
    for r in range(n_regs):
        if small:
            dims = tuple(int(v) for v in rng.integers(40, 81, 3))
            N = int(rng.choice([128, 256, 512, 1024]))
            K = int(rng.integers(8, 17))
        else:
            dims = tuple(int(v) for v in rng.integers(96, 257, 3))
            N = int(rng.choice([512, 1024, 4096, 8192]))
            K = int(rng.integers(20, 61))
        kind = "mask_dice" if r % 2 == 0 else "image_ncc"
        specs.append((kind, seed * 1000 + r, dims))
        if kind == "mask_dice":
            out.append(dict(mode=kind, N=N, K=K, rot=np.deg2rad(15.0), trans=float(0.12 * min(dims))))
        else:
            out.append(dict(mode=kind, N=N, K=K, rot=np.deg2rad(30.0), trans=25.0))
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(n_regs, os.cpu_count() or 1))) as pool:
        for m, pair in zip(out, pool.map(_member_pair, specs)):
            m["pair"] = pair
    return out


def dice_trace(pk, torch, dev, m, est):
    """Dice (Eq. 4) of member m's LV masks warped by each logged estimate
    (est [K][6]): one nearest-neighbour mask measurement per estimate."""
    p = m["pair"]
    mats = []
    a = None
    for e in est:
        M, a = pk.pf_pose_matrix(np.asarray(e, np.float32), p.src_dims, p.src_origin, p.tgt_origin)
        mats.append(M)
    with pk.Registration("mask_dice", src_mask=torch.from_numpy(p.src_mask).to(dev),
                         tgt_mask=torch.from_numpy(p.tgt_mask).to(dev), src_origin=p.src_origin,
                         tgt_origin=p.tgt_origin, n_particles=1) as z:
        mom = z.measure(np.stack(mats), a)
    bfull = int((p.tgt_mask != 0).sum())
    A, C_ = mom[:, 9].astype(np.float64), mom[:, 11].astype(np.float64)
    return np.where(A + bfull > 0, 2.0 * C_ / np.maximum(A + bfull, 1), 0.0)


def run_batch(args, rank, world, local):
    """Batched registrations: all members stepped together (pf_batch, one
    CUDA-graph launch per batch iteration) against the same members stepped
    one after another (each member's iterations back to back), both timed with
    CUDA events around the iterations only (context creation excluded from
    both).  Both give every member the same trajectory bit for bit, so the
    comparison is of time alone.  Time-to-Dice: after the runs, each member's
    per-iteration estimates (its log) are scored by the Dice of its masks; a
    member has settled from the first iteration whose Dice stays within 0.005
    of its final Dice; the set has settled when its last member has.  The
    batched run reaches that when the batch iteration of the latest-settling
    member ends; the sequential run when that member's iteration ends, after
    all the members before it ran in full."""
    import torch

    import paper_2504_19930_gb300 as pk

    torch.cuda.set_device(local)
    pk.build()
    pk.load()
    dist = Dist(world)
    wname = args.workload
    members = batch_members(args.batch_regs, 7 + rank, small=WORKLOADS[wname].get("small", False))
    dev = torch.device("cuda", local)
    dev_vols = []
    for m in members:
        p = m["pair"]
        if m["mode"] == "mask_dice":
            dev_vols.append(dict(src_mask=torch.from_numpy(p.src_mask).to(dev),
                                 tgt_mask=torch.from_numpy(p.tgt_mask).to(dev)))
        else:
            dev_vols.append(dict(src=torch.from_numpy(p.src).to(dev), tgt=torch.from_numpy(p.tgt).to(dev)))

    def make_all():
        return [pk.Registration(m["mode"], src_origin=m["pair"].src_origin, tgt_origin=m["pair"].tgt_origin,
                                n_particles=m["N"], rot_limit=m["rot"], trans_limit=m["trans"], seed=r,
                                autotune=True, **dev_vols[r]) for r, m in enumerate(members)]

    stream = torch.cuda.current_stream()
    units = sum(m["N"] * m["K"] * int(np.prod(m["pair"].tgt.shape)) for m in members)
    Kmax = max(m["K"] for m in members)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {"batched": [], "sequential": []}
    marks = {}
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    launches = 0
    with ClockSampler(gpu_id) as clocks:
        for i in range(args.warmup + args.steps):
            timed = i >= args.warmup
            for how in ("batched", "sequential"):
                regs = make_all()
                batch = pk.Batch(regs, [m["K"] for m in members]) if how == "batched" else None
                flush.fill_(i & 0xFF)
                torch.cuda.synchronize()
                dist.barrier()
                l0 = pk.pf_kernel_launches()
                e0 = torch.cuda.Event(enable_timing=True)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(Kmax if batch is not None else len(members))]
                e0.record(stream)
                if batch is not None:
                    for k in range(Kmax):             # one batch iteration per launch, an event after each
                        batch.step(1)
                        ev[k].record(stream)
                else:
                    for r, (g, m) in enumerate(zip(regs, members)):
                        g.step(m["K"])
                        ev[r].record(stream)
                torch.cuda.synchronize()
                if timed:
                    launches += pk.pf_kernel_launches() - l0
                    res[how].append(e0.elapsed_time(ev[-1]) / 1e3)
                    marks[how] = [e0.elapsed_time(e) / 1e3 for e in ev]
                if how == "sequential" and i == args.warmup + args.steps - 1:
                    logs = [g.log()[0] for g in regs]          # per-iteration estimates
                if batch is not None:
                    batch.close()
                for g in regs:
                    g.close()
    clk = clocks.summary()
    tb = dist.max(sum(res["batched"]))
    ts = dist.max(sum(res["sequential"]))
    total = dist.sum(units * args.steps)

    # time-to-Dice of the whole set (see the docstring)
    settle, final = [], []
    for m, est in zip(members, logs):
        d = dice_trace(pk, torch, dev, m, est)
        final.append(float(d[-1]))
        settle.append(settled_iteration(d, d[-1] - 0.005))
    last = max(settle)
    ttd_b = marks["batched"][last - 1]
    seq_end = marks["sequential"]
    ttd_s = 0.0
    for r, (m, k) in enumerate(zip(members, settle)):
        start = seq_end[r - 1] if r > 0 else 0.0
        ttd_s = max(ttd_s, start + (seq_end[r] - start) * k / m["K"])
    if rank == 0:
        line = {"metric": METRIC, "value": total / tb, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * tb / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS[wname]["name"], "registrations": len(members),
                           "mask_based": sum(m["mode"] == "mask_dice" for m in members),
                           "dims": ["x".join(map(str, m["pair"].src_dims)) for m in members],
                           "particles": [m["N"] for m in members], "iterations": [m["K"] for m in members],
                           "dense_evals_per_step": units,
                           "sequential_ms_per_step": 1e3 * ts / args.steps,
                           "batched_speedup_vs_sequential": ts / tb,
                           "time_to_dice": {
                               "criterion": "every member's estimate Dice within 0.005 of its final Dice from "
                                            "its settle iteration on (the same bits batched and sequential)",
                               "settle_iterations": settle, "final_dice": final,
                               "batched_ms": 1e3 * ttd_b, "sequential_ms": 1e3 * ttd_s,
                               "batched_gain": ttd_s / ttd_b},
                           "l2": "flushed before every step (256 MiB write, outside the timed events)"},
                "roofline": None, "cpu_baseline": None, "e2e": None,
                "gpu_launches": int(launches),
                "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]}}
        print(json.dumps(line), flush=True)
    dist.close()


def conv_roofline(pk, torch, dev, stream, batch, reps=20):
    """Tensor-core roofline of the network's largest convolution, 32^3 x 32
    -> 16^3 x 32 at the training batch, timed alone with CUDA events (the
    input, 67 MB at batch 32, is rewritten between launches by nothing: it is
    read-only and L2-resident after the first launch, which is the training
    pass's situation too)."""
    D = 32
    x = torch.randn((batch, D, D, D, 32), device=dev).abs().to(torch.bfloat16)
    wt = (0.05 * torch.randn((32, 64, 32), device=dev)).to(torch.bfloat16)
    bias = torch.zeros(32, device=dev)
    y = torch.empty((batch, D // 2, D // 2, D // 2, 32), dtype=torch.bfloat16, device=dev)
    for _ in range(3):
        pk.nn_conv3d_forward(x, wt, bias, y)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(reps):
        pk.nn_conv3d_forward(x, wt, bias, y)
    c1.record(stream)
    torch.cuda.synchronize()
    assert pk.nn_status() == 0, "a tensor-core wait gave up"
    conv_s = c0.elapsed_time(c1) / 1e3 / reps
    conv_flops = 2.0 * batch * (D // 2) ** 3 * 32 * 64 * 32
    peaks = measured_peaks()
    bf16_peak = peaks.get("bf16_tflops") or 1900.0
    return {"bound": "tensor", "kernel": "k_conv_planes (tcgen05, bf16 -> fp32, input planes staged once in shared memory)",
            "achieved": conv_flops / conv_s / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": conv_flops / conv_s / 1e12 / bf16_peak, "traffic": None,
            "flops_per_launch": conv_flops, "avg_launch_ms": 1e3 * conv_s,
            "peak_basis": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)" if peaks.get("bf16_tflops")
            else "fallback 1.9 PFLOP/s"}


def run_conv(args, rank, world, local):
    """The network's largest convolution alone (for profiling): one JSON line."""
    import torch

    import paper_2504_19930_gb300 as pk

    torch.cuda.set_device(local)
    pk.build()
    pk.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    r = conv_roofline(pk, torch, dev, stream, 32, reps=args.steps)
    grads = conv_grad_times(pk, torch, dev, stream, 32, reps=args.steps)
    if rank == 0:
        print(json.dumps({"metric": "bf16 TFLOP/s of the proposal network's 32^3 x 32 -> 16^3 x 32 convolution",
                          "value": r["achieved"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
                          "warmup": 3, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                          "config": {"workload": WORKLOADS["conv32"]["name"]}, "roofline": r,
                          "gradients": grads}), flush=True)


def conv_grad_times(pk, torch, dev, stream, batch, reps=20):
    """The same layer's two gradients, each timed alone with CUDA events:
    the data gradient (the 8 taps of each stride phase per input voxel) and
    the weight gradient.  TFLOP/s counts the algorithmic products only (the
    forward's 2 B Do^3 32 64 32 for each)."""
    D, Do = 32, 16
    dy = (0.1 * torch.randn((batch, Do, Do, Do, 32), device=dev)).to(torch.bfloat16)
    wt = (0.05 * torch.randn((32, 64, 32), device=dev)).to(torch.bfloat16)
    act = torch.randn((batch, D, D, D, 32), device=dev).relu().to(torch.bfloat16)
    x = torch.randn((batch, D, D, D, 32), device=dev).abs().to(torch.bfloat16)
    dx = torch.empty((batch, D, D, D, 32), dtype=torch.bfloat16, device=dev)
    dw = torch.zeros((32, 64, 32), dtype=torch.float32, device=dev)
    flops = 2.0 * batch * Do ** 3 * 32 * 64 * 32
    out = {}
    for name, fn in (("data", lambda: pk.nn_conv3d_backward_data(dy, wt, act, dx)),
                     ("weights", lambda: pk.nn_conv3d_backward_weights(x, dy, dw))):
        for _ in range(3):
            fn()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(reps):
            fn()
        c1.record(stream)
        torch.cuda.synchronize()
        assert pk.nn_status() == 0, "a tensor-core wait gave up"
        sec = c0.elapsed_time(c1) / 1e3 / reps
        out[name] = {"avg_launch_ms": 1e3 * sec, "tflops": flops / sec / 1e12}
    return out


def cpu_sample_size(args, w):
    """(particles, iterations) of the oracle's bounded sample: about 10-30 s of
    single-threaded work on the 16-core Arm host for the image and combined
    workloads (64 particles x 2 iterations), the whole registration for the
    small mask workload (a few seconds)."""
    small = w["kind"] == "mask_dice"
    n = getattr(args, "cpu_sample_particles", None) or (w["n_particles"] if small else 64)
    k = getattr(args, "cpu_sample_iters", None) or (w["n_iters"] if small else 2)
    return n, k


def _held_out_pair(seed):
    """Pool worker: one held-out speckle pair with masks (returned, not cached)."""
    return pfsynth.speckle_pair(seed, with_masks=True)


def run_proposal(args, rank, world, local):
    """Learned proposal against the plain filter: train the network on
    synthetic pairs (GPU generator), then on held-out seeded speckle pairs
    compare the time until the estimate's mask Dice comes within 0.005 of the
    plain filter's final Dice: the plain filter (N = 2048, uniform cloud) vs
    prediction + a seeded filter (N = 512).  A seeded run that never gets
    there falls back to the plain filter and is charged both times."""
    import torch

    import paper_2504_19930_gb300 as pk

    torch.cuda.set_device(local)
    pk.build()
    pk.load()
    dist = Dist(world)
    w = WORKLOADS["proposal"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    lr_, lt = np.deg2rad(w["rot_limit_deg"]), w["trans_limit"]
    K = w["n_iters"]
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731

    # --- training (timed with events; not part of a registration's time)
    net = pk.Proposal(max_batch=w["train_batch"], seed=w["seed"] + rank)
    e0, e1 = ev(), ev()
    e0.record(stream)
    loss = net.train(w["train_steps"], batch=w["train_batch"], lr=w["lr"], data_seed=11 + rank,
                     vol_dims=(224, 208, 176), rot_limit=lr_, trans_limit=lt)
    e1.record(stream)
    torch.cuda.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    assert pk.nn_status() == 0, "a tensor-core wait gave up during training"

    roofline = conv_roofline(pk, torch, dev, stream, w["train_batch"])

    # --- held-out pairs, generated on the host cores by spawned processes
    # while the GPU evaluates the previous ones
    n_eval = args.proposal_eval_pairs
    seeds = [5000 + 1000 * rank + i for i in range(n_eval)]
    import multiprocessing as mp
    rows = []
    units_learned, secs_learned = 0, 0.0
    launches0 = pk.pf_kernel_launches()
    with mp.get_context("spawn").Pool(max(1, min(len(seeds), os.cpu_count() or 1))) as pool, \
            ClockSampler(local) as clocks:
        for pair in pool.imap(_held_out_pair, seeds):
            vols = dict(src=torch.from_numpy(pair.src).to(dev), tgt=torch.from_numpy(pair.tgt).to(dev),
                        src_mask=torch.from_numpy(pair.src_mask).to(dev),
                        tgt_mask=torch.from_numpy(pair.tgt_mask).to(dev))
            geo = dict(src_origin=pair.src_origin, tgt_origin=pair.tgt_origin, rot_limit=lr_, trans_limit=lt,
                       seed=w["seed"], trace_estimate=True)
            # plain filter
            torch.cuda.synchronize()
            a0, a1 = ev(), ev()
            a0.record(stream)
            with pk.Registration("image_ncc", n_particles=w["plain_particles"], **geo, **vols) as reg:
                reg.step(K)
                est_plain, _ = reg.estimate(with_score=False)
                a1.record(stream)
                torch.cuda.synchronize()
                _, _, _, _, dice_p = reg.log()
            plain_ms = a0.elapsed_time(a1)
            final = float(dice_p[-1])
            hit_p = settled_iteration(dice_p, final - 0.005) - 1
            plain_ttd = plain_ms * (hit_p + 1) / K
            # learned proposal + seeded filter
            b0, b1, b2 = ev(), ev(), ev()
            b0.record(stream)
            mean, std = net.predict(vols["src"], vols["tgt"], pair.src_origin, pair.tgt_origin)
            b1.record(stream)
            lim = np.array([lr_] * 3 + [lt] * 3, np.float32)
            sd = np.clip(std * w["std_inflate"], 1e-3 * lim, lim).astype(np.float32)
            with pk.Registration("image_ncc", n_particles=w["n_particles"], **geo, **vols) as reg:
                reg.seed_gaussian(np.clip(mean, -lim, lim), sd)
                reg.step(K)
                est_l, _ = reg.estimate(with_score=False)
                b2.record(stream)
                torch.cuda.synchronize()
                _, _, _, evals_l, dice_l = reg.log()
            pred_ms, filt_ms = b0.elapsed_time(b1), b1.elapsed_time(b2)
            units_learned += w["n_particles"] * K * int(np.prod(pair.tgt.shape))
            secs_learned += filt_ms / 1e3
            it_l = settled_iteration(dice_l, final - 0.005)
            if it_l is not None:
                learned_ttd = pred_ms + filt_ms * it_l / K
                fell_back = False
            else:   # never settles within 0.005 of the plain result: charged the plain run as well
                learned_ttd = pred_ms + filt_ms + plain_ttd
                fell_back = True
            err = np.abs(mean.astype(np.float64) - est_plain.astype(np.float64))
            rows.append(dict(plain_ttd_ms=plain_ttd, learned_ttd_ms=learned_ttd, plain_final_dice=final,
                             learned_final_dice=float(dice_l[-1]), fell_back=fell_back, predict_ms=pred_ms,
                             plain_iters=hit_p + 1, learned_iters=it_l,
                             err_rot_deg=float(np.rad2deg(err[:3]).max()), err_trans=float(err[3:].max()),
                             true_err_rot_deg=float(np.rad2deg(np.abs(mean[:3] - pair.true_pose[:3])).max())))
    launches = pk.pf_kernel_launches() - launches0
    clk = clocks.summary()
    t_max = dist.max(secs_learned)
    value = dist.sum(units_learned) / t_max if t_max > 0 else 0.0
    if rank == 0:
        med = lambda k: float(np.median([r[k] for r in rows]))   # noqa: E731
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n_eval,
                "warmup": 0, "ms_per_step": 1e3 * secs_learned / max(len(rows), 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16 network / f32 filter", "data": "synthetic",
                "config": {"workload": w["name"], "n_eval_pairs": len(rows),
                           "time_to_dice": {"plain_ms_median": med("plain_ttd_ms"),
                                            "learned_ms_median": med("learned_ttd_ms"),
                                            "speedup_median": med("plain_ttd_ms") / med("learned_ttd_ms"),
                                            "fallbacks": sum(r["fell_back"] for r in rows),
                                            "criterion": "estimate Dice within 0.005 of the plain filter's final Dice from that iteration on"},
                           "pairs": rows,
                           "training": {"steps": w["train_steps"], "batch": w["train_batch"], "seconds": train_s,
                                        "loss_first100": float(loss[:100].mean()),
                                        "loss_last100": float(loss[-100:].mean())}},
                "roofline": roofline, "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    dist.close()


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload in ("batch64", "batch64_small"):
        run_batch(args, rank, world, local)
        return
    if args.workload == "proposal":
        run_proposal(args, rank, world, local)
        return
    if args.workload == "conv32":
        run_conv(args, rank, world, local)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
