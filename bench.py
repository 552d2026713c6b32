#!/usr/bin/env python3
"""Benchmark of the ReFusion per-frame hot path on GB300.

One step = one whole frame through the public C ABI (rf_process_frame):
registration -> residual mask -> registration without masked pixels ->
integration with free-space carving, on the 640x480 static room workload
(fx=fy=525, 1 cm voxels, tau 0.1 m, 2^20 hash buckets, seeded synthetic
frames with Kinect-like noise).  Prints one JSON line.  The default run is
the configuration's 300-frame forward trajectory (10 warm-up + 290 timed
frames); runs asked for more frames than that play the 300 back and forth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 (under torch.distributed.run): one independent camera stream per GPU
(weak scaling, no data-path collective); the timed region is bracketed by a
barrier and the max over ranks is reported.
--impl reference: the FP64 CPU oracle on one host core, each step one whole
640x480 frame of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import gc
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s @640x480 and % HBM roofline; p99 frame latency, 32 streams"
CONFIG = "static"
VOXEL, TAU, N_BUCKETS, MAX_BLOCKS = 0.01, 0.1, 1 << 20, 400_000
L2_FLUSH_BYTES = 256 << 20


def _render(args):
    seed, i, n = args
    from synth import make_sequence
    seq = make_sequence(CONFIG, seed, n_frames=n)
    d, rgb, T, _ = seq.frame(i)
    return d, rgb, T


MAX_RENDERED = 300  # the static configuration's length; longer runs play it back and forth
PRECISION_RENDERED = 120  # distinct frames of the precision sequence; longer runs play them back and forth


def frame_order(n_rendered: int, n: int):
    """Index of the rendered frame used at step n (0-based over warm-up and
    timed steps): 0, 1, .., n_rendered-1, n_rendered-2, .., 1, 0, 1, .. so the
    camera moves back and forth along the rendered trajectory."""
    if n_rendered == 1:
        return [0] * n
    period = 2 * (n_rendered - 1)
    return [k % period if k % period < n_rendered else period - k % period for k in range(n)]


def make_frames(seed: int, n: int, workers: int):
    """Renders n frames of the seeded sequence in a spawn pool (before CUDA)."""
    jobs = [(seed, i, n) for i in range(n)]
    if workers <= 1:
        return [_render(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_render, jobs)


# ---------------------------------------------------------------------------
# serving workload: 32 streams, mixed 320x240 / 640x480 / 1280x720, voxel
# 1-4 cm, 0-3 movers, Poisson arrivals at a mean of 30 frames/s per stream
# ---------------------------------------------------------------------------
SERVING_CAMS = ("qvga", "vga", "hd")
SERVING_VOXELS = (0.01, 0.02, 0.03, 0.04)
SERVING_BUDGET = 120 * 10 ** 9
SERVING_FPS = 30.0


def serving_plan(n_streams: int):
    plan = []
    for s in range(n_streams):
        cam = SERVING_CAMS[s % 3]
        voxel = SERVING_VOXELS[(s // 3) % 4]
        if cam == "hd":
            voxel = max(voxel, 0.02)
        plan.append(dict(name=f"s{s:02d}", cam=cam, voxel=voxel, movers=(s // 2) % 4, seed=3000 + s))
    return plan


def _render_clip(args):
    """One stream's clip (rendered in a worker process)."""
    st, clip = args
    from synth.scenes import CAM_HD, CAM_QVGA, CAM_VGA, Sequence
    cam = {"qvga": CAM_QVGA, "vga": CAM_VGA, "hd": CAM_HD}[st["cam"]]
    seq = Sequence("dynamic" if st["movers"] else "static", st["seed"], n_frames=clip, camera=cam,
                   movers=st["movers"], coverage_scale=4)
    frames = []
    for i in range(clip):
        d, rgb, _, _ = seq.frame(i)
        frames.append((d, rgb))
    return frames, seq.poses[0].copy()


def render_serving_clips(plan, clip: int, workers: int):
    """Every stream's clip, rendered in a spawn pool (before CUDA), the
    largest frames first so that the pool stays busy."""
    cost = {"hd": 12, "vga": 4, "qvga": 1}
    jobs = sorted(range(len(plan)), key=lambda k: -cost[plan[k]["cam"]])
    if workers <= 1:
        out = {k: _render_clip((plan[k], clip)) for k in jobs}
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_render_clip, [(plan[k], clip) for k in jobs], chunksize=1)
        out = dict(zip(jobs, res))
    return [out[k] for k in range(len(plan))]


def volume_size(voxel: float):
    """Blocks and buckets of a serving volume (room-scale clips)."""
    blocks = {0.01: 300_000, 0.02: 100_000, 0.03: 50_000, 0.04: 30_000}[voxel]
    buckets = 1 << max(10, (blocks // 2 - 1).bit_length())
    return blocks, buckets


def _serving_specs(R, plan, clips, rate, seconds, rng, storage, bursts=None):
    """StreamSpecs of the plan: Poisson arrivals at `rate` frames/s per stream
    for `seconds` (bursts: per stream a list of (start, length) windows with
    arrivals only inside them), each stream playing its clip back and forth."""
    import torch
    from synth.scenes import CAM_HD, CAM_QVGA, CAM_VGA
    from paper_1905_02082_gb300.serving import StreamSpec, pingpong, poisson_arrivals
    cams = {"qvga": CAM_QVGA, "vga": CAM_VGA, "hd": CAM_HD}
    specs = []
    for k, (st, (frames, pinned, T0)) in enumerate(zip(plan, clips)):
        cam = cams[st["cam"]]
        if bursts is None:
            arr = [t for t in poisson_arrivals(rng, int(rate * seconds * 3) + 10, rate) if t < seconds]
        else:
            arr = []
            for t0, length in bursts[k]:
                arr += [t0 + t for t in poisson_arrivals(rng, int(rate * length * 3) + 10, rate) if t < length]
        blocks, buckets = volume_size(st["voxel"])
        specs.append(StreamSpec(name=st["name"], width=cam.width, height=cam.height,
                                K=R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy), voxel_size=st["voxel"], frames=pinned,
                                order=pingpong(len(pinned), len(arr)), arrivals=arr, T0=T0, start=0.0, trunc=TAU,
                                n_buckets=buckets, max_blocks=blocks, storage=storage))
    return specs


def _serve(R, specs, budget, mode, evict_idle_s=0.25):
    from paper_1905_02082_gb300.serving import ServingEngine, StreamSpec, summarize
    eng = ServingEngine(budget, mode=mode, evict_idle_s=evict_idle_s)
    # warm-up: three frames per stream, so that graph capture and first-touch costs stay out of the run
    warm = [StreamSpec(**{**sp.__dict__, "order": sp.order[:3], "arrivals": [0.0, 0.001, 0.002]}) for sp in specs]
    eng.run(warm, time_limit=300.0)
    eng.results.clear()
    eng.batch_ms.clear()
    for k in ("evictions", "restores", "batches", "slot_reuses"):
        eng.stats[k] = 0
    res = eng.run(specs, time_limit=600.0)
    summ = summarize(res)
    summ.update({k: eng.stats[k] for k in ("evictions", "restores", "batches", "peak_bytes")})
    summ["offered_frames"] = sum(len(sp.arrivals) for sp in specs)
    eng.close()
    return summ


def run_serving(R, plan, clips, args):
    """The continuous-batching serving loop against the plain per-stream path
    on the same Poisson arrivals, at offered loads from 30 frames/s per stream
    up past the GPU's capacity, and one run whose memory budget binds."""
    import torch
    pinned = []
    for st, (frames, T0) in zip(plan, clips):
        pinned.append((frames, [(torch.from_numpy(np.ascontiguousarray(d, dtype=np.uint16)).pin_memory(),
                                 torch.from_numpy(np.ascontiguousarray(c)).pin_memory()) for d, c in frames], T0))
    out = {"streams": len(plan), "clip_frames": args.serving_clip, "budget_bytes": SERVING_BUDGET,
           "mix": {c: sum(1 for st in plan if st["cam"] == c) for c in SERVING_CAMS},
           "workload": "32 streams, 320x240/640x480/1280x720 cycled, voxel 1-4 cm (>=2 cm at 1280x720), 0-3 movers, "
                       "Poisson arrivals; each stream plays a rendered clip back and forth; frames in page-locked "
                       "host memory, read by the batch's staging kernel", "loads": []}
    for rate in args.serving_rates:
        row = {"fps_per_stream": rate, "offered_frames_per_s": rate * len(plan)}
        for name, mode, storage in (("batch_fp16", "batch", R.STORAGE_FP16),
                                    ("per_stream_fp32", "per_stream", R.STORAGE_FP32)):
            rng = np.random.default_rng(77)  # the same arrivals for both forms
            specs = _serving_specs(R, plan, pinned, rate, args.serving_seconds, rng, storage)
            row[name] = _serve(R, specs, SERVING_BUDGET, mode)
        out["loads"].append(row)
    # a budget that binds: 40 % of the streams' volumes; each stream sends two
    # bursts (staggered), so idle streams are evicted to the host and restored
    rng = np.random.default_rng(78)
    bursts = [[(0.05 * k % 0.8, 0.35), (1.0 + 0.05 * k % 0.8, 0.35)] for k in range(len(plan))]
    specs = _serving_specs(R, plan, pinned, SERVING_FPS, 0.0, rng, R.STORAGE_FP16, bursts=bursts)
    total = sum(sp.footprint() for sp in specs)
    budget = int(0.4 * total)
    binding = _serve(R, specs, budget, "batch", evict_idle_s=0.1)
    binding.update({"budget_bytes": budget, "all_volumes_bytes": total,
                    "arrivals": "two 0.35 s Poisson bursts per stream at 30 frames/s, starts staggered by 50 ms"})
    out["budget_binding_fp16"] = binding
    return out


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


FLOPS_PER_SAMPLE = 320  # FP32 flops of one sampled pixel and cost evaluation (hand count; the ALU estimate only)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic bytes of one registration on this workload: the distinct voxels and
# blocks its lookups touch, plus every pixel's depth and colour (and the mask of
# the second registration), counted by the FP64 oracle on the static room and
# stored with the script that wrote it.
FOOTPRINT = os.path.join(ROOT, "tests", "golden", "track_footprint_static.json")
# DRAM bytes (read + write) per launch on this workload from one ncu capture of the
# kernel as it stands (None once the kernel has changed since its capture).
REGISTER_DRAM_BYTES = 7.148288e6 + 7.936e3
INTEGRATE_DRAM_BYTES = 37.397248e6 + 107.52e3


def rank_seed(rank: int) -> int:
    """Each rank is an independent camera stream: its own seeded sequence."""
    return 1000 + rank


def max_over_ranks(value_ms: float, dist, device) -> float:
    """The timed region of the slowest rank (the whole job's time)."""
    if dist is None:
        return value_ms
    import torch
    t = torch.tensor([value_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, timed_ms: float) -> float:
    """Frames of all ranks divided by the slowest rank's timed region."""
    return world * steps / (timed_ms / 1000.0)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _oracle_frame(O, d, rgb, cam):
    return O.FrameData(d, rgb, cam.fx, cam.fy, cam.cx, cam.cy)


def _oracle_stream(args):
    """One independent camera stream on the oracle (a worker process): frame 0
    integrated at its pose, then whole frames 1..n timed; returns seconds."""
    seed, n = args
    from oracle import oracle as O
    from synth import make_sequence
    seq = make_sequence(CONFIG, seed)
    cam = seq.camera
    vol = O.OracleVolume(voxel_size=VOXEL, trunc=TAU)
    d, rgb, T, _ = seq.frame(0)
    T, _, _ = vol.process_frame(_oracle_frame(O, d, rgb, cam), T)
    frames = [seq.frame(i)[:2] for i in range(1, n + 1)]
    t0 = time.perf_counter()
    for d, rgb in frames:
        T, _, _ = vol.process_frame(_oracle_frame(O, d, rgb, cam), T)
    return time.perf_counter() - t0


def run_reference(args):
    """FP64 oracle on the host cores, one thread: every step is one whole
    640x480 frame of the workload (track, mask, re-track, integrate)."""
    from oracle import oracle as O
    from synth import make_sequence
    n = args.warmup + args.steps
    seq = make_sequence(CONFIG, 0)
    cam = seq.camera
    frames = make_frames(0, n + 1, max(1, min(16, os.cpu_count() or 1)))
    vol = O.OracleVolume(voxel_size=VOXEL, trunc=TAU)
    T = None
    times = []
    for i in range(n + 1):
        d, rgb, Tgt = frames[i]
        t0 = time.perf_counter()
        T, _, _ = vol.process_frame(_oracle_frame(O, d, rgb, cam), Tgt if T is None else T)
        dt = time.perf_counter() - t0
        if i > args.warmup:  # frame 0 (integration only) and the warm-up frames untimed
            times.append(dt)
    total = sum(times)
    fps = len(times) / total
    sample = (f"whole 640x480 frames {args.warmup + 1}-{n} of the static room (frame 0 integrated at its pose and "
              f"{args.warmup} warm-up frames untimed), one thread")
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "static room 640x480, fx=fy=525, voxel 1 cm, tau 0.1 m", "global_batch": 1,
                       "seq_len": 1, "parallelism": "none (single-threaded CPU oracle)"},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline(n_frames: int = 3):
    """The oracle, as it stands, on bounded samples of the workload: whole
    640x480 frames on one thread; the tiny configuration in full; and all
    host cores at once, one independent stream per core (the oracle itself is
    sequential: streams are its only parallelism)."""
    from oracle import oracle as O
    from synth import make_sequence
    cores = max(1, os.cpu_count() or 1)
    t_single = _oracle_stream((0, n_frames))
    tiny = make_sequence("tiny", 0)
    tcam = tiny.camera
    tfr = [tiny.frame(i) for i in range(len(tiny))]
    tvol = O.OracleVolume(voxel_size=0.02, trunc=TAU)
    T = None
    t0 = time.perf_counter()
    for d, rgb, Tgt, _ in tfr:
        T, _, _ = tvol.process_frame(_oracle_frame(O, d, rgb, tcam), Tgt if T is None else T)
    t_tiny = time.perf_counter() - t0
    with mp.get_context("spawn").Pool(cores) as pool:
        t_all = pool.map(_oracle_stream, [(2000 + k, 1) for k in range(cores)])
    all_fps = cores / max(t_all)
    return {"value": n_frames / t_single, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"whole 640x480 frames 1-{n_frames} of the static room (frame 0 integrated at its pose, "
                      f"untimed), one thread",
            "all_cores": {"value": all_fps, "unit": "frames/s", "cores": cores,
                          "sample": f"{cores} independent streams (one per core, distinct seeds), one whole "
                                    f"640x480 frame each after its first; value = streams / slowest stream's time"},
            "tiny_full": {"frames_per_s": (len(tfr) - 1) / t_tiny, "frames": len(tfr),
                          "sample": "the tiny configuration in full (160x120, 2 cm voxels), one thread"}}


def run_single(R, frames, K, cam, dev, stream, flush, args, storage):
    """The single-stream loop of the headline number in another storage mode
    (same frames, same timing rules): frames/s and per-frame p50/p99."""
    import torch
    d_depth = [torch.from_numpy(f[0].astype(np.int32)).to(dev).to(torch.uint16).contiguous() for f in frames]
    d_rgb = [torch.from_numpy(f[1]).to(dev).contiguous() for f in frames]
    vol = R.Volume(n_buckets=N_BUCKETS, max_blocks=MAX_BLOCKS, max_width=cam.width, max_height=cam.height,
                   voxel_size=VOXEL, trunc=TAU, storage=storage)
    T = torch.as_tensor(frames[0][2], device=dev).contiguous()
    Tn = torch.empty_like(T)
    order = frame_order(len(frames), args.warmup + args.steps)
    for w in range(args.warmup):
        i = order[w]
        R.rf_process_frame(vol.h, vol.frame(d_depth[i], d_rgb[i], K), T, Tn, None, None, stream)
        T, Tn = Tn, T
    vol.sync()
    ms = []
    for k in range(args.steps):
        i = order[args.warmup + k]
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        R.rf_process_frame(vol.h, vol.frame(d_depth[i], d_rgb[i], K), T, Tn, None, None, stream)
        b.record(stream)
        T, Tn = Tn, T
        b.synchronize()
        ms.append(a.elapsed_time(b))
    vol.sync()
    vol.close()
    return {"storage": "fp16" if storage else "fp32", "frames_per_s": len(ms) / (sum(ms) / 1000.0),
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))}}


def _render_precision(args):
    i, n = args
    from synth import make_sequence
    return make_sequence("precision", 0, n_frames=n).frame(i)[:3]


def run_precision(R, frames, order, dev, stream, flush, warmup):
    """The precision configuration (1280x720, voxel 0.5 cm, tau 5 cm, 2^22
    buckets) through rf_process_frame, FP16 storage and FP32 storage on the
    same frames: frames/s and per-frame latency of each (same timing rules as
    the headline loop), and the FP16 form's drift from the FP32 form (pose
    difference per frame; the TSDF difference on the blocks both hold).
    order: the rendered frame used at each step (a sequence longer than the
    rendered frames plays them back and forth)."""
    import torch
    from synth.scenes import CAM_HD as cam
    K = R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy)
    d_depth = [torch.from_numpy(f[0].astype(np.int32)).to(dev).to(torch.uint16).contiguous() for f in frames]
    d_rgb = [torch.from_numpy(f[1]).to(dev).contiguous() for f in frames]
    out = {"workload": f"precision configuration: {len(order)} frames of 1280x720 (fx=fy=1050; {len(frames)} "
                       "rendered, played back and forth), voxel 0.5 cm, tau 5 cm, 2^22 buckets",
           "frames": len(order), "rendered": len(frames)}
    poses, snaps = {}, {}
    for name, storage in (("fp16", R.STORAGE_FP16), ("fp32", R.STORAGE_FP32)):
        vol = R.Volume(n_buckets=1 << 22, max_blocks=1_500_000, max_width=cam.width, max_height=cam.height,
                       voxel_size=0.005, trunc=0.05, storage=storage)
        T = torch.as_tensor(frames[0][2], device=dev).contiguous()
        Tn = torch.empty_like(T)
        ms, P = [], []
        for i, k in enumerate(order):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            R.rf_process_frame(vol.h, vol.frame(d_depth[k], d_rgb[k], K), T, Tn, None, None, stream)
            b.record(stream)
            T, Tn = Tn, T
            b.synchronize()
            if i >= warmup:
                ms.append(a.elapsed_time(b))
            P.append(T.cpu().numpy())
        vol.sync()
        poses[name] = P
        snaps[name] = vol.export()
        out[name] = {"frames_per_s": len(ms) / (sum(ms) / 1000.0),
                     "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
                     "blocks": int(len(snaps[name]["coords"]))}
        vol.close()
    dt = [float(np.linalg.norm(a[:3, 3] - b[:3, 3])) for a, b in zip(poses["fp16"], poses["fp32"])]
    dr = [float(np.arccos(np.clip((np.trace(a[:3, :3] @ b[:3, :3].T) - 1) / 2, -1, 1)))
          for a, b in zip(poses["fp16"], poses["fp32"])]
    gt = [float(np.linalg.norm(a[:3, 3] - frames[k][2][:3, 3])) for a, k in zip(poses["fp16"], order)]
    ka = {tuple(c): i for i, c in enumerate(snaps["fp16"]["coords"])}
    kb = {tuple(c): i for i, c in enumerate(snaps["fp32"]["coords"])}
    common = [c for c in ka if c in kb]
    ia = np.array([ka[c] for c in common], dtype=np.int64)
    ib = np.array([kb[c] for c in common], dtype=np.int64)
    both = (snaps["fp16"]["W"][ia] > 0) & (snaps["fp32"]["W"][ib] > 0)
    fd = np.abs(snaps["fp16"]["F"][ia][both].astype(np.float64) - snaps["fp32"]["F"][ib][both])
    out["fp16_vs_fp32"] = {"pose_m_max": max(dt), "pose_m_last": dt[-1], "pose_rad_max": max(dr),
                           "tsdf_abs_max_over_tau": float(fd.max() / 0.05) if fd.size else 0.0,
                           "tsdf_abs_mean_over_tau": float(fd.mean() / 0.05) if fd.size else 0.0,
                           "blocks_only_in_one": len(ka) + len(kb) - 2 * len(common),
                           "fp16_vs_ground_truth_m_max": max(gt)}
    return out


def run_virtual_depth(R, frames, K, cam, dev, stream, args, n_window=10):
    """Sec. III-E, second option, on the static workload: for each target
    frame, the temporary model of the n_window frames starting at it
    (integrated at their poses, here the ground truth) and the fill of the
    target's zero pixels (its edge dropout).  Per filled frame: the whole
    cost (reset + n_window integrations + ray casting, host clock around a
    synchronised sequence) and the ray-casting kernel alone (CUDA events)."""
    import torch
    n_targets = min(args.vd_frames, len(frames) - n_window)
    if n_targets <= 0:
        return None
    tmp = R.Volume(n_buckets=1 << 18, max_blocks=100_000, max_width=cam.width, max_height=cam.height,
                   voxel_size=VOXEL, trunc=TAU)
    d_depth = [torch.from_numpy(f[0].astype(np.int32)).to(dev).to(torch.uint16).contiguous() for f in frames]
    d_rgb = [torch.from_numpy(f[1]).to(dev).contiguous() for f in frames]
    Ts = [torch.as_tensor(f[2], device=dev).contiguous() for f in frames]
    out = torch.empty(cam.height, cam.width, dtype=torch.uint16, device=dev)
    far = int(round(tmp.params.d_max * tmp.params.depth_scale))
    total_ms, cast_ms, holes, filled = [], [], [], []
    for t in range(-2, n_targets):  # two untimed warm-up targets
        i = max(t, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tmp.reset()
        for j in range(i, i + n_window):
            R.rf_integrate_frame(tmp.h, tmp.frame(d_depth[j], d_rgb[j], K), Ts[j], None, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        R.rf_virtual_depth(tmp.h, tmp.frame(d_depth[i], d_rgb[i], K), Ts[i], 0, out, stream)
        b.record(stream)
        b.synchronize()
        t1 = time.perf_counter()
        tmp.sync(stream)
        if t < 0:
            continue
        total_ms.append(1000.0 * (t1 - t0))
        cast_ms.append(a.elapsed_time(b))
        zero = d_depth[i] == 0
        holes.append(int(zero.sum().item()))
        filled.append(int((zero & (out != far)).sum().item()))
    tmp.close()
    return {"window": n_window, "targets": n_targets, "ms_per_filled_frame": statistics.mean(total_ms),
            "raycast_ms": statistics.mean(cast_ms), "holes_per_frame": statistics.mean(holes),
            "filled_fraction": sum(filled) / max(1, sum(holes)),
            "note": "temporary model of the 10 frames starting at the target (ground-truth poses), rebuilt per "
                    "target; holes = the frames' zero pixels (5 % edge dropout)"}


def run_batch(R, frames, K, cam, dev, stream, flush, args, storage=0):
    """S streams (one volume each, the same rendered sequence) processed in
    lockstep batches through rf_batch_process: aggregate frames/s and the
    per-batch latency (every frame of a batch completes at the batch's end)."""
    import torch
    S = args.batch_streams
    vols = [R.Volume(n_buckets=1 << 18, max_blocks=60_000, max_width=cam.width, max_height=cam.height,
                     voxel_size=VOXEL, trunc=TAU, storage=storage) for _ in range(S)]
    batch = R.Batch(vols)
    n = min(len(frames), args.warmup + args.batch_steps)
    d_depth = [torch.from_numpy(f[0].astype(np.int32)).to(dev).to(torch.uint16).contiguous() for f in frames[:n]]
    d_rgb = [torch.from_numpy(f[1]).to(dev).contiguous() for f in frames[:n]]
    T = [torch.as_tensor(frames[0][2], device=dev).contiguous() for _ in range(S)]
    Tn = [torch.empty(4, 4, dtype=torch.float64, device=dev) for _ in range(S)]

    def step(i):
        fr = [vols[k].frame(d_depth[i], d_rgb[i], K) for k in range(S)]
        batch.process(fr, T, Tn, None, stream)

    for i in range(args.warmup):
        step(i)
        T, Tn = Tn, T
    torch.cuda.synchronize()
    ms = []
    for i in range(args.warmup, n):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(i)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        T, Tn = Tn, T
    for v in vols:
        v.sync()
    batch.close()
    for v in vols:
        v.close()
    return {"streams": S, "storage": "fp16" if storage else "fp32",
            "workload": "static room 640x480 per stream (one volume each, voxel 1 cm)",
            "frames_per_s": S * len(ms) / (sum(ms) / 1000.0), "batches": len(ms),
            "batch_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                         "mean": statistics.mean(ms)},
            "note": "lockstep batches via rf_batch_process; a frame's latency is its batch's time"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=290)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--batch-streams", type=int, default=32)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--vd-frames", type=int, default=20)
    ap.add_argument("--precision-frames", type=int, default=24)
    ap.add_argument("--only", choices=["all", "precision"], default="all",
                    help="precision: run only the precision section (e.g. its full 900-frame sequence)")
    ap.add_argument("--serving-streams", type=int, default=32)
    ap.add_argument("--serving-seconds", type=float, default=1.0)
    ap.add_argument("--serving-rates", type=float, nargs="*", default=[30.0, 120.0, 360.0])
    ap.add_argument("--serving-clip", type=int, default=10)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    workers = max(1, min(16, (os.cpu_count() or 1) // world))  # ranks share the host cores
    pframes, porder = [], []
    if rank == 0 and args.precision_frames > 0:
        nr = min(args.precision_frames, PRECISION_RENDERED)
        porder = frame_order(nr, args.precision_frames)
        with mp.get_context("spawn").Pool(workers) as pool:
            pframes = pool.map(_render_precision, [(i, nr) for i in range(nr)], chunksize=1)
    if args.only == "precision":
        import torch
        torch.cuda.set_device(local)
        from paper_1905_02082_gb300 import build as B
        B.build()
        import paper_1905_02082_gb300.refusion as R
        dev = torch.device("cuda", local)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        prec = run_precision(R, pframes, porder, dev, torch.cuda.current_stream(), flush, min(10, args.warmup))
        print(json.dumps({"precision": prec}))
        return
    n_frames = min(args.warmup + args.steps, MAX_RENDERED)
    order = frame_order(n_frames, args.warmup + args.steps)
    frames = make_frames(seed=rank_seed(rank), n=n_frames, workers=workers)
    splan = serving_plan(args.serving_streams) if args.serving_streams > 0 and rank == 0 else []
    clips = render_serving_clips(splan, args.serving_clip, workers) if splan else []
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1905_02082_gb300 import build as B
    B.build()
    import paper_1905_02082_gb300.refusion as R

    from synth.scenes import CAM_VGA as cam
    K = R.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy)
    dev = torch.device("cuda", local)
    d_depth = [torch.from_numpy(f[0].astype(np.int32)).to(dev).to(torch.uint16).contiguous() for f in frames]
    d_rgb = [torch.from_numpy(f[1]).to(dev).contiguous() for f in frames]
    T0 = torch.as_tensor(frames[0][2], device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    vol = R.Volume(n_buckets=N_BUCKETS, max_blocks=MAX_BLOCKS, max_width=cam.width, max_height=cam.height,
                   voxel_size=VOXEL, trunc=TAU)
    vol.set_profiling(True)
    T = T0.clone()
    Tn = torch.empty_like(T)
    mask = torch.empty(cam.height, cam.width, dtype=torch.uint8, device=dev)
    for w in range(args.warmup):
        i = order[w]
        fr = vol.frame(d_depth[i], d_rgb[i], K)
        R.rf_process_frame(vol.h, fr, T, Tn, mask, None, stream)
        T, Tn = Tn, T
    vol.sync()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    profs, infos, errs = [], [], []
    info_dev = torch.zeros(ctypes.sizeof(R.rf_track_info), dtype=torch.uint8, device=dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        i = order[args.warmup + k]
        flush.zero_()  # L2 flush between steps, outside the step's events
        fr = vol.frame(d_depth[i], d_rgb[i], K)
        ev[k][0].record(stream)
        R.rf_process_frame(vol.h, fr, T, Tn, mask, info_dev, stream)
        ev[k][1].record(stream)
        T, Tn = Tn, T
        profs.append(vol.profile(stream))  # synchronises; reads this frame's events
        infos.append(R.Volume.info_of(info_dev))
        errs.append(float(np.linalg.norm(T.cpu().numpy()[:3, 3] - frames[i][2][:3, 3])))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    vol.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    timed_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = job_throughput(world, args.steps, timed_ms)

    peak, peak_kind = measured_peaks()
    # integration kernel (the HBM byte mover): 18 B per updated voxel (9 read, 9
    # written), 4.5 KB per new block, plus the masked depth it reads (2 B/pixel)
    kern_ms = [p.integrate_kernel_ms for p in profs]
    upd = [p.updated_voxels for p in profs]
    newb = [p.new_blocks for p in profs]
    npx = cam.width * cam.height
    bytes_per = [18 * u + 9 * 512 * nb + 2 * npx for u, nb in zip(upd, newb)]
    int_ms = sum(kern_ms) / len(kern_ms)
    ach = (sum(bytes_per) / len(bytes_per)) / (int_ms / 1000.0) / 1e9
    # registration kernel: its algorithmic bytes per launch (oracle-counted
    # footprint of this workload) over the mean of both registrations' launches
    foot = json.load(open(FOOTPRINT))
    reg_bytes = foot["mean_bytes_fp32"]
    reg_launch_ms = statistics.mean((pr.track_ms[0] + pr.track_ms[1]) / 2.0 for pr in profs)
    reg_gbs = reg_bytes / (reg_launch_ms / 1000.0) / 1e9
    # the ALU view of the same kernel (an estimate: hand-counted flops per sample)
    p = vol.params
    npix = [((cam.width + p.lm_strides[l] - 1) // p.lm_strides[l]) * ((cam.height + p.lm_strides[l] - 1) //
                                                                          p.lm_strides[l]) for l in range(3)]
    reg_ms = [pr.track_ms[1] for pr in profs]  # the second registration (its info is returned)
    reg_flops = [FLOPS_PER_SAMPLE * sum(inf.level_evals[l] * npix[l] for l in range(3)) for inf in infos]
    reg_tflops = (sum(reg_flops) / len(reg_flops)) / (sum(reg_ms) / len(reg_ms) / 1000.0) / 1e12
    roof_reg = {"bound": "hbm", "kernel": "k_register (one registration: 3 levels, all LM evaluations)",
                "achieved": reg_gbs, "peak": peak, "unit": "GB/s", "frac": reg_gbs / peak,
                "traffic": REGISTER_DRAM_BYTES,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                                   "(profiles/k_register_static_640x480.md)" if REGISTER_DRAM_BYTES is not None else
                                   "null: the kernel changed since its last ncu capture"),
                "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs), of " + peak_kind,
                "bytes_per_launch": reg_bytes,
                "bytes_source": "oracle-counted footprint: 5 B per pixel (+1 B mask) + 8 B per distinct voxel read + "
                                "8 B per distinct block probed (tests/golden/track_footprint_static.json)",
                "launch_ms": reg_launch_ms, "launches_per_frame": 2,
                "note": "latency-bound: a dependent chain of LM evaluations, each a grid-wide reduction",
                "alu_estimate": {"achieved": reg_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": reg_tflops / FP32_PEAK_TFLOPS,
                                 "note": f"estimate: {FLOPS_PER_SAMPLE} hand-counted FP32 flops per sample; peak "
                                         "derived as 152 SMs x 128 lanes x 2 flops x 2.07 GHz"}}
    roof_int = {"bound": "hbm", "kernel": "k_integrate (per-voxel TSDF/colour update)",
                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": INTEGRATE_DRAM_BYTES,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                                   "(profiles/k_integrate_static_640x480.md)" if INTEGRATE_DRAM_BYTES is not None else
                                   "null: the kernel changed since its last ncu capture"),
                "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs), of " + peak_kind,
                "bytes_per_launch": statistics.mean(bytes_per),
                "bytes_source": "18 B per updated voxel + 4.5 KB per new block + 2 B per pixel of masked depth",
                "launch_ms": int_ms, "launches_per_frame": 1}
    # the dominant kernel by device time per frame carries the headline roofline
    dominant = roof_reg if 2 * reg_launch_ms >= int_ms else roof_int
    # whole frame: input once, the model reads of both registrations, the mask
    # written, the integration's read-modify-write
    model_reads = reg_bytes - 5 * npx - 0.5 * npx  # mean registration minus its pixel reads
    frame_bytes = [b + 5 * npx + 2 * model_reads + npx for b in bytes_per]
    frame_gbs = (sum(frame_bytes) / len(frame_bytes)) / (statistics.mean(step_ms) / 1000.0) / 1e9
    stage = {k: statistics.mean(getattr(p, k) if k != "track_ms" else p.track_ms[0] + p.track_ms[1] for p in profs)
             for k in ("frame_ms", "track_ms", "mask_ms", "integrate_ms", "integrate_kernel_ms")}

    # end to end through the host-buffer entry point (pinned host inputs)
    e2e = None
    n_e2e = min(args.e2e_steps, args.steps)
    if n_e2e > 0:
        vol2 = R.Volume(n_buckets=N_BUCKETS, max_blocks=MAX_BLOCKS, max_width=cam.width, max_height=cam.height,
                        voxel_size=VOXEL, trunc=TAU)
        h_depth = [torch.from_numpy(f[0]).pin_memory() for f in frames]
        h_rgb = [torch.from_numpy(f[1]).pin_memory() for f in frames]
        Th = np.array(frames[0][2], dtype=np.float64)  # a copy: updated in place below
        To = np.zeros((4, 4))
        for w in range(args.warmup):
            i = order[w]
            R.rf_process_frame_host(vol2.h, h_depth[i].numpy(), h_rgb[i].numpy(), [K.fx, K.fy, K.cx, K.cy], Th, To,
                                    None, stream)
            Th = To.copy()
        torch.cuda.synchronize()
        hd = [h_depth[order[args.warmup + k]].numpy() for k in range(n_e2e)]
        hc = [h_rgb[order[args.warmup + k]].numpy() for k in range(n_e2e)]
        intr = [K.fx, K.fy, K.cx, K.cy]
        gc.collect()
        gc.disable()  # host-clocked: keep collector pauses out of the region
        t0 = time.perf_counter()
        for k in range(n_e2e):
            R.rf_process_frame_host(vol2.h, hd[k], hc[k], intr, Th, To, None, stream)
            Th[...] = To
        e2e_s = time.perf_counter() - t0
        gc.enable()
        e2e = {"value": world * n_e2e / e2e_s, "unit": "frames/s",
               "h2d_bytes_per_step": cam.width * cam.height * 5 + 128, "d2h_bytes_per_step": 128,
               "steps": n_e2e, "api": "rf_process_frame_host"}
        vol2.close()

    # kernels of this library per whole frame (graph nodes): one cooperative
    # launch per registration (2), mask: seeds, erosion, flood fill,
    # dilation (4), integration: frustum search, cull, update, neighbour
    # tables (4)
    launches_per_frame = 2 + 4 + 4
    batch = None
    batch_fp16 = None
    if args.batch_streams > 0:
        batch = run_batch(R, frames, K, cam, dev, stream, flush, args)
        batch_fp16 = run_batch(R, frames, K, cam, dev, stream, flush, args, storage=R.STORAGE_FP16)
    single_fp16 = run_single(R, frames, K, cam, dev, stream, flush, args, storage=R.STORAGE_FP16)
    virtual_depth = run_virtual_depth(R, frames, K, cam, dev, stream, args) if args.vd_frames > 0 else None
    serving = run_serving(R, splan, clips, args) if splan else None
    precision = run_precision(R, pframes, porder, dev, stream, flush, 4) if pframes else None

    if rank == 0:
        st = vol.stats()
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": timed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "static room 640x480 (fx=fy=525), voxel 1 cm, tau 0.1 m, 2^20 buckets, "
                                   "track+mask+re-track+integrate per frame",
                       "global_batch": world, "seq_len": 1, "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between steps, outside the step events"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "mean": statistics.mean(step_ms)},
            "stages_ms": stage,
            "e2e": e2e,
            "gpu_launches": launches_per_frame * args.steps,
            "gpu_launches_per_frame": launches_per_frame,
            "clocks": clk,
            "roofline": dominant,
            "roofline_integrate": roof_int,
            "frame_hbm": {"achieved": frame_gbs, "peak": peak, "unit": "GB/s", "frac": frame_gbs / peak,
                          "bytes_per_frame": statistics.mean(frame_bytes),
                          "bytes_source": "5 B per pixel input + both registrations' model reads + 1 B per pixel "
                                          "mask + the integration's bytes"},
            "cpu_baseline": cpu,
            "batch": batch,
            "batch_fp16": batch_fp16,
            "single_fp16": single_fp16,
            "tracking": {"rmse_m": float(np.sqrt(np.mean(np.square(errs)))), "max_m": float(np.max(errs)),
                         "note": "free-running pose vs the ground truth of the timed frames (no loop closure)"},
            "work": {"updated_voxels": statistics.mean(upd), "new_blocks": statistics.mean(newb),
                     "candidates": statistics.mean(p.candidates for p in profs), "blocks": st.n_blocks,
                     "guard_pixels": statistics.mean(p.guard_pixels for p in profs)},
            "roofline_register": roof_reg,
            "wall_s_timed": wall,
            "virtual_depth": virtual_depth,
            "precision": precision,
            "serving": serving,
        }
        print(json.dumps(line))
    vol.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
