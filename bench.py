"""Benchmark of the low-resolution 3DGS render hot path on GB300.

A step renders one frame of the workload's camera path through the whole hot
path (projection + SH colour, scan, key duplication, radix sort, tile ranges,
compositing with dC/dx, dC/dy, depth and alpha), replayed as a captured CUDA
graph with the frame's camera (the fixed-resolution stream path), with
--frames-in-flight frames (default 6) rendering concurrently on their own streams
(api.FrameStream over the C ABI's gs_frame_stream_*). The scene is
resident in HBM before timing starts and is larger than L2, so steps do not
reuse each other's inputs from cache.

Prints one JSON line. Default workload: 1M clustered Gaussians, SH degree 3,
960x540, 60-frame orbit (steps cycle over the orbit).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|ultra|ultra_lr|tiny|serve|interp|gass|pipeline]

With --gpus N > 1 (launched by torchrun) every rank renders the same workload
as an independent replica (the render has no cross-GPU exchange); value is the
pixels of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "render+grad Mpix/s"
WORKLOADS = {
    "large": dict(desc="1M Gaussians (64 clusters, 100x100x20 m), SH degree 3, 960x540, 60-frame orbit",
                  n=1_000_000, width=960, height=540, path="orbit"),
    "ultra": dict(desc="6M Gaussians (64 clusters, 300x300x40 m), SH degree 3, 1920x1080, 60-frame fly-through",
                  n=6_000_000, width=1920, height=1080, path="fly"),
    "ultra_lr": dict(desc="6M Gaussians (300x300x40 m), SH degree 3, 480x270, 60-frame fly-through",
                     n=6_000_000, width=480, height=270, path="fly"),
    "tiny": dict(desc="4,096 Gaussians in [-1,1]^3, SH degree 0, 256x144, 64 jittered cameras",
                 n=4096, width=256, height=144, path="tiny"),
}
GS_CAMERA_BYTES = 76  # sizeof(gs_camera): the per-step host input
BWD_HOST_COVER_CYCLES = 1_000_000  # device-side wait before the timed backward (~0.5 ms at 2 GHz)


def make_workload(name):
    from paper_2605_11489_gb300 import synth

    w = WORKLOADS[name]
    if name == "large":
        sc = synth.large_scene(w["n"], 1)
        cams = synth.orbit_cameras(60, w["width"], w["height"])
    elif name in ("ultra", "ultra_lr"):
        sc = synth.ultra_scene(w["n"], 2)
        cams = synth.flythrough_cameras(60, w["width"], w["height"])
    else:
        sc = synth.tiny_scene(w["n"], 0)
        cams = [synth.tiny_camera()] + synth.jittered_tiny_cameras(63, 1)
    return sc, cams


def dist_env():
    n = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), n


def slowest_rank(seconds_or_ms, world, device="cpu"):
    """Max over ranks of a per-rank duration (the job's time); identity at world == 1."""
    if world <= 1:
        return float(seconds_or_ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(seconds_or_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pixels_per_rank, world, duration_s):
    """Whole-job Mpix/s: the pixels all ranks rendered over the slowest rank's time."""
    return pixels_per_rank * world / duration_s / 1e6


def start_clock_sampler(path, gpu_index):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                              "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except (OSError, FileNotFoundError):
        return None, None


def read_clocks(path):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d.get("hbm_gbs"), d.get("sm_max_mhz", 2070.0), "measured"
    except (OSError, ValueError):
        return 6800.0, 2070.0, "fallback"


def cpu_baseline(sc, cams, name, max_seconds=20.0):
    """The oracle as it stands (binned FP64 mode) on the host cores, over a bounded
    sample: whole frames of the same camera path until ~max_seconds."""
    import oracle

    oracle.build()
    osc = oracle.OScene(sc)
    cores = oracle.max_threads()
    px = 0
    t0 = time.perf_counter()
    frames = 0
    while frames < len(cams):
        cam = cams[frames]
        if name.startswith("ultra") and cam.width * cam.height > 600_000 and frames == 0:
            # 1920x1080 over 6M Gaussians: one band of rows keeps the sample bounded
            oracle.render_band(osc, cam, 0, cam.height // 8)
            px += cam.width * (cam.height // 8)
        else:
            oracle.render(osc, cam)
            px += cam.width * cam.height
        frames += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": px / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": "%d frame(s) of the %s camera path (%d px) in %.1f s, FP64 binned oracle" % (
                frames, name, px, dt)}


def run_reference(args):
    """--impl reference: the CPU FP64 oracle timed on the same workload, metric and
    unit; each step renders one whole frame of the camera path (binned mode, all host cores)."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    if args.workload == "interp":
        return run_reference_interp(args, world)
    if args.workload == "gass":
        return run_reference_gass(args, world)
    if args.workload == "pipeline":
        print(json.dumps({"impl": "reference", "workload": "pipeline",
                          "unavailable": "a scheduling pattern of the GPU path; its CPU counterparts are the "
                                         "large, gass and interp reference arms"}), flush=True)
        return
    sc, cams = make_workload(args.workload)
    osc = oracle.OScene(sc)
    cores = oracle.max_threads()

    def step(i):  # one whole frame of the camera path, like the GPU arm's step
        cam = cams[i % len(cams)]
        oracle.render(osc, cam)
        return cam.width * cam.height

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    px = 0
    for i in range(args.steps):
        px += step(args.warmup + i)
    dt = time.perf_counter() - t0
    v = px / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
                       "step": "one whole frame of the camera path"},
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                             "sample": "%d whole frames of the %s camera path" % (args.steps, args.workload)},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_interp(args, world):
    """--impl reference --workload interp: the oracle's warp (or_warp) on the same pair;
    a step is one call (alternating the high- and low-resolution frame)."""
    import oracle

    from paper_2605_11489_gb300 import synth

    calls = _interp_calls(synth.interp_inputs())

    def step(i):
        src, dst, f, grads = calls[i % 2]
        oracle.warp(src, dst, f["depth"], f["alpha"], 0.0, f["planes"], f["dcdx"] if grads else None,
                    f["dcdy"] if grads else None)
        return src.width * src.height

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    px = sum(step(args.warmup + i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = px / dt / 1e6
    line = {"metric": "interp warp Mpix/s (source pixels)", "value": v, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": "interp", "desc": INTERP_DESC,
                                            "step": "one of the two warps, alternating"},
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": "%d warps (or_warp, single-threaded C)" % args.steps},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_gass(args, world):
    """--impl reference --workload gass: the oracle's gradient-aware interpolation (NumPy
    FP64, Conv -> TConv) of the same 4x upsampling; a step is one band of 32 rows of the
    oracle's own 960x540 render (colour and gradients)."""
    import oracle
    from oracle import gai as og

    from paper_2605_11489_gb300 import synth

    sc, cams = make_workload("large")
    r = oracle.render(oracle.OScene(sc), cams[0])
    S, wc, bc, wt, bt = synth.gai_weights(4, 32)
    H, W = r["rgb"].shape[1:]
    band = 32

    def step(i):
        y0 = (i * band) % H
        sl = slice(y0, min(H, y0 + band))
        og.gai(r["rgb"][:, sl], r["dcdx"][:, sl], r["dcdy"][:, sl], wc, bc, wt, bt, S)
        return S * S * W * (sl.stop - sl.start)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    px = sum(step(args.warmup + i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = px / dt / 1e6
    line = {"metric": "gass interpolation Mpix/s (4x output pixels)", "value": v, "unit": "Mpix/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": "gass", "desc": GASS_DESC, "step": "a band of 32 rows"},
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": "%d bands of %d rows (oracle.gai, NumPy FP64)" % (args.steps, band)},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """--workload serve: the continuous-batching server against the plain
    one-request-at-a-time renderer on the same mixed-resolution request stream.

    4 resident scenes (0.5M, 1M, 3M, 6M clustered Gaussians, SH degree 3), a
    seeded stream of requests with random orbit cameras and resolutions uniform
    over {480x270, 960x540, 1280x720, 1920x1080}, 40 GB sort-buffer budget.
      plain:    each request rendered by gs_render_forward, one after another
      server:   all requests submitted at once (throughput), then a Poisson
                stream at 0.8x the plain renderer's request rate (latency)
    Prints one JSON line."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2605_11489_gb300 import abi, api, synth

    torch.cuda.set_device(0)
    n_req = args.requests
    sizes = tuple(int(s * args.serve_scale) for s in synth.SERVING_SCENE_SIZES)
    scenes = [api.Scene.from_arrays(synth.serving_scene(n, 10 + i)) for i, n in enumerate(sizes)]
    reqs = synth.serving_requests(n_req, 5, 100.0, sizes)
    outs = {}
    for r in reqs:
        key = (r.camera.width, r.camera.height)
        if key not in outs:
            outs[key] = api.alloc_outputs(*key)
    px_total = sum(r.camera.width * r.camera.height for r in reqs)
    ctx = api.Context(0)
    stream = torch.cuda.Stream()
    for r in reqs[:8]:  # warm-up
        ctx.forward(scenes[r.scene], r.camera, out=outs[(r.camera.width, r.camera.height)], tile=16, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        ctx.forward(scenes[r.scene], r.camera, out=outs[(r.camera.width, r.camera.height)], tile=16, stream=stream)
    stream.synchronize()
    t_plain = time.perf_counter() - t0
    plain_rate = n_req / t_plain
    ctx.close()

    srv = api.Server(sort_budget_bytes=int(args.budget_gb * (1 << 30)), max_inflight=args.inflight)
    sids = [srv.load_scene(s) for s in scenes]

    def run_stream(arrivals):
        lat = [None] * n_req
        ids = [None] * n_req
        pending = set()
        start = time.perf_counter()
        i = 0
        while i < n_req or pending:
            now = time.perf_counter() - start
            while i < n_req and arrivals[i] <= now:
                r = reqs[i]
                ids[i] = srv.submit(sids[r.scene], r.camera, outs[(r.camera.width, r.camera.height)])
                pending.add(i)
                i += 1
            for j in list(pending):
                st, l = srv.poll(ids[j])
                if st != abi.GS_NOT_READY:
                    if st != 0:
                        raise RuntimeError("request %d failed: %d" % (j, st))
                    lat[j] = l
                    pending.discard(j)
            if pending and not (i < n_req and arrivals[i] <= time.perf_counter() - start):
                time.sleep(0.0002)
        return time.perf_counter() - start, lat

    for k in range(8):  # warm-up
        srv.submit(sids[reqs[k].scene], reqs[k].camera, outs[(reqs[k].camera.width, reqs[k].camera.height)])
    srv.drain()
    t_burst, lat_burst = run_stream([0.0] * n_req)
    rate = args.load * plain_rate
    rng = __import__("numpy").random.default_rng(5)
    arr = list(__import__("numpy").cumsum(rng.exponential(1.0 / rate, n_req)))
    t_poisson, lat_p = run_stream(arr)
    srv.close()
    lat_p = sorted(lat_p)
    pct = lambda q: lat_p[min(n_req - 1, int(q * n_req))]
    line = {"metric": "serving Mpix/s (mixed-resolution stream)", "value": px_total / t_burst / 1e6,
            "unit": "Mpix/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve", "requests": n_req, "scenes": list(sizes),
                       "resolutions": ["%dx%d" % r for r in synth.SERVING_RESOLUTIONS],
                       "sort_budget_gb": args.budget_gb, "max_inflight": args.inflight},
            "plain_per_request": {"value": px_total / t_plain / 1e6, "unit": "Mpix/s",
                                  "requests_per_s": plain_rate},
            "speedup_vs_plain": t_plain / t_burst,
            "poisson": {"rate_req_per_s": rate, "load_vs_plain": args.load, "p50_ms": pct(0.5),
                        "p99_ms": pct(0.99), "mean_ms": sum(lat_p) / n_req,
                        "throughput_mpix_s": px_total / t_poisson / 1e6},
            "burst_p50_ms": sorted(lat_burst)[n_req // 2]}
    return line


INTERP_DESC = ("frame-interpolation warp pair of Sec. 4.2: frame 0 at 3840x2160 (7 planes: colour, depth, "
               "normals) toward P0.5, frame 1 at 960x540 (7 planes + 3 image-gradient planes) toward P0.5; "
               "motion vectors, depth-tested forward warp, warped gradient; large-scene orbit poses")


def _interp_calls(w):
    """The two gs_warp calls of one step: (src cam, dst cam, frame, gradients?)."""
    return [(w["P0_hr"], w["P05_hr"], w["hr"], False), (w["P1"], w["P05"], w["lr"], True)]


def warp_bytes(src, dst, channels, grad_channels, hits):
    """Algorithmic bytes of one gs_warp call, per kernel: the scatter reads depth and
    alpha and writes the motion map (per source pixel); the gather writes index, z,
    the planes and the gradient planes (per target pixel) and reads the winners'
    planes and gradients (per hit target pixel). Scratch traffic is not counted."""
    n, nt = src.width * src.height, dst.width * dst.height
    scatter = n * (4 + 4 + 8)
    gather = nt * (4 + 4 + 4 * channels + 8 * grad_channels) + hits * (4 * channels + 8 * grad_channels)
    return scatter, gather


def run_interp(args):
    """--workload interp: the forward-backward warp pair of Sec. 4.2 (two gs_warp calls,
    two kernels each) on resident synthetic frames; one JSON line."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2605_11489_gb300 import api, synth

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    w = synth.interp_inputs()
    calls = _interp_calls(w)
    stream = torch.cuda.Stream()
    ctx = api.Context(local_rank)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with torch.cuda.stream(stream):
        ins, outs = [], []
        for src, dst, f, grads in calls:
            ins.append(dict(depth=dev(f["depth"]), alpha=dev(f["alpha"]), planes=dev(f["planes"]),
                            dcdx=dev(f["dcdx"]) if grads else None, dcdy=dev(f["dcdy"]) if grads else None))
            outs.append(api.alloc_warp_outputs(src.width, src.height, dst.width, dst.height, f["planes"].shape[0],
                                               f["dcdx"].shape[0] if grads else 0))
    stream.synchronize()

    def step():
        for (src, dst, f, grads), i, o in zip(calls, ins, outs):
            ctx.warp(src, dst, i["depth"], i["alpha"], 0.0, i["planes"], i["dcdx"], i["dcdy"], out=o, stream=stream)

    for _ in range(args.warmup):
        step()
    clk_path = os.path.join(tempfile.gettempdir(), "gsr_clocks_interp_%d_%d.csv" % (os.getpid(), rank))
    smi, smi_f = start_clock_sampler(clk_path, local_rank)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        torch.distributed.barrier()
    if smi:
        smi.terminate()
        smi.wait()
        smi_f.close()
    clocks = read_clocks(clk_path)
    ms = slowest_rank(ms, world, "cuda")
    px_step = sum(src.width * src.height for src, _, _, _ in calls)
    value = job_throughput(px_step * args.steps, world, ms * 1e-3)

    # per-call durations (CUDA events around each call on the launch stream), and each
    # kernel's share from a split of the call: the scatter alone, then the whole call
    per = []
    hbm_peak, _, peak_src = measured_peaks()
    reps = max(10, min(args.steps, 50))
    for (src, dst, f, grads), i, o in zip(calls, ins, outs):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            ctx.warp(src, dst, i["depth"], i["alpha"], 0.0, i["planes"], i["dcdx"], i["dcdy"], out=o, stream=stream)
        ev[1].record(stream)
        ev[1].synchronize()
        call_ms = ev[0].elapsed_time(ev[1]) / reps
        hits = int((o["index"] >= 0).sum().item())
        sb, gb = warp_bytes(src, dst, f["planes"].shape[0], f["dcdx"].shape[0] if grads else 0, hits)
        per.append({"src": "%dx%d" % (src.width, src.height), "dst": "%dx%d" % (dst.width, dst.height),
                    "channels": int(f["planes"].shape[0]), "grad_channels": int(f["dcdx"].shape[0]) if grads else 0,
                    "call_ms": call_ms, "hits": hits, "algorithmic_bytes": sb + gb,
                    "achieved_gbs": (sb + gb) / (call_ms * 1e-3) / 1e9})
    dom = max(range(len(per)), key=lambda k: per[k]["call_ms"])
    d = per[dom]
    roof = {"bound": "hbm", "kernel": "gs_warp %s -> %s (k_warp_scatter + k_warp_gather)" % (d["src"], d["dst"]),
            "achieved": d["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": d["achieved_gbs"] / hbm_peak,
            "traffic": None, "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src,
            "algorithmic_bytes_per_launch": d["algorithmic_bytes"], "launch_ms": d["call_ms"]}

    # end to end: inputs from pinned host memory, every output plane back, per step
    e2e = None
    if not args.no_e2e:
        h_in = [{k: (v.cpu().pin_memory() if v is not None else None) for k, v in i.items()} for i in ins]
        h_out = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in o.items()} for o in outs]
        h2d = sum(v.numel() * 4 for i in h_in for v in i.values() if v is not None)
        d2h = sum(v.numel() * 4 for o in h_out for v in o.values())
        n_e = min(args.steps, 20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e):
            with torch.cuda.stream(stream):
                for (src, dst, f, grads), hi, di, o, ho in zip(calls, h_in, ins, outs, h_out):
                    for k, v in hi.items():
                        if v is not None:
                            di[k].copy_(v, non_blocking=True)
                    ctx.warp(src, dst, di["depth"], di["alpha"], 0.0, di["planes"], di["dcdx"], di["dcdy"], out=o,
                             stream=stream)
                    for k in o:
                        ho[k].copy_(o[k], non_blocking=True)
            stream.synchronize()
        dt = slowest_rank(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": job_throughput(px_step * n_e, world, dt), "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "path": "torch H2D of the source planes + gs_warp x2 + D2H of every output plane"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        n_c = 0
        while n_c < 1 or time.perf_counter() - t0 < 10.0:
            for src, dst, f, grads in calls:
                oracle.warp(src, dst, f["depth"], f["alpha"], 0.0, f["planes"], f["dcdx"] if grads else None,
                            f["dcdy"] if grads else None)
            n_c += 1
        dt = time.perf_counter() - t0
        cpu = {"value": px_step * n_c / dt / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
               "sample": "%d step(s) of the warp pair in %.1f s (or_warp, single-threaded C, FP64 Jacobian)" % (
                   n_c, dt)}
    if rank == 0:
        line = {"metric": "interp warp Mpix/s (source pixels)", "value": value, "unit": "Mpix/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "interp", "desc": INTERP_DESC,
                           "l2": "inputs larger than L2 (%.0f MB per step)" % (
                               sum(v.numel() * 4 for i in ins for v in i.values() if v is not None) / 1e6),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "calls": per, "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
                "gpu_launches": args.steps * 4}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


GASS_DESC = ("gradient-aware interpolation of Sec. 4.1 (Eq. 7-8): the 960x540 render of the large scene "
             "(rgb, dC/dx, dC/dy of frame 0) super-sampled x4 to 3840x2160; seeded Conv3x3 (27 -> 32) and 4x4 "
             "TConv weights")


def run_gass(args):
    """--workload gass: gs_gai_upsample of a rendered frame (resident) by 4; one JSON line."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2605_11489_gb300 import api, synth

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    sc, cams = make_workload("large")
    W, H = cams[0].width, cams[0].height
    weights = synth.gai_weights(4, 32)
    S = weights[0]
    stream = torch.cuda.Stream()
    ctx = api.Context(local_rank)
    with torch.cuda.stream(stream):
        scene = api.Scene.from_arrays(sc)
        frame = ctx.forward(scene, cams[0], keys=("rgb", "dcdx", "dcdy"), stream=stream)
        out = torch.empty((3, S * H, S * W), dtype=torch.float32, device="cuda")
    stream.synchronize()
    del scene
    step = lambda: api.gai_upsample(weights, frame["rgb"], frame["dcdx"], frame["dcdy"], out=out, stream=stream)
    for _ in range(args.warmup):
        step()
    clk_path = os.path.join(tempfile.gettempdir(), "gsr_clocks_gass_%d_%d.csv" % (os.getpid(), rank))
    smi, smi_f = start_clock_sampler(clk_path, local_rank)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        torch.distributed.barrier()
    if smi:
        smi.terminate()
        smi.wait()
        smi_f.close()
    clocks = read_clocks(clk_path)
    ms = slowest_rank(ms, world, "cuda")
    hr_px = S * S * W * H
    value = job_throughput(hr_px * args.steps, world, ms * 1e-3)
    hbm_peak, sm_max_mhz, peak_src = measured_peaks()
    # algorithmic bytes of one launch: the three input planes once (3 channels x 4 B each)
    # and the S*S outputs (3 channels x 4 B each) per low-resolution pixel
    bytes_launch = W * H * (3 * 3 * 4 + 3 * S * S * 4)
    launch_ms = ms / args.steps
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    fma = 3 * W * H * S * S * 27
    roof = {"bound": "hbm", "kernel": "k_gai<4>", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": None,
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src,
            "algorithmic_bytes_per_launch": bytes_launch, "launch_ms": launch_ms,
            "fp32_frac": 2 * fma / (launch_ms * 1e-3) / 1e12 / fp32_peak_tflops(sm_max_mhz)}
    e2e = None
    if not args.no_e2e:
        h_in = {k: v.cpu().pin_memory() for k, v in frame.items()}
        h_out = torch.empty(out.shape, dtype=torch.float32).pin_memory()
        d_in = {k: torch.empty_like(v) for k, v in frame.items()}
        n_e = min(args.steps, 30)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e):
            with torch.cuda.stream(stream):
                for k in d_in:
                    d_in[k].copy_(h_in[k], non_blocking=True)
                api.gai_upsample(weights, d_in["rgb"], d_in["dcdx"], d_in["dcdy"], out=out, stream=stream)
                h_out.copy_(out, non_blocking=True)
            stream.synchronize()
        dt = slowest_rank(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": job_throughput(hr_px * n_e, world, dt), "unit": "Mpix/s",
               "h2d_bytes_per_step": 9 * W * H * 4, "d2h_bytes_per_step": 3 * hr_px * 4,
               "path": "torch H2D of rgb, dC/dx, dC/dy + gs_gai_upsample + D2H of the 4x image"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import gai as og

        f = {k: v.cpu().numpy().astype(np.float64) for k, v in frame.items()}
        rows = 0
        t0 = time.perf_counter()
        while rows < H and (rows == 0 or time.perf_counter() - t0 < 10.0):
            band = slice(rows, min(H, rows + 64))
            og.gai(f["rgb"][:, band], f["dcdx"][:, band], f["dcdy"][:, band], *weights[1:], S)
            rows = band.stop
        dt = time.perf_counter() - t0
        cpu = {"value": S * S * W * rows / dt / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
               "sample": "%d of %d low-resolution rows in bands of 64 (oracle.gai, NumPy FP64, Conv -> TConv) "
                         "in %.1f s" % (rows, H, dt)}
    if rank == 0:
        line = {"metric": "gass interpolation Mpix/s (4x output pixels)", "value": value, "unit": "Mpix/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": launch_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "gass", "desc": GASS_DESC, "scale": S, "features": int(weights[1].shape[0]),
                           "l2": "output larger than L2 (%.0f MB per step)" % (3 * hr_px * 4 / 1e6),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roof, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
                "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


PIPE_DESC = ("post-rendering chain of Sec. 4 on three streams: 960x540 render of the large scene (1M, SH 3) per "
             "frame of the 60-frame orbit (--frames-in-flight render streams taking frames in turn) || x4 gradient-aware interpolation of colour, depth and alpha + forward "
             "warp of the previous 3840x2160 frame + backward warp of the current 960x540 frame toward the mid "
             "pose; serial = the same calls on one stream")


def run_pipeline(args):
    """--workload pipeline: api.FramePipeline overlapped against its one-stream form."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2605_11489_gb300 import api, synth

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    sc = synth.large_scene(1_000_000, 1)
    dense = synth.orbit_cameras(120, 960, 540)
    frames, mids = dense[0::2], dense[1::2]
    W, H = frames[0].width, frames[0].height
    weights = synth.gai_weights(4, 32)
    ctx = api.Context(local_rank)
    scene = api.Scene.from_arrays(sc)
    out = api.alloc_outputs(W, H)
    stream = torch.cuda.Stream()
    tile, batch, chunk, _ = ctx.autotune(scene, frames[0], out, iters=10, stream=stream)
    for cam in frames:
        ctx.forward(scene, cam, out=out, tile=tile, batch=batch, chunk=chunk, stream=stream)
    capacity = int(ctx.stats(reset=True, stream=stream)["instances_max"] * 1.25) + 4096
    del out

    def timed(overlap):
        pipe = api.FramePipeline(ctx, scene, frames[0], weights, capacity, tile, batch, chunk, overlap=overlap,
                                 slots=args.frames_in_flight)
        for t in range(args.warmup):
            pipe.step(frames[t % len(frames)], mids[(t - 1) % len(mids)])
        pipe.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        render_streams = [pipe.rs[0]] if pipe.rs[1] is pipe.rs[0] else pipe.rs
        e0.record(pipe.ps)
        for st_ in render_streams:
            if st_ is not pipe.ps:
                st_.wait_event(e0)
        for i in range(args.steps):
            t = args.warmup + i
            pipe.step(frames[t % len(frames)], mids[(t - 1) % len(mids)])
        for st_ in render_streams:  # the post stream joins the render streams
            if st_ is not pipe.ps:
                done = torch.cuda.Event()
                done.record(st_)
                pipe.ps.wait_event(done)
        e1.record(pipe.ps)
        e1.synchronize()
        ms = slowest_rank(e0.elapsed_time(e1), world, "cuda")
        for k, g in enumerate(pipe.graphs):
            g.check(stream=pipe.rs[k])  # raises if a frame overflowed the instance capacity
        pipe.close()
        return ms

    ms_serial = timed(False)
    clk_path = os.path.join(tempfile.gettempdir(), "gsr_clocks_pipe_%d_%d.csv" % (os.getpid(), rank))
    smi, smi_f = start_clock_sampler(clk_path, local_rank)
    time.sleep(0.3)
    ms = timed(True)
    if smi:
        smi.terminate()
        smi.wait()
        smi_f.close()
    clocks = read_clocks(clk_path)
    fps = 1e3 * args.steps * world / ms
    if rank == 0:
        line = {"metric": "pipeline frames/s (render + x4 interpolation + warp pair)", "value": fps,
                "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "pipeline", "desc": PIPE_DESC, "tile": tile, "batch": batch, "chunk": chunk,
                           "parallelism": "replicas" if world > 1 else "single GPU, two streams"},
                "hr_mpix_s": 16 * W * H * fps / 1e6,
                "serial": {"frames_per_s": 1e3 * args.steps * world / ms_serial, "ms_per_step": ms_serial / args.steps},
                "speedup_vs_serial": ms_serial / ms, "clocks": clocks,
                # per frame: the render graph's kernels (13 + 2 tile-sort passes), 2 interpolations,
                # 2 warps x 2
                "gpu_launches": args.steps * (13 + 2 + 2 + 4)}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def algorithmic(stage, w, deg, n, K_avg, V_avg, tile_passes, pixels, pairs):
    """Algorithmic work of one launch of `stage` (bytes, or FP32 ops for compositing)."""
    sh_bytes = 12 * (deg + 1) ** 2
    if stage == "project":  # means of all; scales, quaternion, opacity, SH of the visible; 48-byte record out
        return "hbm", 12.0 * n + (12 + 16 + 4 + sh_bytes + 48) * V_avg
    if stage == "scan":
        return "hbm", 8.0 * n / 1024
    if stage == "compact":  # tile count of all, depth of the visible; 4-byte key + 4-byte index out
        return "hbm", 4.0 * n + (4.0 + 8.0) * V_avg
    if stage == "depth_sort":  # 4 passes, each reads and writes a 4-byte key and a 4-byte value
        return "hbm", V_avg * 16 * 4
    if stage == "duplicate":  # index, tile count and rectangle per visible Gaussian; key + index per instance
        return "hbm", (4.0 + 4.0 + 12.0) * V_avg + 8.0 * K_avg
    if stage == "tile_sort":
        return "hbm", K_avg * 16 * tile_passes
    if stage == "ranges":  # plain forwards: the sorted tile key read per instance (compositing
        # gathers the records by index, so no sorted record copy is made); the ranges are tiny
        return "hbm", 4.0 * K_avg
    # composite: FP32 FLOP of the per-pair work, an FMA counted as 2: 16 per evaluated pair
    # (alpha: offset, quadratic form, exponent, opacity), 38 more per blended pair (the
    # Eq. 2-4 updates of colour, depth, T and the x/y gradient terms), on the census' counts
    p_eval, p_blend = pairs
    return "alu", FLOP_PER_EVAL * p_eval + FLOP_PER_BLEND * p_blend


FLOP_PER_EVAL = 16.0
FLOP_PER_BLEND = 38.0
SMS, FP32_LANES = 152, 128


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak: SMs x FP32 lanes x 2 FLOP x clock."""
    return SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


def recorded_traffic(stage, tile, batch, chunk, workload):
    """DRAM bytes per frame of a stage's kernels from the committed ncu summary
    (profiles/traffic.txt), if it was taken on the current source of those kernels
    and the same workload and tile / batch / chunk (else None)."""
    import hashlib

    src = {"composite": "composite.cu", "depth_sort": "sort.cu", "tile_sort": "sort.cu",
           "project": "project.cu"}.get(stage)
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not src or not os.path.exists(path):
        return None
    sha = hashlib.sha1(open(os.path.join(ROOT, "paper_2605_11489_gb300", "csrc", src), "rb").read()).hexdigest()
    want = {"stage": stage, "source_sha1": sha, "tile": str(tile), "batch": str(batch), "chunk": str(chunk),
            "workload": workload}
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if all(f.get(k) == v for k, v in want.items()):
            return float(f["dram_bytes_per_launch"])
    return None


def measure_render(args, name, ctx, stream, sc, cams, world, rank, local_rank, full=True, cpu_seconds=12.0):
    """Times one render workload the way the headline is timed and returns its fields:
    value (whole-job Mpix/s), the per-stage breakdown and rooflines, e2e through the
    host frame stream, and (full=True) the backward and normal-channel timings."""
    import torch

    from paper_2605_11489_gb300 import abi, api, synth

    W, H = cams[0].width, cams[0].height
    with torch.cuda.stream(stream):
        scene = api.Scene.from_arrays(sc)
        out = api.alloc_outputs(W, H)
    stream.synchronize()
    # untimed: the autotuner's choice of tile / batch / chunk (unless given), then
    # plain renders of every camera for the instance counts that size the graph
    tile, batch, chunk = args.tile, args.batch, args.chunk
    if not (tile and batch and chunk):
        t, b, c, _ = ctx.autotune(scene, cams[0], out, iters=10, stream=stream)
        tile, batch, chunk = tile or t, batch or b, chunk or c
    # the pair census runs the sequential pass (no list splitting), so its counts are
    # the method's own: pairs up to each pixel's stop
    for cam in cams:
        ctx.forward(scene, cam, out=out, tile=tile, batch=batch, chunk=1 << 24, count=True, stream=stream)
    pre = ctx.stats(reset=True, stream=stream)
    census = (pre["pairs_evaluated"] / len(cams), pre["pairs_blended"] / len(cams))
    capacity = int(pre["instances_max"] * 1.25) + 4096
    # the timed replays: api.FrameStream, --frames-in-flight frames at once (one captured
    # graph and stream per slot, taking the frames in turn, so one frame's compositing runs
    # beside the next frames' projection and sorts). Each graph carries two events per frame
    # around compositing (the dominant kernel, whose launch duration the roofline needs); the
    # per-stage breakdown comes from one more graph, replayed alone afterwards, with events
    # at every stage boundary (nine event nodes per frame cost about 5 % of a frame)
    fs = api.FrameStream(ctx, scene, cams[0], capacity, tile, batch, chunk, timed="composite",
                         slots=args.frames_in_flight)
    for i in range(args.warmup):
        fs.render(cams[i % len(cams)])
    fs.synchronize()
    fs.stats(reset=True)

    def timed_replays(frame_stream):
        """Times args.steps frames (CUDA events on `stream`: every slot's first frame waits
        for the start event, and the end event waits for every slot's last frame)."""
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        frame_stream.follow(stream)
        for i in range(args.steps):
            frame_stream.render(cams[(args.warmup + i) % len(cams)])
        frame_stream.join(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    clk_path = os.path.join(tempfile.gettempdir(), "gsr_clocks_%d_%d_%s.csv" % (os.getpid(), rank, name))
    smi, smi_f = start_clock_sampler(clk_path, local_rank)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = timed_replays(fs)
    if world > 1:
        torch.distributed.barrier()
    if smi:
        smi.terminate()
        smi.wait()
        smi_f.close()
    clocks = read_clocks(clk_path)
    sts = fs.stats(reset=True)
    st = {key: sum(x[key] for x in sts) for key in ("frames", "instances_total", "visible_total", "timed_frames")}
    ms = slowest_rank(ms, world, "cuda")
    value = job_throughput(W * H * args.steps, world, ms * 1e-3)
    # the dominant kernel's launch duration inside the timed region (every slot's frames,
    # sharing the GPU with the other frames in flight)
    composite_ms_in_flight = (sum(x["stage_ms"]["composite"] * x["timed_frames"] for x in sts)
                              / max(1, sum(x["timed_frames"] for x in sts)))
    fs.close()
    # the same replays one frame at a time (a one-slot frame stream): a timed region of its
    # own, where the compositing events measure the kernel alone (the roofline's launch
    # duration)
    fs1 = api.FrameStream(ctx, scene, cams[0], capacity, tile, batch, chunk, timed="composite", slots=1)
    for i in range(args.warmup):
        fs1.render(cams[i % len(cams)])
    fs1.synchronize()
    fs1.stats(reset=True)
    ms_one = slowest_rank(timed_replays(fs1), world, "cuda")
    sts1 = fs1.stats(reset=True)
    composite_ms_alone = (sum(x["stage_ms"]["composite"] * x["timed_frames"] for x in sts1)
                          / max(1, sum(x["timed_frames"] for x in sts1)))
    fs1.close()
    one_stream = {"value": job_throughput(W * H * args.steps, world, ms_one * 1e-3), "unit": "Mpix/s",
                  "ms_per_step": ms_one / args.steps}

    # per-stage times: a replay of the camera path with events at every stage boundary
    staged = ctx.graph(scene, cams[0], out, capacity=capacity, tile=tile, batch=batch, chunk=chunk, timed=True,
                       stream=stream)
    for cam in cams[:3]:
        staged.render(cam, stream=stream)
    staged.stats(reset=True, stream=stream)
    for cam in cams:
        staged.render(cam, stream=stream)
    stage_ms = staged.stats(reset=True, stream=stream)["stage_ms"]
    staged.close()
    frames = max(st["frames"], 1)
    K_avg = st["instances_total"] / frames
    V_avg = st["visible_total"] / frames
    n_tiles = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    tile_passes = math.ceil(max(1, math.ceil(math.log2(max(n_tiles, 2)))) / 8)
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    hbm_peak, sm_max_mhz, peak_src = measured_peaks()

    def roofline(stage, ms_stage=None):
        bound, amount = algorithmic(stage, (W, H), sc.deg, sc.n, K_avg, V_avg, tile_passes, W * H, census)
        ms_stage = stage_ms[stage] if ms_stage is None else ms_stage
        if bound == "hbm":
            achieved = amount / (ms_stage * 1e-3) / 1e9
            return {"bound": "hbm", "kernel": stage, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak,
                    "traffic": recorded_traffic(stage, tile, batch, chunk, name),
                    "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src,
                    "algorithmic_bytes_per_launch": amount, "launch_ms": ms_stage}
        peak = fp32_peak_tflops(sm_max_mhz)
        achieved = amount / (ms_stage * 1e-3) / 1e12
        return {"bound": "alu", "kernel": stage, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": recorded_traffic(stage, tile, batch, chunk, name),
                "peak_source": "derived: %d SMs x %d FP32 lanes x 2 FLOP x %.0f MHz" % (SMS, FP32_LANES, sm_max_mhz),
                "algorithmic_flop_per_launch": amount, "launch_ms": ms_stage,
                "pairs_evaluated_per_frame": census[0], "pairs_blended_per_frame": census[1]}

    # the dominant kernel at its launch duration measured one frame at a time (the one-stream
    # timed replays); beside it, the same kernel while the other frames in flight share the GPU
    alone_ms = composite_ms_alone if dom == "composite" and composite_ms_alone > 0 else None
    roof = roofline(dom, alone_ms)
    roof["launch_ms_source"] = ("CUDA events around compositing in each replay of the one-stream timed region "
                                "(one frame at a time)")
    if dom == "composite":
        shared = roofline(dom, composite_ms_in_flight)
        roof["in_flight"] = {"launch_ms": composite_ms_in_flight, "achieved": shared["achieved"],
                             "frac": shared["frac"],
                             "note": "compositing's events inside the frames-in-flight timed region, where "
                                     "the other frames' kernels share the SMs: not a kernel duration"}
    stage_roofline = {k: {kk: v[kk] for kk in ("bound", "achieved", "unit", "frac")}
                      for k, v in ((s_, roofline(s_)) for s_ in abi.STAGES)}

    # end to end through the C ABI's frame stream (gs_frame_stream_*, wrapped by
    # api.HostFrameStream): each frame's camera from the host, all five output planes back to
    # pinned host memory (one host set per slot), every step, with one frame's copies
    # overlapping the other slots' renders; plus, for context, the one-frame synchronous call
    # gs_render_forward_to_host
    e2e = None
    if not args.no_e2e:
        nh = args.frames_in_flight
        hosts = [{k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in out.items()}
                 for _ in range(nh)]
        hfs = api.HostFrameStream(ctx, scene, cams[0], capacity, tile, batch, chunk, slots=args.frames_in_flight)
        for i in range(3):
            hfs.render(cams[i % len(cams)], hosts[i % nh])
        hfs.synchronize()
        e2e_steps = min(args.steps, 60)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            hfs.render(cams[i % len(cams)], hosts[i % nh])
        hfs.synchronize()
        dt = slowest_rank(time.perf_counter() - t0, world, "cuda")
        hfs.close()
        host = hosts[0]
        for i in range(2):
            ctx.forward_to_host(scene, cams[i], host, tile=tile, batch=batch, stream=stream)
        n_sync = min(args.steps, 30)
        t0 = time.perf_counter()
        for i in range(n_sync):
            ctx.forward_to_host(scene, cams[i % len(cams)], host, tile=tile, batch=batch, stream=stream)
        dt_sync = slowest_rank(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": job_throughput(W * H * e2e_steps, world, dt), "unit": "Mpix/s",
               "h2d_bytes_per_step": GS_CAMERA_BYTES, "d2h_bytes_per_step": 11 * W * H * 4,
               "path": "gs_frame_stream_submit (C ABI; api.HostFrameStream): graph replay per frame with the "
                       "camera from the host, --frames-in-flight frames on their own streams, D2H of rgb, dC/dx, "
                       "dC/dy, depth, alpha into pinned host memory, copies overlapping the other frames' renders",
               "sync_call": {"value": job_throughput(W * H * n_sync, world, dt_sync), "unit": "Mpix/s",
                             "path": "gs_render_forward_to_host per frame (plain forward + D2H, synchronous)"}}

    # the backward workload: forward keeping the state, then the backward of
    # N(0,1) upstream gradients on rgb, dC/dx and dC/dy (CUDA events, plain calls)
    bwd = None
    if full and not args.no_backward:
        ups = synth.upstream_grads(W, H, 3)
        g_in = {k: torch.from_numpy(v).to("cuda") for k, v in ups.items()}
        grads = scene.zeros_like_grads()
        torch.cuda.synchronize()  # inputs made on the default stream, used on `stream`
        for i in range(2):
            o, state = ctx.forward(scene, cams[i], out=out, tile=tile, batch=batch, chunk=chunk, state=True,
                                   stream=stream)
            ctx.backward(state, scene, g_in, grads=grads, stream=stream)
            state.free()
        n_b = min(args.steps, 20)
        ef, ef2, eb, ee = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        f_ms = b_ms = 0.0
        for i in range(n_b):
            ef.record(stream)
            o, state = ctx.forward(scene, cams[i % len(cams)], out=out, tile=tile, batch=batch, chunk=chunk,
                                   state=True, stream=stream)
            ef2.record(stream)
            # the plain forward returns after reading its counts back, so the device
            # would idle while the host sets up the backward call: a device-side wait
            # of ~0.5 ms covers that, and eb..ee spans the backward's kernels alone
            with torch.cuda.stream(stream):
                torch.cuda._sleep(BWD_HOST_COVER_CYCLES)
            eb.record(stream)
            ctx.backward(state, scene, g_in, grads=grads, stream=stream)
            ee.record(stream)
            ee.synchronize()
            f_ms += ef.elapsed_time(ef2)
            b_ms += eb.elapsed_time(ee)
            state.free()
        bwd = {"frames": n_b, "forward_with_state_ms": f_ms / n_b, "backward_ms": b_ms / n_b,
               "fwd_bwd_mpix_s": W * H / ((f_ms + b_ms) / n_b * 1e-3) / 1e6,
               "path": "gs_render_forward (GS_EMIT_BWD_STATE, plain) + gs_render_backward; upstream N(0,1) on "
                       "rgb, dC/dx, dC/dy; grads of means, log-scales, quaternions, opacity logits, SH; "
                       "backward_ms: CUDA events around the backward's kernels, the host's call setup "
                       "covered by a device-side wait"}

    # the normal channel (plain forward, whole tile lists) against the same plain forward
    # without it, CUDA events, after two warm-up frames each
    nrm = None
    if full and not args.no_normals:
        def plain_ms(keys, chunk_):
            o = api.alloc_outputs(W, H, keys)
            for i in range(2):
                ctx.forward(scene, cams[i], out=o, tile=tile, batch=batch, chunk=chunk_, stream=stream)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n_f = min(args.steps, 20)
            ea.record(stream)
            for i in range(n_f):
                ctx.forward(scene, cams[i % len(cams)], out=o, tile=tile, batch=batch, chunk=chunk_, stream=stream)
            eb.record(stream)
            eb.synchronize()
            return ea.elapsed_time(eb) / n_f

        nrm = {"forward_ms": plain_ms(api.OUTPUT_KEYS, chunk),
               "forward_unsplit_ms": plain_ms(api.OUTPUT_KEYS, 1 << 24),
               "forward_with_normals_ms": plain_ms(api.OUTPUT_KEYS + api.NORMAL_KEYS, chunk),
               "path": "gs_render_forward (plain, one host sync per frame); the normal channel composites "
                       "whole tile lists, so forward_unsplit_ms is its like-for-like reference"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, cams, name, max_seconds=cpu_seconds)
    del scene, out
    return {"value": value, "ms_per_step": ms / args.steps, "frames_per_s": 1e3 * args.steps * world / ms,
            "config": {"workload": name, "desc": WORKLOADS[name]["desc"], "width": W, "height": H,
                       "gaussians": sc.n, "sh_degree": sc.deg, "tile": tile, "batch": batch, "chunk": chunk,
                       "path": "CUDA graph replay per frame, %d frames in flight (gs_frame_stream_* via api.FrameStream)"
                               % args.frames_in_flight, "frames_in_flight": args.frames_in_flight,
                       "l2": "inputs larger than L2 (scene %.0f MB)" % (sc.nbytes() / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "backward": bwd, "normals": nrm, "stage_ms": stage_ms, "one_stream": one_stream,
            "stage_ms_source": "a replay of the camera path one frame at a time with events at every stage "
                               "boundary",
            "instances_per_frame": K_avg, "visible_per_frame": V_avg,
            "roofline": roof, "stage_roofline": stage_roofline, "clocks": clocks, "e2e": e2e,
            "cpu_baseline": cpu,
            # kernels per frame: projection, colour, block scan, compaction, 4 depth-sort
            # passes, duplication, `tile_passes` tile-sort passes, ranges, plan, the long-tile
            # and the short-tile compositing kernels
            "gpu_launches": args.steps * (13 + tile_passes)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS) + ["serve", "interp", "gass", "pipeline"])
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests in the stream")
    ap.add_argument("--serve-scale", type=float, default=1.0, help="serve: scale of the scene sizes")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="serve: sort-buffer budget")
    ap.add_argument("--inflight", type=int, default=16, help="serve: in-flight request slots")
    ap.add_argument("--load", type=float, default=0.8, help="serve: Poisson rate / plain renderer's rate")
    ap.add_argument("--tile", type=int, default=0, help="tile side 8/16/32 (0 = autotune)")
    ap.add_argument("--batch", type=int, default=0, help="Gaussians per shared-memory batch (0 = autotune)")
    ap.add_argument("--chunk", type=int, default=0, help="records per chunk of a split tile list (0 = autotune)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-backward", action="store_true", help="skip the forward+backward timing")
    ap.add_argument("--no-normals", action="store_true", help="skip the normal-channel timing")
    ap.add_argument("--no-legs", action="store_true",
                    help="the headline workload only (without the 6M and serving legs of the default line)")
    ap.add_argument("--frames-in-flight", type=int, default=6,
                    help="frames rendered concurrently, one graph and stream each (api.FrameStream)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload == "interp":
        return run_interp(args)
    if args.workload == "gass":
        return run_gass(args)
    if args.workload == "pipeline":
        return run_pipeline(args)

    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2605_11489_gb300 import api, synth  # noqa: F401

    stream = torch.cuda.Stream()
    ctx = api.Context(local_rank)
    sc, cams = make_workload(args.workload)
    head = measure_render(args, args.workload, ctx, stream, sc, cams, world, rank, local_rank, full=True)
    del sc
    # The metric's other legs, in the same line, for the default workload: the 6M scene
    # (1920x1080 and 480x270 fly-throughs), and the serving stream (p50 / p99 latency and
    # Mpix/s against the plain one-request-per-launch renderer).
    legs = None
    if args.workload == "large" and not args.no_legs:
        legs = {}
        sc6, _ = make_workload("ultra")
        for leg in ("ultra", "ultra_lr"):
            w = WORKLOADS[leg]
            cams6 = synth.flythrough_cameras(60, w["width"], w["height"])
            legs[leg] = measure_render(args, leg, ctx, stream, sc6, cams6, world, rank, local_rank, full=False,
                                       cpu_seconds=8.0)
        del sc6
        torch.cuda.empty_cache()
        if world == 1:
            legs["serve"] = run_serving(args)
        else:
            legs["serve"] = {"skipped": "the serving leg runs at N = 1"}
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
        line.update({k: v for k, v in head.items() if k not in ("value", "ms_per_step")})
        if legs is not None:
            line["legs"] = legs
            launches = line["gpu_launches"]
            for leg in ("ultra", "ultra_lr"):
                launches += legs[leg]["gpu_launches"]
            line["gpu_launches_all_legs"] = launches
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
