#!/usr/bin/env python3
"""Benchmark of the meshless ray-caster on the whole-cell-scale frame.

Workload (default, "cell4k"): 100,000,000 atoms (20,000 protein-like blobs in
a 12,000 A cube), 3840x2160, van der Waals spheres, Blinn-Phong, 16-sample
SSAO, overview camera 36,000 A away.  One step = one full frame: cull,
precise setup + direct splat, tile binning, tile ray-cast, resolve, shading,
SSAO.  Inputs (1.6 GB of atom records) are larger than L2, so no flush is
needed between steps.

The timed frames record two CUDA events around the cull (its live duration
feeds the roofline object); events between all stages would serialise the
kernels' programmatically dependent launches, so the per-stage breakdown
comes from the same frames re-run after the timed region, and the frames are
timed once more with no event inside them ("unprofiled").

Also measured in the same run (keys under "extra", skipped with --no-extra):
the 8K frame and its RGBA8 export, the 1.07e6 / 1.10e7-atom size sweep, the
SES of the 1e5-atom system, the batched trajectory (500,000 atoms x 256
frames x 4 views at 1280x720, one graph launch) against the plain per-frame
loop, the soft-edge renderer's forward+backward time (20,000 atoms, 16 views
at 512x512), and the 1e5-atom protein frame at 1920x1080.  --ses-only,
--soft-only and --protein-only print just one of these (for profiling).

--impl reference times the CPU FP64 oracle (the only reference there is) on
a bounded sample of the same frame on the host cores.

Prints ONE JSON line (rank 0).  Multi-GPU runs are replicas: every rank
renders the same frame (weak scaling), value = frames of all ranks / time.
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

KERNELS_PER_FRAME = 8  # clear, cull, setup, scan, scatter, raster, resolve list, resolve/shade


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vtx", choices=["vtx", "reference"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--clusters", type=int, default=20000, help="blobs of 5,000 atoms (20,000 = 1e8 atoms)")
    ap.add_argument("--ses-only", action="store_true",
                    help="only the SES of the 1e5-atom system (one JSON line; for profiling its kernels)")
    ap.add_argument("--protein-only", action="store_true",
                    help="only the 1e5-atom protein frame at 1920x1080 (one JSON line; for profiling its kernels)")
    ap.add_argument("--soft-only", action="store_true",
                    help="only the soft-edge forward and backward (one JSON line; for profiling their kernels)")
    ap.add_argument("--fp32-only", action="store_true",
                    help="only the FP32 multiply-add rate microbenchmark (one JSON line)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batched trajectory (one JSON line; for profiling its kernels)")
    ap.add_argument("--batch-frames", type=int, default=256,
                    help="trajectory frames of the batched extra (256 = the full workload; fewer for profiling)")
    return ap.parse_args()


def frame_config(n_atoms, width, height, world=1):
    """The benchmark workload's config, shared by the GPU arm and the reference arm."""
    return {"workload": "cell4k: 1e8-atom whole-cell stand-in (20,000 protein-like blobs in a 12,000 A cube), "
                        "3840x2160, vdW spheres + Blinn-Phong + SSAO16, view V1 at 36,000 A",
            "atoms": int(n_atoms), "width": int(width), "height": int(height),
            "l2": "inputs (1.6 GB) larger than L2; no flush",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def fp32_rates(vtx, torch, dev, iters=4000):
    """Measured FP32 multiply-add rate of this GPU (scalar FFMA and paired FFMA2) with the SM clock sampled
    during the runs.  The scalar rate / 64 flops is the warp-instruction issue rate."""
    import ctypes
    lib = vtx.load()
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    res = {}
    for name, paired in (("scalar_ffma", 0), ("paired_ffma2", 1)):
        best = None
        for _ in range(3):
            ms, fl = ctypes.c_float(), ctypes.c_double()
            code = lib.vtx_measure_fp32_rate(paired, iters, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                             ctypes.byref(ms), ctypes.byref(fl))
            if code != 0:
                raise RuntimeError("vtx_measure_fp32_rate failed: %d" % code)
            t = fl.value / (ms.value * 1e-3) / 1e12
            best = t if best is None or t > best else best
        res[name] = {"tflops": best, "ms": ms.value}
    clk = clocks.stop()
    scalar = res["scalar_ffma"]["tflops"]
    return {"fp32_tflops": max(scalar, res["paired_ffma2"]["tflops"]), "scalar_ffma_tflops": scalar,
            "paired_ffma2_tflops": res["paired_ffma2"]["tflops"],
            "warp_instr_per_s": scalar * 1e12 / 64.0, "clocks": clk,
            "note": "8 blocks of 256 threads per SM, 8 independent FMA chains per thread, CUDA events, best of 3"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def aggregate_replicas(elapsed_ms, steps, world, device):
    """Whole-job timing of N replicas: the slowest rank's time (MAX all-reduce) and all ranks' frames/s."""
    if world > 1:
        import torch
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, world * steps / (elapsed_ms / 1e3)


def oracle_baseline(scene, kernel, cam_index, target_s, max_pixels=4096):
    """Time the oracle on a bounded random pixel sample of the frame; frames/s extrapolated to W*H pixels."""
    import oracle
    cam = scene.cameras[cam_index]
    W, H = cam.width, cam.height
    rng = np.random.default_rng(99)
    threads = os.cpu_count() or 1
    n = 8
    while True:
        pix = np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], 1).astype(np.int32)
        t0 = time.perf_counter()
        oracle.render_pixels(scene, cam_index, pix, kernel=kernel, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or n >= max_pixels:
            break
        n = int(min(max_pixels, max(2 * n, n * target_s / max(dt, 1e-3))))
    per_pixel = dt / n
    fps = 1.0 / (per_pixel * W * H)
    return {"value": fps, "unit": "frames/s", "cores": threads, "kind": "oracle",
            "sample": "%d random pixels of the %dx%d frame, brute force over all %d atoms incl. SSAO fetches, "
                      "%.1f s; frames/s extrapolated to %d pixels" % (n, W, H, scene.xyzr.shape[0], dt, W * H),
            "seconds": dt}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2501_12750_gb300 import scenes

    if args.impl == "reference":
        if rank != 0:
            return 0
        s = scenes.config3(n_clusters=args.clusters)
        k = scenes.ssao_kernel()
        # each step is one bounded sample of the same frame
        vals, sample_s = [], []
        cb = None
        for i in range(max(1, args.warmup // 5) + args.steps):
            cb = oracle_baseline(s, k, 0, max(1.0, args.cpu_seconds / max(1, args.steps)), max_pixels=512)
            if i >= max(1, args.warmup // 5):
                vals.append(cb["value"])
                sample_s.append(cb["seconds"])
        v = float(np.median(vals))
        cb["value"] = v
        # a step is one bounded pixel sample of the frame: ms_per_step is its measured wall time, and value
        # extrapolates the sample's per-pixel time to the whole frame
        step_ms = 1e3 * float(np.median(sample_s))
        line = {"impl": "reference", "metric": "frames/s", "value": v, "unit": "frames/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": frame_config(s.xyzr.shape[0], s.cameras[0].width, s.cameras[0].height),
                "extrapolated_ms_per_frame": 1e3 / v,
                "step_note": "each step renders a bounded random pixel sample of the frame with the FP64 oracle; "
                             "value = frames/s extrapolated from the sample's time per pixel",
                "cpu_baseline": cb, "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import paper_2501_12750_gb300 as vtx

    if args.ses_only:
        if rank == 0:
            print(json.dumps({"metric": "ses_ms", "unit": "ms", "higher_is_better": False, "data": "synthetic",
                              **ses_extra(vtx, torch, dev)}))
        return 0
    if args.protein_only:
        if rank == 0:
            print(json.dumps({"metric": "protein_frame_ms", "unit": "ms", "higher_is_better": False,
                              "data": "synthetic", **protein_extra(vtx, torch, dev)}))
        return 0
    if args.fp32_only:
        if rank == 0:
            print(json.dumps({"metric": "fp32_tflops", "unit": "TFLOP/s", "higher_is_better": True,
                              **fp32_rates(vtx, torch, dev)}))
        return 0
    if args.batch_only:
        if rank == 0:
            print(json.dumps({"metric": "batch_ms", "unit": "ms", "higher_is_better": False, "data": "synthetic",
                              **batch_extra(vtx, torch, dev, vtx.Renderer(dev.index), n_frames=args.batch_frames)}))
        return 0
    if args.soft_only:
        if rank == 0:
            peak = fp32_rates(vtx, torch, dev)["fp32_tflops"]
            print(json.dumps({"metric": "soft_fwd_bwd_ms", "unit": "ms", "higher_is_better": False,
                              "data": "synthetic",
                              **soft_extra(vtx, torch, dev, vtx.Renderer(dev.index), fp32_peak=peak)}))
        return 0

    t_gen = time.time()
    s = scenes.config3(n_clusters=args.clusters)
    gen_s = time.time() - t_gen
    cam = s.cameras[0]
    W, H = cam.width, cam.height
    N = s.xyzr.shape[0]
    k = scenes.ssao_kernel()
    r = vtx.Renderer(dev.index)
    xyzr = torch.from_numpy(s.xyzr).to(dev)
    elem = torch.from_numpy(s.elem).to(dev)
    r.upload_atoms(xyzr, elem, s.palette)
    r.set_camera(cam)
    out = r.alloc_outputs(W, H)
    warm = vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC)
    timed = vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_PROFILE_CULL)
    for _ in range(max(3, args.warmup)):
        r.render_frame(warm, out=out)
    r.sync_status()
    try:
        r.stage_times()
    except vtx.VtxError:
        pass
    stream = r.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index if world == 1 else local)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        r.render_frame(timed, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    cull_ms = r.stage_times()["cull"]  # live, from the two events around each timed frame's cull
    r.sync_status()  # raises on a capacity overflow inside the timed region
    ms_total, fps = aggregate_replicas(elapsed_ms, args.steps, world, dev)
    ms_per_step = ms_total / args.steps

    # per-stage breakdown: the same frames again with all eight stage events (outside the timed region;
    # events between every pair of kernels serialise their programmatically dependent launches)
    for _ in range(args.steps):
        r.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_PROFILE), out=out)
    stages = r.stage_times()
    # and with no event at all inside the frames
    unprof_ms = _frame_ms(vtx, torch, r, vtx.default_settings(ssao_kernel=k), out, reps=args.steps)

    peak, peak_kind = measured_peaks()
    alg_bytes = 16.0 * N
    achieved = alg_bytes / (cull_ms * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "k_cull_direct_traffic.txt")
    if os.path.exists(prof):
        kv = {}
        for ln in open(prof):
            if ":" in ln:
                key, val = ln.split(":", 1)
                kv[key.strip()] = val.strip()
        if kv.get("kernel") == "k_cull_direct" and kv.get("atoms") == str(N) and kv.get("current") == "yes":
            traffic = float(kv["bytes_per_launch"])

    # end to end through the host-buffer entry point (copies inside the timed region)
    host_x = torch.from_numpy(s.xyzr).pin_memory()
    host_e = torch.from_numpy(s.elem).pin_memory()
    ho = {"depth": torch.empty((H, W), dtype=torch.float32).pin_memory(),
          "id": torch.empty((H, W), dtype=torch.int32).pin_memory(),
          "normal": torch.empty((3, H, W), dtype=torch.float32).pin_memory(),
          "rgb": torch.empty((3, H, W), dtype=torch.float32).pin_memory(),
          "ao": torch.empty((H, W), dtype=torch.float32).pin_memory()}
    hon = {kk: v.numpy() for kk, v in ho.items()}
    he = vtx.default_settings(ssao_kernel=k)
    r.render_frame_host(host_x.numpy(), host_e.numpy(), cam, he, hon, s.palette)
    n_e2e = max(2, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        r.render_frame_host(host_x.numpy(), host_e.numpy(), cam, he, hon, s.palette)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    h2d = 17 * N
    d2h = 4 * 9 * W * H

    # end to end with the atoms left in page-locked host memory: the kernels stream them over the host link
    # every frame (nothing is copied up front) and the output planes are copied back every frame
    rh = vtx.Renderer()
    rh.upload_atoms(host_x, host_e, s.palette)
    rh.set_camera(cam)
    dout = rh.alloc_outputs(W, H)
    rh.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=dout)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        rh.render_frame(he, out=dout)
        for kk in ho:
            ho[kk].copy_(dout[kk], non_blocking=True)
        torch.cuda.current_stream().synchronize()
    stream_s = (time.perf_counter() - t0) / n_e2e
    del rh, dout

    # pipelined end to end: two contexts on two streams take alternate frames, atoms stay in page-locked host
    # memory and every frame's output planes are written straight into page-locked host buffers, so one
    # frame's outputs travel device-to-host while the next frame's atoms travel host-to-device
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    rp = [vtx.Renderer(stream=st_) for st_ in streams]
    hop = [{kk: torch.empty_like(v).pin_memory() for kk, v in ho.items()} for _ in range(2)]
    for i in range(2):
        rp[i].upload_atoms(host_x, host_e, s.palette)
        rp[i].set_camera(cam)
        rp[i].render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=hop[i])
    torch.cuda.synchronize()
    n_pipe = max(4, 2 * n_e2e)
    t0 = time.perf_counter()
    for j in range(n_pipe):
        rp[j & 1].render_frame(he, out=hop[j & 1])
    for st_ in streams:
        st_.synchronize()
    pipe_s = (time.perf_counter() - t0) / n_pipe
    del rp, hop

    extra = {}
    if not args.no_extra:
        extra = run_extras(vtx, torch, dev, r, s, cam, k)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_baseline(s, k, 0, args.cpu_seconds)

    line = {
        "metric": "frames/s", "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": frame_config(N, W, H, world),
        "gatoms_per_s": fps * N / 1e9,
        "roofline": {"bound": "hbm", "kernel": "k_cull_direct", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": cull_ms},
        "stages_ms": {kk: v for kk, v in stages.items() if kk != "runs"},
        "stages_note": "stages_ms: the same frames re-run after the timed region with an event after every "
                       "stage; the timed frames record events around the cull only (its live duration feeds "
                       "the roofline)",
        "unprofiled": {"ms_per_step": unprof_ms, "frames_per_s": 1e3 / unprof_ms,
                       "note": "the same frames timed with no event inside them"},
        "e2e": {"value": 1.0 / pipe_s, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "vtx_upload_atoms(page-locked host atoms) + vtx_render_frame into page-locked host output "
                       "planes, two contexts on two streams taking alternate frames (%d frames)" % n_pipe},
        "e2e_variants": {
            "render_frame_host": {"value": 1.0 / e2e_s, "unit": "frames/s",
                                  "api": "vtx_render_frame_host: copy up, render, copy down, synchronise"},
            "host_resident_one_stream": {"value": 1.0 / stream_s, "unit": "frames/s",
                                         "api": "host-resident atoms, vtx_render_frame, output copies, "
                                                "synchronise every frame"}},
        "gpu_launches": KERNELS_PER_FRAME * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "gen_seconds": gen_s,
        "extra": extra,
    }
    if rank == 0:
        print(json.dumps(line))
    r.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _frame_ms(vtx, torch, r, settings, out, reps=10):
    """Mean device time of `reps` frames (CUDA events on the renderer's stream) after 3 warm-ups."""
    for _ in range(3):
        r.render_frame(settings, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(r.stream)
    for _ in range(reps):
        r.render_frame(settings, out=out)
    e1.record(r.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


OUT_BYTES_PER_PX = 36  # depth 4, id 4, normal 12, rgb 12, ao 4: the output planes every frame writes


def hbm_roofline(alg_bytes, ms, what):
    """Roofline object of an HBM-bound workload: algorithmic bytes over its measured time."""
    peak, kind = measured_peaks()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak, "peak_kind": kind,
            "frac": achieved / peak, "traffic": None, "algorithmic_bytes": alg_bytes, "bytes": what}


def protein_extra(vtx, torch, dev, reps=20):
    """The 1e5-atom protein-like system at 1920x1080 with SSAO16: library-default tiles (with per-stage device
    times) and autotuned tiles."""
    from paper_2501_12750_gb300 import scenes
    s2 = scenes.config2()
    k = scenes.ssao_kernel()
    r = vtx.Renderer(dev.index)
    r.upload_atoms(torch.from_numpy(s2.xyzr).to(dev), torch.from_numpy(s2.elem).to(dev), s2.palette)
    cam = s2.cameras[0]
    r.set_camera(cam)
    out = r.alloc_outputs(cam.width, cam.height)
    r.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=out)
    default_ms = _frame_ms(vtx, torch, r, vtx.default_settings(ssao_kernel=k), out, reps)
    for _ in range(reps):
        r.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_PROFILE), out=out)
    stages = r.stage_times()
    r.render_frame(vtx.default_settings(ssao_kernel=k, tile_w=0, flags=vtx.FLAG_SYNC), out=out)
    tuned = r.tuned_settings()
    tuned_ms = _frame_ms(vtx, torch, r, vtx.default_settings(ssao_kernel=k, tile_w=0), out, reps)
    r.close()
    alg = 16.0 * s2.xyzr.shape[0] + OUT_BYTES_PER_PX * cam.width * cam.height
    return {"protein_1080p": {"workload": "1e5 protein-like atoms, 1920x1080, vdW, SSAO16",
                              "roofline": hbm_roofline(alg, default_ms, "16 B per atom read + 36 B per pixel "
                                                       "written (the frame at library-default tiles)"),
                              "default_tiles_ms": default_ms, "frames_per_s": 1e3 / default_ms,
                              "stages_ms": {kk: v for kk, v in stages.items() if kk != "runs"},
                              "autotuned_ms": tuned_ms, "autotuned": {"tile_w": tuned[0], "tile_h": tuned[1],
                                                                      "splat_max_px": tuned[2]}}}


def ses_extra(vtx, torch, dev, reps=5):
    """SES of the 1e5-atom protein-like system on a 0.5 A grid (probe 1.4 A): wall time of the synchronous call."""
    import ctypes

    from paper_2501_12750_gb300 import scenes
    s2 = scenes.config2()
    rs = vtx.Renderer()
    x2 = torch.from_numpy(s2.xyzr).to(dev)
    g2 = rs.ses_fit_grid(x2, probe=1.4, spacing=0.5)
    first = rs.ses_mesh(x2, g2)
    n_tri = first["n"]
    tri_buf = first["tris"]
    cnt = ctypes.c_int64(0)

    def call():
        code = rs.lib.vtx_ses_mesh(rs.ctx, x2.data_ptr(), x2.shape[0], ctypes.byref(g2), tri_buf.data_ptr(), n_tri,
                                   None, None, None, ctypes.byref(cnt))
        assert code == 0 and cnt.value == n_tri
    for _ in range(2):
        call()
    t0 = time.perf_counter()
    for _ in range(reps):
        call()
    ses_ms = (time.perf_counter() - t0) / reps * 1e3
    pts = int(g2.dims[0]) * int(g2.dims[1]) * int(g2.dims[2])
    return {"workload": "1e5 atoms, SES (probe 1.4 A) on a 0.5 A grid, marching cubes", "grid_points": pts,
            "triangles": int(n_tri), "ms": ses_ms, "gpoints_per_s": pts / ses_ms / 1e6,
            "note": "wall time of the synchronous call (SAS, 3 distance passes, count, scan, emit)"}


# FP32 operations of one composited soft term (the definition's arithmetic, counted from the formula with an
# FMA as 2 and exp, sqrt, rsqrt and a reciprocal as 1 each): the ray offset at the reference depth (6), o.u and
# |o|^2 (9), the closest approach and rho^2 (4), delta (4), the sigmoid and clamp (5), the smoothed entry depth
# (9), the normal (9) and the front-to-back accumulation of coverage, depth, normal and transmittance (14).
SOFT_FWD_FLOPS_PER_TERM = 60
# The backward recomputes the term (46, without the accumulation) and forms its vector-Jacobian product:
# the carry and the opacity derivative (12), the gradients through delta (16), through the entry depth and the
# normal (44) and the view-to-world rotation of the per-sphere sum (amortised over the warp, not counted).
SOFT_BWD_FLOPS_PER_TERM = 118


def soft_extra(vtx, torch, dev, r, reps=5, fp32_peak=None):
    """Soft-edge forward and backward on 20,000 atoms x 16 views at 512x512: the asynchronous calls with the
    forward's per-pixel state (the autograd wrapper's path), the synchronous calls, and the hard renderer on the
    same views."""
    from paper_2501_12750_gb300 import scenes
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    res = {}
    s5 = scenes.config5()
    x = torch.from_numpy(s5.xyzr).to(dev)
    tgt = torch.from_numpy(s5.extra["target"]).to(dev)
    with torch.no_grad():
        A_t, D_t, N_t = r.render_soft_fwd(tgt, s5.cameras)
    state = r.soft_state(s5.cameras)
    for _ in range(2):
        A, D, Nn = r.render_soft_fwd(x, s5.cameras, state=state)
        gA, gD, gN = 2 * (A - A_t), 0.2 * (D - D_t), 2 * (Nn - N_t)
        r.render_soft_bwd(x, s5.cameras, gA, gD, gN, state=state)
        r.render_soft_bwd(x, s5.cameras, gA, gD, gN)
    r.render_soft_fwd(x, s5.cameras, state=state)
    n_terms = r.soft_terms()  # of the forward call just made

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(r.stream)
        for _ in range(reps):
            fn()
        e1.record(r.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # asynchronous calls with the forward's per-pixel state, the backward reusing the forward's tile lists (no
    # host synchronisation inside): one forward + backward pair per step, as the autograd wrapper issues them
    def pair():
        r.render_soft_fwd(x, s5.cameras, state=state, sync=False)
        r.render_soft_bwd(x, s5.cameras, gA, gD, gN, state=state, sync=False, reuse_lists=True)

    pair_ms = timed(pair)
    fwd_ms = timed(lambda: r.render_soft_fwd(x, s5.cameras, state=state, sync=False))
    bwd_ms = timed(lambda: r.render_soft_bwd(x, s5.cameras, gA, gD, gN, state=state, sync=False,
                                             reuse_lists=True))
    bwd_rebuild_ms = timed(lambda: r.render_soft_bwd(x, s5.cameras, gA, gD, gN, state=state, sync=False))
    r.sync_status()
    # per-kernel device times of the same calls (events around each call's soft kernel are not available
    # through the API, so the kernel share is read from the launch list in profiles/)
    fwd_sync_ms = timed(lambda: r.render_soft_fwd(x, s5.cameras))
    bwd_sync_ms = timed(lambda: r.render_soft_bwd(x, s5.cameras, gA, gD, gN))
    # hard renderer on the same 16 views
    r.upload_atoms(x, torch.from_numpy(s5.elem).to(dev), s5.palette)
    hs = vtx.default_settings()
    ho = r.alloc_outputs(512, 512)
    for c in s5.cameras[:2]:
        r.set_camera(c)
        r.render_frame(vtx.default_settings(flags=vtx.FLAG_SYNC), out=ho)
    torch.cuda.synchronize()
    e0.record(r.stream)
    for c in s5.cameras:
        r.set_camera(c)
        r.render_frame(hs, out=ho)
    e1.record(r.stream)
    torch.cuda.synchronize()
    hard_ms = e0.elapsed_time(e1)
    flops = n_terms * (SOFT_FWD_FLOPS_PER_TERM + SOFT_BWD_FLOPS_PER_TERM)
    achieved = flops / (pair_ms * 1e-3) / 1e12
    soft = {"workload": "20,000 atoms, 16 views at 512x512, sigma 0.5 px", "fwd_bwd_ms": pair_ms,
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
            "api": "vtx_render_soft_fwd_ex / _bwd_ex, asynchronous, with the forward's per-pixel state and the "
            "backward reusing the forward's tile lists (the autograd wrapper's path); fwd_bwd_ms times the pair",
            "bwd_rebuild_ms": bwd_rebuild_ms, "sync_fwd_ms": fwd_sync_ms, "sync_bwd_ms": bwd_sync_ms,
            "hard_16_views_ms": hard_ms, "terms": n_terms}
    if fp32_peak:
        soft["roofline"] = {"bound": "fp32", "unit": "TFLOP/s", "achieved": achieved, "peak": fp32_peak,
                            "peak_kind": "measured (FFMA microbenchmark, same run)", "frac": achieved / fp32_peak,
                            "traffic": None,
                            "algorithmic_flops": flops,
                            "units": "%d composited terms x (%d forward + %d backward) FP32 operations"
                                     % (n_terms, SOFT_FWD_FLOPS_PER_TERM, SOFT_BWD_FLOPS_PER_TERM),
                            "time": "one forward + backward pair (the forward's binning included)"}
    res["soft"] = soft
    return res


def batch_extra(vtx, torch, dev, r, n_frames=256):
    """Batched trajectory: n_frames frames x 4 views of the 500,000-atom system at 1280x720 with SSAO16, one graph
    launch per batch, against the plain per-frame loop on the same images."""
    from paper_2501_12750_gb300 import scenes
    res = {}
    s4 = scenes.config4(n_frames=n_frames)
    frames = torch.from_numpy(s4.frames).to(dev)
    F, N4 = s4.frames.shape[0], s4.frames.shape[1]
    cams = s4.cameras
    k = scenes.ssao_kernel()
    st = vtx.default_settings(ssao_kernel=k)
    out = r.alloc_outputs(cams[0].width, cams[0].height, F * len(cams))
    elem = torch.from_numpy(s4.elem).to(dev)
    r.upload_atoms(frames[0], elem, s4.palette)
    counts = [N4] * F
    r.render_batch(frames, counts, cams, vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=out)
    r.render_batch(frames, counts, cams, st, out=out, use_graph=True)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(r.stream)
    for _ in range(reps):
        r.render_batch(frames, counts, cams, st, out=out, use_graph=True)
    e1.record(r.stream)
    torch.cuda.synchronize()
    r.sync_status()
    batch_ms = e0.elapsed_time(e1) / reps
    # plain per-frame loop on the same images (one render_frame per image)
    single = r.alloc_outputs(cams[0].width, cams[0].height)
    loop_frames = min(32, F)
    for f in range(min(2, F)):
        r.upload_atoms(frames[f], elem, s4.palette)
        r.set_camera(cams[0])
        r.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=single)
    torch.cuda.synchronize()
    e0.record(r.stream)
    for f in range(loop_frames):
        r.upload_atoms(frames[f], elem, s4.palette)
        for c in cams:
            r.set_camera(c)
            r.render_frame(st, out=single)
    e1.record(r.stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1) / (loop_frames * len(cams))
    alg = 16.0 * F * N4 + OUT_BYTES_PER_PX * F * len(cams) * cams[0].width * cams[0].height
    res["batched_traj"] = {"workload": "500,000 atoms x %d frames x 4 views, 1280x720, SSAO16" % F,
                           "roofline": hbm_roofline(alg, batch_ms, "16 B per atom and frame read once + 36 B "
                                                    "per pixel of the %d images written" % (F * len(cams))),
                           "images_per_s": F * len(cams) / (batch_ms / 1e3), "batch_ms": batch_ms,
                           "per_frame_loop_images_per_s": 1e3 / loop_ms, "graph": True}
    del out, frames
    torch.cuda.empty_cache()
    return res


def run_extras(vtx, torch, dev, r, s3, cam, k):
    import dataclasses

    from paper_2501_12750_gb300 import scenes
    res = {}
    # 8K headless export of the benchmark frame (1e8 atoms, V1, SSAO), transparent background
    cam8 = dataclasses.replace(cam, width=7680, height=4320)
    r.set_camera(cam8)
    out8 = r.alloc_outputs(7680, 4320)
    st8 = vtx.default_settings(ssao_kernel=k)
    r.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=out8)
    f8 = _frame_ms(vtx, torch, r, st8, out8)
    rgba = r.export_rgba8(out8)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(r.stream)
    for _ in range(10):
        r.export_rgba8(out8, rgba=rgba)
    e1.record(r.stream)
    torch.cuda.synchronize()
    x8 = e0.elapsed_time(e1) / 10
    res["export_8k"] = {"workload": "1e8 atoms, V1, 7680x4320, SSAO16, RGBA8 with background alpha",
                        "frame_ms": f8, "frames_per_s": 1e3 / f8, "export_ms": x8,
                        "export_gb_per_s": 7680 * 4320 * 20 / x8 / 1e6}
    del out8, rgba
    r.set_camera(cam)
    torch.cuda.empty_cache()
    # size sweep on the whole-cell generator (the paper's 1.07e6 and 1.10e7 systems), 3840x2160, V1, SSAO
    sweep = []
    for nc in (214, 2200):
        ss = scenes.config3(n_clusters=nc)
        rs = vtx.Renderer()
        rs.upload_atoms(torch.from_numpy(ss.xyzr).to(dev), torch.from_numpy(ss.elem).to(dev), ss.palette)
        rs.set_camera(ss.cameras[0])
        so = rs.alloc_outputs(3840, 2160)
        rs.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), out=so)
        ms = _frame_ms(vtx, torch, rs, vtx.default_settings(ssao_kernel=k), so, reps=20)
        sweep.append({"atoms": int(ss.xyzr.shape[0]), "frame_ms": ms, "frames_per_s": 1e3 / ms,
                      "gatoms_per_s": ss.xyzr.shape[0] / ms / 1e6})
        del rs, so, ss
        torch.cuda.empty_cache()
    res["size_sweep_3840x2160"] = sweep
    res["ses_config2"] = ses_extra(vtx, torch, dev)
    torch.cuda.empty_cache()
    res["batched_traj"] = batch_extra(vtx, torch, dev, r)["batched_traj"]
    torch.cuda.empty_cache()
    peaks = fp32_rates(vtx, torch, dev)
    res["fp32_peak"] = peaks
    res["soft"] = soft_extra(vtx, torch, dev, r, fp32_peak=peaks["fp32_tflops"])["soft"]
    res["protein_1080p"] = protein_extra(vtx, torch, dev)["protein_1080p"]
    return res


if __name__ == "__main__":
    sys.exit(main())
