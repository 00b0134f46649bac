#!/usr/bin/env python3
"""Benchmark: stereo VR frames/s at 2 x 2064x2208 with 500k Gaussians (foveated,
hierarchical 4/8/16 per-ray windows) against the plain full-resolution render on the
same GPU, p99 frame time, the dominant kernel's roofline fraction, an end-to-end
number through host buffers, and the FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one stereo frame of the seeded head trajectory (both eyes: preprocess ->
duplicate -> sort -> render -> composite).  Inputs are synthetic (the paper's scenes
are not available): a 6 m room-shaped shell of 500k Gaussians, SH degree 3.
N > 1 runs N independent replicas (the path shards by view; no collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stereo VR frames/s at 2×2064×2208, 500k Gaussians, vs plain; p99 frame ms"
N_GAUSS = 500_000
W_IMG, H_IMG = 2064, 2208
WINDOWS = (4, 8, 16)
# FP32 work of the render kernel per unit, counted from its arithmetic (FMA = 2 flops):
# an evaluated pair (plane map, conic, cut test), a kept pair (alpha with exp2, depth
# t*, window insert compares), a blended pair (transmittance test and colour FMAs).
FLOPS_EVAL, FLOPS_KEPT, FLOPS_BLEND = 24, 22, 10
FP32_LANES_PER_SM = 128


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n_frames, rank=0):
    from paper_2505_10144_gb300 import synth
    scene = synth.shell_scene(N_GAUSS, synth.rng_for(1), sh_degree=3)
    wl = synth.vr_trajectory(n_frames, synth.rng_for(1, salt=100 + rank), W_IMG, H_IMG)
    return scene, wl


def crop_camera(cam, x0, y0, w, h):
    from paper_2505_10144_gb300 import synth
    return synth.Camera(cam.world_to_cam, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.near_z)


def oracle_frame_estimate(scene64, frame, budget_s=12.0, crops=None):
    """Seconds per stereo frame of the FP64 oracle, from a bounded sample: the fixed
    per-view cost (projection of every Gaussian, one 32x32 tile) plus the per-sample
    cost of 128x128 crops of the same foveated, hierarchical frame, scaled to the
    frame's sample count.  Returns (seconds_per_frame, description, threads)."""
    from oracle import native as on
    from paper_2505_10144_gb300 import synth
    on.build()
    cam, fv = frame.cameras[0], frame.foveas[0]

    def shifted(x0, y0):
        return synth.Fovea(fv.gaze_x - x0, fv.gaze_y - y0, fv.radius_px, fv.band_px)

    x0, y0 = 1024, 1088
    t = time.perf_counter()
    on.render(scene64, crop_camera(cam, x0, y0, 32, 32), "hier", WINDOWS, 32, shifted(x0, y0))
    t_fixed = time.perf_counter() - t
    spots = crops or [(int(fv.gaze_x) // 32 * 32, int(fv.gaze_y) // 32 * 32), (128, 256), (1792, 1920), (512, 1600),
                      (1536, 384), (960, 160)]
    t_samples, n_samples, used = 0.0, 0, 0
    for (cx, cy) in spots:
        cx, cy = min(max(cx, 0), W_IMG - 128) // 32 * 32, min(max(cy, 0), H_IMG - 128) // 32 * 32
        t = time.perf_counter()
        r = on.render(scene64, crop_camera(cam, cx, cy, 128, 128), "hier", WINDOWS, 32, shifted(cx, cy))
        dt = time.perf_counter() - t
        t_samples += max(dt - t_fixed, 0.0)
        n_samples += r["stats"]["samples"]
        used += 1
        if t_samples + used * t_fixed > budget_s:
            break
    # samples of a whole eye: full-res pixels of focus/hybrid tiles + groups of periphery tiles
    full = on.render(synth.Scene(*[a[..., :0] for a in scene64.arrays()], 3),
                     cam, "exact", WINDOWS, 32, fv)
    samples_eye = full["stats"]["samples"]
    per_sample = t_samples / max(n_samples, 1)
    sec = 2 * (t_fixed + per_sample * samples_eye)
    desc = (f"FP64 oracle, hierarchical 4/8/16, foveated: fixed per-view cost (projection of all {N_GAUSS} Gaussians) "
            f"+ {used} crops of 128x128 ({n_samples} samples) scaled to {samples_eye} samples per eye x 2 eyes")
    return sec, desc, on.num_threads()


def run_reference(args, ws, rank):
    """The reference arm: the oracle as it stands, on the host cores, same metric."""
    if rank != 0:
        return
    from paper_2505_10144_gb300 import synth
    scene, wl = make_workload(max(args.steps + args.warmup, 1))
    scene64 = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in scene.arrays()], scene.sh_degree)
    vals = []
    desc, thr = "", 1
    for i in range(args.warmup + args.steps):
        fr = wl.frames[i % len(wl.frames)]
        sec, desc, thr = oracle_frame_estimate(scene64, fr, budget_s=4.0, crops=[(int(fr.foveas[0].gaze_x), int(fr.foveas[0].gaze_y)), (128, 256)])
        if i >= args.warmup:
            vals.append(sec)
    mean = statistics.mean(vals)
    value = 1.0 / mean
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "vr_stereo_2064x2208_500k_foveated_hier_4_8_16", "n_gaussians": N_GAUSS,
                       "width": W_IMG, "height": H_IMG, "views": 2},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": thr, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(args, api, torch):
    """Frames only: the workload at args.scale resolution, nothing else on the GPU."""
    from paper_2505_10144_gb300 import synth
    W, H = int(W_IMG * args.scale) // 32 * 32, int(H_IMG * args.scale) // 32 * 32
    scene = synth.shell_scene(N_GAUSS, synth.rng_for(1), sh_degree=3)
    wl = synth.vr_trajectory(args.warmup + args.steps, synth.rng_for(1, salt=100), W, H)
    ds = api.DeviceScene.from_host(scene)
    R = api.Renderer()
    cfg = api.RenderConfig(sort_mode=args.mode, windows=WINDOWS, key_tile=32, fovea_mode="bilinear")
    out = torch.empty((2, 3, H, W), device="cuda")
    for fr in wl.frames:
        R.render([ds], [0, 0], fr.cameras, fr.foveas, cfg, out=out)
    R.check()
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": True, "width": W, "height": H, "frames": len(wl.frames), **R.stats()}))
    R.close()


def psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=40)
    ap.add_argument("--ncu-case", action="store_true",
                    help="only render warmup + steps foveated frames (for profiler captures)")
    ap.add_argument("--scale", type=float, default=1.0, help="resolution scale of --ncu-case")
    ap.add_argument("--mode", default="hier", choices=["exact", "window", "hier"], help="sort mode of --ncu-case")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2505_10144_gb300 import api, build
    build.build()
    if args.ncu_case:
        ncu_case(args, api, torch)
        return
    n_frames = args.warmup + args.steps
    scene, wl = make_workload(n_frames, rank)
    ds = api.DeviceScene.from_host(scene)
    R = api.Renderer()
    fov_cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=32, fovea_mode="bilinear")
    plain_cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=16, fovea_mode="plain")
    out = torch.empty((2, 3, H_IMG, W_IMG), device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")  # > 129 MB L2: written between frames

    def frame(i, cfg, o=out):
        fr = wl.frames[i % len(wl.frames)]
        return R.render([ds], [0, 0], fr.cameras, fr.foveas, cfg, out=o)

    def barrier():
        torch.cuda.synchronize()
        if pg:
            pg.barrier()

    def timed(cfg, steps, profile=False):
        for i in range(args.warmup):
            frame(i, cfg)
        R.check()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if profile:
            R.profile_begin(steps)
        for i in range(steps):
            flush.zero_()
            ev[i][0].record()
            frame(args.warmup + i, cfg)
            ev[i][1].record()
        barrier()
        stages, ncalls = R.profile_end() if profile else ({}, 0)
        R.check()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, stages, ncalls

    # foveated frames (the headline)
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    with ClockSampler(gpu_index) as clk:
        t_wall = time.perf_counter()
        ms_fov, stages, ncalls = timed(fov_cfg, args.steps, profile=True)
        t_wall = time.perf_counter() - t_wall
    kernels_per_frame = R.stats()["kernels"]
    total_ms = sum(ms_fov)
    if pg:
        t = torch.tensor([total_ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * args.steps / (total_ms / 1e3)
    # plain full-resolution render on the same GPU
    ms_plain, _, _ = timed(plain_cfg, min(args.plain_steps, args.steps))
    # quality of the foveated frame against the plain render
    ps = []
    o2 = torch.empty_like(out)
    for i in range(3):
        a = frame(i, fov_cfg).clone()
        b = frame(i, plain_cfg, o2)
        ps.append(psnr(a, b))
    # device counters for the roofline's algorithmic work (one extra pass, not timed)
    stat_cfg = api.RenderConfig(**{**fov_cfg.__dict__, "stats": True})
    cnt = {"evaluated": 0, "kept": 0, "blended": 0, "instances": 0, "work_items": 0}
    n_stat = min(8, args.steps)
    for i in range(n_stat):
        frame(args.warmup + i, stat_cfg)
        st = R.stats()
        for k in cnt:
            cnt[k] += st[k]
    cnt = {k: v / n_stat for k, v in cnt.items()}
    render_ms = stages.get("render", 0.0) / max(ncalls, 1)
    flops = FLOPS_EVAL * cnt["evaluated"] + FLOPS_KEPT * cnt["kept"] + FLOPS_BLEND * cnt["blended"]
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local)
    sm_mhz = clocks["sm_mhz"] or 2070.0
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (render_ms / 1e3) / 1e12 if render_ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": "render_kernel<hier>", "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops if peak_tflops else None, "traffic": None,
                "peak_source": f"FP32 FMA peak: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                               f"{sm_mhz:.0f} MHz (median SM clock under load)",
                "work_per_launch": {"evaluated_pairs": cnt["evaluated"], "kept_pairs": cnt["kept"],
                                    "blended_pairs": cnt["blended"], "flops": flops},
                "avg_launch_ms": render_ms}
    # end to end through the public API: camera/gaze in, both images back to pinned host
    host = torch.empty((2, 3, H_IMG, W_IMG), dtype=torch.float32, pin_memory=True)
    for i in range(args.warmup):
        frame(i, fov_cfg)
        host.copy_(out, non_blocking=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = min(40, args.steps)
    e0.record()
    for i in range(n_e2e):
        frame(args.warmup + i, fov_cfg)
        host.copy_(out, non_blocking=True)
    e1.record()
    barrier()
    e2e_fps = ws * n_e2e / (e0.elapsed_time(e1) / 1e3)
    import ctypes
    from paper_2505_10144_gb300 import _lib
    h2d = 2 * (ctypes.sizeof(_lib.Camera) + ctypes.sizeof(_lib.Fovea))
    d2h = out.numel() * 4
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(ms_fov), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "vr_stereo_2064x2208_500k_foveated_hier_4_8_16", "n_gaussians": N_GAUSS,
                   "width": W_IMG, "height": H_IMG, "views": 2, "sh_degree": 3, "windows": list(WINDOWS),
                   "fovea": "circle r=0.15W, band 0.1r, periphery 1/2 res, bilinear",
                   "l2": "flushed between frames (256 MB write outside the timed events)",
                   "timing": "CUDA events around each frame on the launching stream"},
        "p50_ms": float(np.percentile(ms_fov, 50)), "p99_ms": float(np.percentile(ms_fov, 99)),
        "plain": {"value": len(ms_plain) / (sum(ms_plain) / 1e3), "unit": "frames/s",
                  "ms_per_step": statistics.mean(ms_plain), "p99_ms": float(np.percentile(ms_plain, 99)),
                  "config": "full resolution, 16x16 tiles, hierarchical 4/8/16, same pipeline"},
        "speedup_vs_plain": statistics.mean(ms_plain) / statistics.mean(ms_fov),
        "psnr_vs_plain_db": statistics.mean(ps),
        "stage_ms_per_frame": {k: v / max(ncalls, 1) for k, v in stages.items()},
        "counters_per_frame": cnt,
        "roofline": roofline,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "Renderer.render (vrs_render) + device-to-host copy of both eyes into pinned memory"},
        "gpu_launches": kernels_per_frame * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        from paper_2505_10144_gb300 import synth
        scene64 = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in scene.arrays()], scene.sh_degree)
        sec, desc, thr = oracle_frame_estimate(scene64, wl.frames[0])
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "frames/s", "cores": thr, "kind": "oracle",
                                "sample": desc, "host_cpus": os.cpu_count()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
