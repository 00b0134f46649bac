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
import platform
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
# Issue basis of the render roofline: about 35 FP32 operations and one exp2 per evaluated
# pair (plane map and quadratic form ~9, t* ~9, blend ~6, window compares ~log2 k per
# level), against the lane-issue peak SMs x 4 schedulers x 32 lanes x clock.
ALU_OPS_PER_PAIR = 36
LANES_PER_SM = 4 * 32


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest value of x over the ranks of the process group (a job's time is its
    slowest rank's); x itself without a group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return ws * units_per_rank / (max_ms / 1e3)


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


def rank_trajectory(n_frames, rank=0):
    """The head trajectory of one rank: every rank renders its own frames of the same
    scene (weak scaling), each from its own seed."""
    from paper_2505_10144_gb300 import synth
    return synth.vr_trajectory(n_frames, synth.rng_for(1, salt=100 + rank), W_IMG, H_IMG)


def make_workload(n_frames, rank=0):
    from paper_2505_10144_gb300 import synth
    scene = synth.shell_scene(N_GAUSS, synth.rng_for(1), sh_degree=3)
    return scene, rank_trajectory(n_frames, rank)


def crop_camera(cam, x0, y0, w, h):
    from paper_2505_10144_gb300 import synth
    return synth.Camera(cam.world_to_cam, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.near_z)


def oracle_view_estimate(scene64, cam, fv, mode, key_tile, budget_s, bands):
    """Seconds per view of the FP64 oracle, from a bounded sample of the view: full-width
    bands of 64 rows, each rendered by the oracle as it stands (the band is the view with
    the principal point shifted, so every sample is the view's).  The per-row cost scales
    to the image height; the per-view fixed cost (projection of every Gaussian) is
    measured on a 32-row band and counted once.  fv None renders plain (no fovea).
    Returns (seconds_per_view, bands used, samples)."""
    from oracle import native as on
    from paper_2505_10144_gb300 import synth
    on.build()
    W, H = int(cam.width), int(cam.height)

    def band(y0, h):
        c = crop_camera(cam, 0, y0, W, h)
        f = None if fv is None else synth.Fovea(fv.gaze_x, fv.gaze_y - y0, fv.radius_px, fv.band_px)
        t = time.perf_counter()
        r = on.render(scene64, c, mode, WINDOWS, key_tile, f)
        return time.perf_counter() - t, r["stats"]["samples"]

    # fixed cost from two heights of the same band: t(h) = fixed + h * per_row
    yc = H // 2 if fv is None else int(fv.gaze_y)
    yg = min(max(yc - 32, 0), H - 64) // 32 * 32
    t32, t64 = band(yg, 32)[0], band(yg, 64)[0]
    t_fixed = max(t32 - (t64 - t32), 0.0)
    rows, t_rows, samples, used = 0, 0.0, 0, 0
    for y in bands:
        y = min(max(y, 0), H - 64) // 32 * 32
        dt, ns = band(y, 64)
        t_rows += max(dt - t_fixed, 0.0)
        rows += 64
        samples += ns
        used += 1
        if t_rows + used * t_fixed > budget_s:
            break
    return t_fixed + t_rows / rows * H, used, samples


def oracle_frame_estimate(scene64, frame, budget_s=20.0, bands=None):
    """Seconds per stereo frame of the FP64 oracle on the foveated, hierarchical frame:
    bands of eye 0 (one through the gaze point, others in the periphery), x 2 eyes.
    Returns (seconds_per_frame, description, threads)."""
    from oracle import native as on
    cam, fv = frame.cameras[0], frame.foveas[0]
    sec, used, samples = oracle_view_estimate(scene64, cam, fv, "hier", 32, budget_s,
                                              bands or [int(fv.gaze_y), 256, 1792, 1024])
    desc = (f"FP64 oracle, hierarchical 4/8/16, foveated: {used} full-width bands of 64 rows ({samples} samples) "
            f"of eye 0, per-row cost scaled to {H_IMG} rows, plus the per-view fixed cost, x 2 eyes")
    return 2 * sec, desc, on.num_threads()


def oracle_other_workloads(scene64, frame):
    """The oracle as it stands on the other workloads, each rendered whole: the plain
    stereo frame (full resolution, 16x16 tiles, both eyes), the 256^2 10k-Gaussian single
    view in exact order, and the four 1280^2 views of the 500k-Gaussian fine-tuning scene
    (forward render only)."""
    from oracle import native as on
    from paper_2505_10144_gb300 import synth
    out = {"plain_stereo_frame_s": oracle_whole_frame(scene64, frame, fovea=False)}
    sc = synth.tiny_scene(10_000, synth.rng_for(0))
    sc64 = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in sc.arrays()], sc.sh_degree)
    t = time.perf_counter()
    on.render(sc64, synth.identity_camera(256, 256, 90.0), "exact", key_tile=16)
    out["single_view_256_10k_exact_s"] = time.perf_counter() - t
    ft = synth.shell_scene(N_GAUSS, synth.rng_for(3), sh_degree=3)
    ft64 = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in ft.arrays()], ft.sh_degree)
    t = time.perf_counter()
    for cam in synth.ring_views(4, 1280, 1280, 110.0, synth.rng_for(3, salt=1)):
        on.render(ft64, cam, "hier", WINDOWS, 16)
    out["finetune_4x1280_forward_s"] = time.perf_counter() - t
    out["sample"] = "each rendered whole by the FP64 oracle"
    return out


def cpu_model() -> str:
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def oracle_whole_frame(scene64, frame, mode="hier", fovea=True):
    """Seconds of the FP64 oracle, as it stands, for one whole stereo frame (both eyes,
    every sample), foveated (32x32 key tiles) or plain (16x16)."""
    from oracle import native as on
    t = time.perf_counter()
    for e in range(2):
        on.render(scene64, frame.cameras[e], mode, WINDOWS, 32 if fovea else 16, frame.foveas[e] if fovea else None)
    return time.perf_counter() - t


def run_reference(args, ws, rank):
    """The reference arm: the oracle as it stands, on the host cores, same metric: every
    step renders one whole stereo frame of the trajectory (both eyes, every sample)."""
    if rank != 0:
        return
    from paper_2505_10144_gb300 import synth
    scene, wl = make_workload(max(args.steps + args.warmup, 1))
    scene64 = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in scene.arrays()], scene.sh_degree)
    from oracle import native as on
    on.build()
    thr = on.num_threads()
    vals = []
    for i in range(args.warmup + args.steps):
        sec = oracle_whole_frame(scene64, wl.frames[i % len(wl.frames)])
        if i >= args.warmup:
            vals.append(sec)
    mean = statistics.mean(vals)
    value = 1.0 / mean
    desc = ("FP64 oracle, hierarchical 4/8/16, foveated: one whole stereo frame of the trajectory per step "
            "(both eyes, every sample)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "p99_ms": float(np.percentile(vals, 99)) * 1e3,
            "config": {"workload": "vr_stereo_2064x2208_500k_foveated_hier_4_8_16", "n_gaussians": N_GAUSS,
                       "width": W_IMG, "height": H_IMG, "views": 2},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": thr, "kind": "oracle", "sample": desc,
                             "host_cpus": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(args, api, torch):
    """Frames only: the workload at args.scale resolution, nothing else on the GPU (or,
    with --train, periphery-network training steps only)."""
    from paper_2505_10144_gb300 import synth
    if args.sort:
        # keys like the frame's: 14 tile bits over the order-preserving bits of a depth in
        # [0.5, 8) m; values the instance index; checked against a stable argsort
        n = 2_470_000
        rng = np.random.default_rng(5)
        tile = rng.integers(0, 8970, size=n).astype(np.uint64)
        depth = rng.uniform(0.5, 8.0, size=n).astype(np.float32).view(np.uint32).astype(np.uint64) | np.uint64(1 << 31)
        keys = (tile << np.uint64(32)) | depth
        k = torch.from_numpy(keys.view(np.int64)).cuda()
        v = torch.from_numpy(np.arange(n, dtype=np.int32)).cuda()
        R = api.Renderer()
        for _ in range(args.warmup):
            ok, ov = R.sort_pairs(k, v, 46)
        torch.cuda.synchronize()
        assert np.array_equal(ov.cpu().numpy(), np.argsort(keys, kind="stable").astype(np.int32))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(args.steps):
            R.sort_pairs(k, v, 46)
        ev[1].record()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": True, "sort_pairs": n, "bits": 46,
                          "ms_per_sort": ev[0].elapsed_time(ev[1]) / max(args.steps, 1)}))
        R.close()
        return
    if args.train:
        from paper_2505_10144_gb300 import periphery
        R = api.Renderer()
        net = periphery.PeripheryNet(R, seed=4)
        rng = np.random.default_rng(7)
        x = torch.tensor(rng.uniform(0, 1, size=(8, 3, 256, 256)).astype(np.float32)).cuda()
        t = torch.tensor(rng.uniform(0, 1, size=(8, 3, 256, 256)).astype(np.float32)).cuda()
        for _ in range(args.warmup + args.steps):
            y, acts = net.forward(x)
            _, dy = net.mse(y, t)
            net.grad.zero_()
            net.backward(x, acts, dy)
            net.step(1e-3)
        R.check()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": True, "train_steps": args.warmup + args.steps, "batch": 8, "crop": 256}))
        R.close()
        return
    W, H = int(W_IMG * args.scale) // 32 * 32, int(H_IMG * args.scale) // 32 * 32
    scene = synth.shell_scene(N_GAUSS, synth.rng_for(1), sh_degree=3)
    wl = synth.vr_trajectory(args.warmup + args.steps, synth.rng_for(1, salt=100), W, H)
    ds = api.DeviceScene.from_host(scene)
    R = api.Renderer()
    cfg = api.RenderConfig(sort_mode=args.mode, windows=WINDOWS, key_tile=32,
                           fovea_mode="net" if args.net else "bilinear")
    out = torch.empty((2, 3, H, W), device="cuda")
    low = torch.empty((2, 3, H // 2, W // 2), device="cuda") if args.net else None
    net = None
    if args.net:  # the periphery network (random weights: the same work as trained ones)
        from paper_2505_10144_gb300 import periphery
        net = periphery.PeripheryNet(R, seed=4)
    grads = ds.zeros_like() if args.backward else None
    dout = torch.randn((2, 3, H, W), device="cuda", generator=torch.Generator("cuda").manual_seed(7)) * 1e-3 \
        if args.backward else None
    for fr in wl.frames:
        R.render([ds], [0, 0], fr.cameras, fr.foveas, cfg, out=out, low=low, save=args.backward)
        if net is not None:
            net.apply_periphery(low, out)
        if args.backward:  # the replay of the same frame, one backward launch per forward launch
            R.backward([ds], [0, 0], fr.cameras, fr.foveas, cfg, dout, [grads])
    R.check()
    torch.cuda.synchronize()
    st = R.stats()
    if args.stats:  # device counters of the last frame, from one more render with counters on
        fr = wl.frames[-1]
        R.render([ds], [0, 0], fr.cameras, fr.foveas, api.RenderConfig(**{**cfg.__dict__, "stats": True}), out=out, low=low)
        st = R.stats()
    print(json.dumps({"ncu_case": True, "width": W, "height": H, "frames": len(wl.frames), **st}))
    R.close()


def batched_line(api, torch, n_steps, warmup, cache, ws=1, pg=None, quiet=False):
    """Three scenes (200k, 1M, 3M Gaussians) x 8 head poses x 2 eyes = 48 views of
    2064x2208, foveated, in one vrs_render (one sort, one persistent render launch)
    captured in a CUDA graph; the autotuner picks the key-tile size, the windows and the
    CTA cap (the fastest candidate above its PSNR floor against the exact order)."""
    from paper_2505_10144_gb300 import autotune, synth
    sizes = [200_000, 1_000_000, 3_000_000]
    scenes = [api.DeviceScene.from_host(synth.shell_scene(n, synth.rng_for(2, salt=k), sh_degree=3))
              for k, n in enumerate(sizes)]

    def views(step):
        cams, fovs, vs = [], [], []
        for k in range(3):
            for fr in synth.batched_poses(8, synth.rng_for(2, salt=10 + k + 97 * step), W_IMG, H_IMG):
                cams += fr.cameras
                fovs += fr.foveas
                vs += [k, k]
        return cams, fovs, vs

    cams, fovs, vs = views(0)
    R = api.Renderer()
    base = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=32, fovea_mode="bilinear")
    best, cands = autotune.autotune(R, scenes, vs, cams, fovs, base, cache_path=cache, reps=2)
    R.set_tuning(best["max_ctas_per_sm"])
    cfg = api.RenderConfig(sort_mode="hier", windows=tuple(best["windows"]), key_tile=best["key_tile"],
                           fovea_mode="bilinear")
    if not quiet:
        log("autotune candidates (key tile, windows, CTA cap: ms per replay, PSNR vs exact, % pixels > 2e-4):")
        for c in cands:
            log(f"  {c['key_tile']:2d}x{c['key_tile']:<2d} {tuple(c['windows'])} cap {c['max_ctas_per_sm']}: "
                f"{c['ms']:8.2f} ms  {c['psnr_db']:6.2f} dB  {c['over_2e-4_pct']:6.2f} %"
                f"{'' if c['meets_floor'] else '  (below the floor)'}")
        log(f"chosen: {best['key_tile']}x{best['key_tile']} {tuple(best['windows'])} cap {best['max_ctas_per_sm']} "
            f"(floor {best['psnr_floor_db']:.2f} dB)")
    gr = api.GraphedRender(R, scenes, vs, cams, fovs, cfg)
    frames = [views(1 + i) for i in range(n_steps + warmup)]
    for i in range(warmup):
        gr.replay(frames[i][0], frames[i][1])
    torch.cuda.synchronize()
    ms = []
    for i in range(n_steps):
        c, f, _ = frames[warmup + i]
        R.update_views(c, f, cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()  # replay() launches on the current stream
        gr.graph.replay()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    R.check()
    st = R.stats()
    R.close()
    return {"value": job_rate(ws, 48 * len(ms), max_over_ranks(sum(ms), pg)), "unit": "views/s",
            "ms_per_step": statistics.mean(ms), "p99_ms": float(np.percentile(ms, 99)), "steps": len(ms),
            "config": {"workload": "batched_3_scenes_200k_1M_3M_48_views_foveated", "views": 48,
                       "gaussians": sizes, "graph": "one vrs_render captured in a CUDA graph, poses via vrs_update_views"},
            "autotune": {"best": {k: best[k] for k in ("key_tile", "windows", "max_ctas_per_sm", "ms", "psnr_db",
                                                       "over_2e-4_pct")},
                         "psnr_floor_db": best["psnr_floor_db"], "reference": best["reference"],
                         "candidates": cands},
            "instances_per_batch": st["instances"], "work_items": st["work_items"],
            "gpu_launches": st["kernels"] * len(ms)}


def run_batched(args, api, torch, ws, rank, pg=None):
    """The batched workload as its own line (see batched_line)."""
    cache = args.tune_cache or os.path.join(ROOT, "_build", "autotune.json")
    b = batched_line(api, torch, max(args.steps // 10, 3), args.warmup, cache, ws, pg)
    line = {"metric": "batched views/s (3 scenes x 8 poses x 2 eyes, 2064x2208, one graph replay)",
            "value": b["value"], "unit": "views/s", "n_gpus": ws, "steps": b["steps"], "warmup": args.warmup,
            "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", **{k: v for k, v in b.items() if k not in ("value", "steps")}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_finetune(args, api, torch, ws, rank, pg=None):
    """Fine-tuning step through the rasterizer: 500k Gaussians, 4 views of 1280x1280,
    110 deg FOV, 0.8 L1 + 0.2 (1 - SSIM), gradients for every parameter, Adam.  The
    targets are renders of a perturbed copy of the scene (means + N(0, 0.01), log-scales +
    N(0, 0.1)) made by this renderer; the oracle pins the gradients in the tests.
    With N ranks the step is data-parallel over views: each rank renders 4 views of its
    own, and one all-reduce of the flat gradient buffer averages the gradients before
    every rank takes the same Adam step."""
    from paper_2505_10144_gb300 import synth
    scene = synth.shell_scene(N_GAUSS, synth.rng_for(3), sh_degree=3)
    cams = synth.ring_views(4, 1280, 1280, 110.0, synth.rng_for(3, salt=1 + 1000 * rank))
    target_scene = synth.perturbed(scene, synth.rng_for(3, salt=2))
    R = api.Renderer()
    cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=16)
    target = R.render([api.DeviceScene.from_host(target_scene)], [0] * 4, cams, None, cfg).clone()
    names = ["mean", "log_scale", "quat", "opacity_logit", "sh"]
    params = {k: torch.tensor(np.asarray(v), device="cuda") for k, v in zip(names, scene.arrays())}
    lrs = {"mean": 1.6e-4, "log_scale": 5e-3, "quat": 1e-3, "opacity_logit": 5e-2, "sh": 2.5e-3}
    opt = api.Adam(params, lrs)
    ds = api.DeviceScene(*[params[k] for k in names], 3)
    grads, gflat = ds.flat_zeros_like()

    def step():
        img = R.render([ds], [0] * 4, cams, None, cfg, save=True)
        loss, dimg = R.loss(img, target)
        gflat.zero_()
        R.backward([ds], [0] * 4, cams, None, cfg, dimg, [grads])
        api.average_gradients(gflat, pg)
        opt.step(dict(zip(names, grads.tensors())))
        return loss

    losses = []
    for _ in range(args.warmup):
        losses.append(float(step().item()))
    torch.cuda.synchronize()
    steps = max(args.steps // 4, 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        loss = step()
    e1.record()
    torch.cuda.synchronize()
    losses.append(float(loss.item()))
    ms = e0.elapsed_time(e1) / steps
    R.check()
    line = {"metric": "fine-tuning steps/s (4 views 1280x1280, 500k Gaussians, render+loss+backward+Adam)",
            "value": job_rate(ws, steps, max_over_ranks(ms * steps, pg)), "unit": "steps/s", "n_gpus": ws,
            "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "finetune_500k_4x1280", "windows": list(WINDOWS),
                                            "parallelism": f"dp{ws} over views" + (
                                                ", one gradient all-reduce per step" if ws > 1 else "")},
            "loss_first": losses[0], "loss_last": losses[-1]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()


def run_net(args, api, torch, ws, rank, pg=None):
    """Learned periphery: 1M Gaussians (room shell, SH degree 3), stereo 2064x2208,
    periphery at 1/4 of the pixels.  The network is trained on the GPU (library kernels)
    on 2000 seeded pose pairs (256x256 crops of random head poses: half-resolution
    foveated render -> plain full-resolution render) and evaluated on 200 held-out stereo
    frames against the plain render, next to its bilinear fallback; then frames/s of the
    foveated + network frame."""
    from paper_2505_10144_gb300 import periphery, synth
    R = api.Renderer()
    scene = api.DeviceScene.from_host(synth.shell_scene(1_000_000, synth.rng_for(4), sh_degree=3))
    t0 = time.perf_counter()
    xs, ts = periphery.make_pairs(R, scene, 2000, np.random.default_rng(synth.BASE_SEED + 4), crop=256,
                                  sort_mode="hier")
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = periphery.PeripheryNet(R, seed=4, zero_last=True)
    t0 = time.perf_counter()
    losses = periphery.train(net, xs, ts, steps=2000, batch=8, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del xs, ts
    frames = synth.vr_trajectory(200, synth.rng_for(4, salt=200)).frames
    ev = periphery.evaluate_frames(R, net, scene, frames[:: max(1, 200 // max(args.steps, 1))] if args.steps < 200 else frames)
    # frame timing: foveated render + network on the periphery tiles, vs plain
    net_cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=32, fovea_mode="net")
    plain_cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=16, fovea_mode="plain")
    out = torch.empty((2, 3, H_IMG, W_IMG), device="cuda")
    low = torch.empty((2, 3, H_IMG // 2, W_IMG // 2), device="cuda")

    def timed(fn, n):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        ms = []
        for i in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(i)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    def fnet(i):
        fr = frames[i % len(frames)]
        R.render([scene], [0, 0], fr.cameras, fr.foveas, net_cfg, out=out, low=low)
        net.apply_periphery(low, out)

    def fplain(i):
        fr = frames[i % len(frames)]
        R.render([scene], [0, 0], fr.cameras, None, plain_cfg, out=out)

    n = max(args.steps // 4, 10)
    ms_net, ms_plain = timed(fnet, n), timed(fplain, n)
    R.check()
    line = {"metric": "stereo frames/s with the learned periphery (1M Gaussians, 2x2064x2208) and its PSNR vs plain",
            "value": job_rate(ws, len(ms_net), max_over_ranks(sum(ms_net), pg)), "unit": "frames/s",
            "n_gpus": ws, "steps": len(ms_net),
            "warmup": 3, "ms_per_step": statistics.mean(ms_net), "p99_ms": float(np.percentile(ms_net, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 network, f32 render",
            "data": "synthetic", "config": {"workload": "learned_periphery_1M_stereo", "train_pairs": 2000,
                                            "train_steps": 2000, "eval_frames": len(frames)},
            "plain": {"value": len(ms_plain) / (sum(ms_plain) / 1e3), "ms_per_step": statistics.mean(ms_plain),
                      "p99_ms": float(np.percentile(ms_plain, 99))},
            "quality_vs_plain": ev, "train_loss_first": float(losses[:50].mean()),
            "train_loss_last": float(losses[-50:].mean()), "pairs_s": t_pairs, "train_s": t_train}
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()


# FLOPs of the periphery network per reconstructed pixel: 3x3 convolutions 3 -> 32 -> 32 -> 3
# (3*32*9 + 32*32*9 + 32*3*9 = 10,944 multiply-adds)
NET_FLOP_PER_PX = 2 * (3 * 32 * 9 + 32 * 32 * 9 + 32 * 3 * 9)
WEIGHTS = os.path.join(ROOT, "paper_2505_10144_gb300", "weights", "periphery_1m.npy")


def learned_periphery(api, torch, n_steps, warmup):
    """The learned-periphery frame: 1M Gaussians (room shell, SH degree 3), stereo
    2064x2208, periphery at 1/4 of the pixels reconstructed by the BF16 network (weights
    trained by the library's kernels: paper_2505_10144_gb300/train_periphery.py).
    Frames/s and p99 of foveated render + network against the plain full-resolution
    render of the same scene, and PSNR / maximum error of the network and of its bilinear
    fallback against the plain render on 200 held-out trajectory frames."""
    from paper_2505_10144_gb300 import periphery, synth
    if not os.path.exists(WEIGHTS):
        return {"unavailable": "no trained weights at paper_2505_10144_gb300/weights/periphery_1m.npy"}
    R = api.Renderer()
    scene = api.DeviceScene.from_host(synth.shell_scene(1_000_000, synth.rng_for(4), sh_degree=3))
    net = periphery.PeripheryNet(R, seed=4)
    net.params.copy_(torch.from_numpy(np.load(WEIGHTS)).cuda())
    frames = synth.vr_trajectory(200, synth.rng_for(4, salt=200)).frames
    net_cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=32, fovea_mode="net")
    plain_cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=16, fovea_mode="plain")
    out = torch.empty((2, 3, H_IMG, W_IMG), device="cuda")
    low = torch.empty((2, 3, H_IMG // 2, W_IMG // 2), device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")

    def timed(fn, n):
        for i in range(warmup):
            fn(i)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n)]
        for i in range(n):
            flush.zero_()
            fn(warmup + i, ev[i])
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, _, c in ev], [b.elapsed_time(c) for _, b, c in ev]

    def fnet(i, ev=None):
        fr = frames[i % len(frames)]
        if ev:
            ev[0].record()
        R.render([scene], [0, 0], fr.cameras, fr.foveas, net_cfg, out=out, low=low)
        if ev:
            ev[1].record()
        net.apply_periphery(low, out)
        if ev:
            ev[2].record()

    def fplain(i, ev=None):
        fr = frames[i % len(frames)]
        if ev:
            ev[0].record()
            ev[1].record()
        R.render([scene], [0, 0], fr.cameras, None, plain_cfg, out=out)
        if ev:
            ev[2].record()

    ms_net, ms_netk = timed(fnet, n_steps)
    ms_plain, _ = timed(fplain, n_steps)
    R.check()
    ev = periphery.evaluate_frames(R, net, scene, frames)
    # the same in the exact per-ray order (reconstruction error only) on every 25th frame
    ev_exact = periphery.evaluate_frames(R, net, scene, frames[::25], sort_mode="exact")
    R.check()
    px = statistics.mean(periphery_pixels(frames[(warmup + i) % len(frames)]) for i in range(n_steps))
    k_ms = statistics.mean(ms_netk)
    tfl = NET_FLOP_PER_PX * px / (k_ms / 1e3) / 1e12
    rp = roofline_peaks()
    meta = {}
    try:
        with open(WEIGHTS[:-4] + ".json") as fh:
            meta = json.load(fh)
    except (OSError, ValueError):
        pass
    del scene
    train_step = network_training_step(R, periphery, torch, rp)
    R.close()
    return {"value": len(ms_net) / (sum(ms_net) / 1e3), "unit": "frames/s", "ms_per_step": statistics.mean(ms_net),
            "p50_ms": float(np.percentile(ms_net, 50)), "p99_ms": float(np.percentile(ms_net, 99)),
            "plain": {"value": len(ms_plain) / (sum(ms_plain) / 1e3), "ms_per_step": statistics.mean(ms_plain),
                      "p99_ms": float(np.percentile(ms_plain, 99)),
                      "config": "1M Gaussians, full resolution, 16x16 tiles, hierarchical 4/8/16"},
            "speedup_vs_plain": statistics.mean(ms_plain) / statistics.mean(ms_net),
            "quality_vs_plain_exact_order": {**ev_exact, "frames": len(frames[::25]),
                                             "gain_db": ev_exact["net_periph_psnr_db"] - ev_exact["bil_periph_psnr_db"],
                                             "note": "foveated and plain renders in the exact per-ray order: the "
                                                     "periphery error is what reconstruction from half resolution "
                                                     "loses; periphery pixels (32x32 tiles outside radius + band) and "
                                                     "whole frames; net = BF16 network, bil = its bilinear fallback"},
            "quality_vs_plain_hier": {**ev, "frames": len(frames),
                                      "gain_db": ev["net_periph_psnr_db"] - ev["bil_periph_psnr_db"],
                                      "note": "as timed: hierarchical 4/8/16 windows on 32x32 tiles (foveated) "
                                              "against 16x16 tiles (plain), whose window approximations differ"},
            "net_kernel_roofline": {"bound": "tensor", "kernel": "net_periphery_kernel (tcgen05.mma BF16 -> FP32)",
                                    "achieved": tfl, "peak": rp["bf16_tflops_sustained"], "unit": "TFLOP/s",
                                    "frac": tfl / rp["bf16_tflops_sustained"], "avg_launch_ms": k_ms,
                                    "algorithmic_flops": NET_FLOP_PER_PX * px,
                                    "basis": f"{NET_FLOP_PER_PX} FLOP per reconstructed periphery pixel x {px:.0f} "
                                             "pixels (halo recompute not counted); peak: sustained BF16 "
                                             + rp["source"]},
            "weights": "paper_2505_10144_gb300/weights/periphery_1m.npy", "training": meta,
            "training_step": train_step,
            "config": {"workload": "learned_periphery_1M_stereo_2064x2208", "timing": "CUDA events per frame, "
                       "eager render + network launch, L2 flushed between frames"}}


# multiply-adds per pixel of one training step: forward 27x32 + 288x32 + 288x3, data
# gradients 27x32 (through w3) + 288x32 (through w2), weight gradients 288x3 + 288x32 + 27x32
TRAIN_FLOP_PER_PX = 2 * ((27 * 32 + 288 * 32 + 288 * 3) + (27 * 32 + 288 * 32) + (288 * 3 + 288 * 32 + 27 * 32))


def network_training_step(R, periphery, torch, rp, batch=8, size=256, steps=30, warmup=5):
    """One training step of the periphery network as train_periphery runs it (batch 8 of
    256x256 crops): forward, MSE, backward and Adam, every contraction on the tensor cores.
    Timed with CUDA events over `steps` steps on seeded synthetic images (the time does
    not depend on the values), with the tensor roofline of its algorithmic FLOPs."""
    net = periphery.PeripheryNet(R, seed=4)
    rng = np.random.default_rng(7)
    x = torch.tensor(rng.uniform(0, 1, size=(batch, 3, size, size)).astype(np.float32)).cuda()
    t = torch.tensor(rng.uniform(0, 1, size=(batch, 3, size, size)).astype(np.float32)).cuda()

    def step():
        y, acts = net.forward(x)
        _, dy = net.mse(y, t)
        net.grad.zero_()
        net.backward(x, acts, dy)
        net.step(1e-3)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    R.check()
    ms = e0.elapsed_time(e1) / steps
    flops = TRAIN_FLOP_PER_PX * batch * size * size
    tfl = flops / (ms * 1e-3) / 1e12
    return {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "batch": batch, "crop": size,
            "roofline": {"bound": "tensor", "achieved": tfl, "peak": rp["bf16_tflops_sustained"], "unit": "TFLOP/s",
                         "frac": tfl / rp["bf16_tflops_sustained"], "algorithmic_flops": flops,
                         "basis": f"{TRAIN_FLOP_PER_PX} FLOP per pixel (forward, data and weight gradients, no "
                                  "padding counted) over the step's CUDA-event time, MSE and Adam included; peak: "
                                  "sustained BF16 " + rp["source"]},
            "kernels": "conv_tc_kernel (forward layers, data gradients), wgrad_tc_kernel (weight gradients): "
                       "tcgen05.mma BF16 -> FP32"}


GRAD_BYTES_PER_BLEND = 64  # each blended pair adds its 16 record-gradient floats with four 16-byte atomics


def backward_line(api, torch, warmup, n_steps, peaks):
    """The fine-tuning step of the workload (500k Gaussians, 4 views of 1280x1280, 0.8 L1 +
    0.2 (1 - SSIM), every parameter, Adam) and its backward render's roofline: the replay
    of each blended pair adds 64 bytes of record gradient by vector atomics in L2, against
    the measured L2 read bandwidth (the atomics' unit); and the issue basis of the replay
    (the forward's 36 lane-ops per evaluated pair again, about twice that per blended pair
    for the gradient)."""
    from paper_2505_10144_gb300 import synth
    scene = synth.shell_scene(N_GAUSS, synth.rng_for(3), sh_degree=3)
    cams = synth.ring_views(4, 1280, 1280, 110.0, synth.rng_for(3, salt=1))
    target_scene = synth.perturbed(scene, synth.rng_for(3, salt=2))
    R = api.Renderer()
    cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=16)
    target = R.render([api.DeviceScene.from_host(target_scene)], [0] * 4, cams, None, cfg).clone()
    names = ["mean", "log_scale", "quat", "opacity_logit", "sh"]
    params = {k: torch.tensor(np.asarray(v), device="cuda") for k, v in zip(names, scene.arrays())}
    opt = api.Adam(params, {"mean": 1.6e-4, "log_scale": 5e-3, "quat": 1e-3, "opacity_logit": 5e-2, "sh": 2.5e-3})
    ds = api.DeviceScene(*[params[k] for k in names], 3)
    grads, gflat = ds.flat_zeros_like()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_steps)]

    def step(e=None):
        if e:
            e[0].record()
        img = R.render([ds], [0] * 4, cams, None, cfg, save=True)
        loss, dimg = R.loss(img, target)
        gflat.zero_()
        if e:
            e[1].record()
        R.backward([ds], [0] * 4, cams, None, cfg, dimg, [grads])
        if e:
            e[2].record()
        opt.step(dict(zip(names, grads.tensors())))
        return loss

    l0 = float(step().item())
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(n_steps):
        loss = step(ev[i])
    e1.record()
    torch.cuda.synchronize()
    R.check()
    ms = e0.elapsed_time(e1) / n_steps
    bwd_ms = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    R.render([ds], [0] * 4, cams, None, api.RenderConfig(**{**cfg.__dict__, "stats": True}))
    st = R.stats()
    R.close()
    gbs = GRAD_BYTES_PER_BLEND * st["blended"] / (bwd_ms / 1e3) / 1e9
    return {"value": 1e3 / ms, "unit": "steps/s", "ms_per_step": ms, "loss_first": l0, "loss_last": float(loss.item()),
            "backward_ms": bwd_ms,
            "backward_roofline": {"bound": "l2", "achieved": gbs, "peak": peaks["l2_read_gbs"], "unit": "GB/s",
                                  "frac": gbs / peaks["l2_read_gbs"],
                                  "basis": f"{GRAD_BYTES_PER_BLEND} B of record-gradient atomics per blended pair x "
                                           f"{st['blended']} blended pairs of the four views; peak: measured L2 read "
                                           "bandwidth (vrs_measure_peaks)",
                                  "work": {"evaluated_pairs": st["evaluated"], "kept_pairs": st["kept"],
                                           "blended_pairs": st["blended"]}},
            "config": {"workload": "finetune_500k_4x1280", "step": "render (saved) + loss + backward + Adam",
                       "timing": "CUDA events; backward_ms is the vrs_render_backward call alone"}}


REUSE_FAR_M = 92.0  # 0.25 px of eye-to-cyclopean disparity at f = 722.6 and IPD 64 mm


def stereo_reuse(api, torch, n_steps, warmup):
    """Stereo reuse of distant content (Sec. 7's future work): an open room (500k
    Gaussians, no ceiling, no front wall) with a landscape of 200k Gaussians at 150-600 m,
    plain stereo 2064x2208, hierarchical 4/8/16.  The fused stereo render (both eyes,
    every Gaussian) against vrs_render_stereo_reuse (near layer per eye, far layer once from
    the cyclopean eye), and the reuse image's PSNR against the fused one."""
    from paper_2505_10144_gb300 import synth
    scene = synth.open_room_with_landscape(500_000, 200_000, synth.rng_for(5), sh_degree=3)
    ds = api.DeviceScene.from_host(scene)
    wl = synth.vr_trajectory(warmup + n_steps, synth.rng_for(5, salt=3), W_IMG, H_IMG)
    cfg = api.RenderConfig(sort_mode="hier", windows=WINDOWS, key_tile=16)
    R = api.Renderer()
    out = torch.empty((2, 3, H_IMG, W_IMG), device="cuda")
    out2 = torch.empty_like(out)
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")

    def timed(fn):
        for i in range(warmup):
            fn(i, out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        for i in range(n_steps):
            flush.zero_()
            ev[i][0].record()
            fn(warmup + i, out)
            ev[i][1].record()
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    def fused(i, o):
        fr = wl.frames[i]
        R.render([ds], [0, 0], fr.cameras, None, cfg, out=o)

    def reuse(i, o):
        R.render_stereo_reuse(ds, wl.frames[i].cameras, REUSE_FAR_M, cfg, out=o)

    ms_fused, ms_reuse = timed(fused), timed(reuse)
    ps = []
    for i in range(0, n_steps, max(1, n_steps // 8)):
        fused(i, out2)
        reuse(i, out)
        ps.append(psnr(out, out2))
    R.check()
    n_far = 200_000
    R.close()
    return {"value": len(ms_reuse) / (sum(ms_reuse) / 1e3), "unit": "frames/s",
            "ms_per_step": statistics.mean(ms_reuse), "p99_ms": float(np.percentile(ms_reuse, 99)),
            "fused_stereo": {"value": len(ms_fused) / (sum(ms_fused) / 1e3), "ms_per_step": statistics.mean(ms_fused),
                             "p99_ms": float(np.percentile(ms_fused, 99))},
            "speedup": statistics.mean(ms_fused) / statistics.mean(ms_reuse),
            "psnr_vs_fused_db": statistics.mean(ps), "far_distance_m": REUSE_FAR_M,
            "config": {"workload": "open room 500k + landscape 200k at 150-600 m, plain stereo 2064x2208, "
                                   "hierarchical 4/8/16, 16x16 key tiles", "far_gaussians": n_far,
                       "timing": "CUDA events per eager stereo frame, L2 flushed between frames"}}


def approximation_error(R, api, ds, frame, cfg_hier, torch):
    """Error of the hierarchical per-ray windows against the exact per-ray order on one
    foveated stereo frame (both on the GPU; the exact order is the parity-checked mode)."""
    exact_cfg = api.RenderConfig(**{**cfg_hier.__dict__, "sort_mode": "exact"})
    a = R.render([ds], [0, 0], frame.cameras, frame.foveas, cfg_hier).clone()
    b = R.render([ds], [0, 0], frame.cameras, frame.foveas, exact_cfg)
    d = (a - b).abs()
    mse = float((d ** 2).mean())
    return {"mean_abs": float(d.mean()), "max_abs": float(d.max()),
            "psnr_db": float("inf") if mse == 0 else 10 * math.log10(1.0 / mse),
            "pixels_over_2e-4_pct": float((d.amax(dim=1) > 2e-4).float().mean() * 100)}


RENDER_SOURCES = ["paper_2505_10144_gb300/csrc/render.cu", "paper_2505_10144_gb300/csrc/common.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "render_traffic_vr_stereo_500k.txt")


def render_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in RENDER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the render kernel from the committed ncu summary, or None
    when the kernel's source changed since that capture (or there is none)."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != render_source_hash():
            return None, "render source changed since the ncu capture", None, None
        issue = float(kv["issue_slots_busy_pct"]) / 100.0 if "issue_slots_busy_pct" in kv else None
        ipp = float(kv["thread_inst_per_evaluated_pair"]) if "thread_inst_per_evaluated_pair" in kv else None
        return float(kv["dram_bytes_per_launch"]), kv.get("capture", ""), issue, ipp
    except (OSError, KeyError, ValueError):
        return None, "no ncu traffic summary", None, None


def order_flips(ids_a, len_a, ids_b, len_b, torch, batch=256):
    """Frame-to-frame order flips of probe rays: for each probe, the pairs of Gaussians
    blended in both frames whose front-to-back order differs (the Kendall distance of the
    two blend orders restricted to their common Gaussians).  ids [P, L] int32 padded,
    len [P].  Returns (total flips, probes with a flip, common pairs)."""
    P, L = ids_a.shape
    ar = torch.arange(L, device=ids_a.device)
    flips = flipped = common = 0
    upper = ar[:, None] < ar[None, :]
    for s0 in range(0, P, batch):
        a, b = ids_a[s0:s0 + batch].long(), ids_b[s0:s0 + batch].long()
        va = ar[None, :] < len_a[s0:s0 + batch, None].clamp(max=L)
        vb = ar[None, :] < len_b[s0:s0 + batch, None].clamp(max=L)
        m = (a[:, :, None] == b[:, None, :]) & va[:, :, None] & vb[:, None, :]
        has = m.any(-1)
        pos = torch.where(has, m.float().argmax(-1), torch.full_like(a, -1))
        both = has[:, :, None] & has[:, None, :] & upper[None]
        inv = both & (pos[:, :, None] > pos[:, None, :])
        per = inv.sum((1, 2))
        flips += int(per.sum())
        flipped += int((per > 0).sum())
        common += int(both.sum())
    return flips, flipped, common


def popping(api, ds, wl, cfg, torch, n_steps=12, grid=16, max_len=512):
    """Popping of an order as order flips on unchanged world rays.  Each step takes eye
    0 of a trajectory frame (camera A) and the next frame's viewing rotation about the
    same eye position (camera B).  Rays through the pixel centres of a grid of A are
    probed in A and, at the image points where the same world rays land, in B
    (vrs_probe_orders); a flip is a pair of Gaussians the ray blends in both in the
    opposite order.  A per-ray order depends on the ray alone, so it cannot flip here
    (up to FP32 near-ties); an order keyed per Gaussian by the viewing direction can."""
    from paper_2505_10144_gb300 import synth
    ys, xs = np.mgrid[grid // 2:H_IMG:grid, grid // 2:W_IMG:grid]
    px, py = xs.ravel() + 0.5, ys.ravel() + 0.5
    steps = []
    for f in range(n_steps):
        ca, nxt = wl.frames[f].cameras[0], wl.frames[f + 1].cameras[0]
        Ra = ca.world_to_cam[:, :3].astype(np.float64)
        cb = synth.camera_from_pose(nxt.world_to_cam[:, :3].astype(np.float64).T, ca.center(), ca.width, ca.height,
                                    ca.fx, ca.fy, ca.near_z, ca.cx, ca.cy)
        Rb = cb.world_to_cam[:, :3].astype(np.float64)
        d = np.stack([(px - ca.cx) / ca.fx, (py - ca.cy) / ca.fy, np.ones_like(px)])
        db = Rb @ (Ra.T @ d)
        z = np.where(db[2] > 1e-6, db[2], 1.0)
        qx, qy = ca.fx * db[0] / z + ca.cx, ca.fy * db[1] / z + ca.cy
        inside = (db[2] > 1e-6) & (qx >= 0) & (qx < W_IMG) & (qy >= 0) & (qy < H_IMG)
        pa = np.stack([np.zeros(inside.sum()), px[inside], py[inside]], 1)
        pb = np.stack([np.zeros(inside.sum()), qx[inside], qy[inside]], 1)
        ang = np.degrees(np.arccos(np.clip((np.trace(Rb @ Ra.T) - 1) / 2, -1, 1)))
        steps.append((ca, cb, wl.frames[f].foveas[0], torch.tensor(pa, dtype=torch.float32, device="cuda"),
                      torch.tensor(pb, dtype=torch.float32, device="cuda"), ang))
    R = api.Renderer()
    out = {}
    for mode in ("exact", "global_z", "global_dist"):
        mcfg = api.RenderConfig(**{**cfg.__dict__, "sort_mode": mode})
        tot = {"flips": 0, "flipped": 0, "common": 0, "blended": 0, "truncated": 0, "rays": 0}
        for ca, cb, fv, pa, pb, _ in steps:
            R.render([ds], [0], [ca], [fv], mcfg)
            ids_a, _, la = R.probe_orders(pa, max_len)
            R.render([ds], [0], [cb], [fv], mcfg)
            ids_b, _, lb = R.probe_orders(pb, max_len)
            R.check()
            fl, fp, cm = order_flips(ids_a, la, ids_b, lb, torch)
            tot["flips"] += fl
            tot["flipped"] += fp
            tot["common"] += cm
            tot["blended"] += int(la.clamp(min=0).sum())
            tot["truncated"] += int((la > max_len).sum() + (lb > max_len).sum())
            tot["rays"] += pa.shape[0]
        n = max(tot["rays"], 1)
        out[mode] = {"flips_per_ray_per_step": tot["flips"] / n, "rays_with_flip_pct": 100.0 * tot["flipped"] / n,
                     "flipped_pairs_pct": 100.0 * tot["flips"] / max(tot["common"], 1),
                     "blended_per_ray": tot["blended"] / n, "truncated_rays": tot["truncated"]}
    R.close()
    out["config"] = (f"{n_steps} steps of the trajectory (72 Hz), each the next frame's viewing rotation about the "
                     f"same eye position (mean {np.mean([s[5] for s in steps]):.2f} deg); rays through the pixel "
                     f"centres of a {grid}-pixel grid of eye 0 that stay in view ({tot['rays'] // n_steps} per step), "
                     f"foveated frames")
    return out


def grid_flicker(api, ds, wl, torch, n_steps=12):
    """Popping of the image on unchanged world rays, for every order including the
    hierarchical windows.  A head rotation moves the content across the image, so the
    tile and block grid of the next frame sits elsewhere on the same rays.  Each step
    renders eye 0 of a trajectory frame (camera A) and the same camera with its principal
    point moved by the image motion of that frame step rounded to whole pixels (camera
    B: its pixel (x, y) looks along A's ray through (x + dx, y + dy)), and compares the
    two images on their common rays.  The per-ray orders (exact, view-space z, distance)
    depend on the ray alone and cannot change (up to FP32 noise of the shifted principal
    point); the hierarchical windows see other tile lists and blocks, so their result on
    a ray may change: that is the method's residual flicker (Sec. 7)."""
    from paper_2505_10144_gb300 import synth
    R = api.Renderer()
    steps = []
    for f in range(n_steps):
        ca, nxt = wl.frames[f].cameras[0], wl.frames[f + 1].cameras[0]
        Ra = ca.world_to_cam[:, :3].astype(np.float64)
        Rb = nxt.world_to_cam[:, :3].astype(np.float64)
        db = Rb @ (Ra.T @ np.array([0.0, 0.0, 1.0]))
        dx = int(round(ca.fx * db[0] / db[2])) or 1
        dy = int(round(ca.fy * db[1] / db[2]))
        steps.append((ca, wl.frames[f].foveas[0], dx, dy))
    out = {}
    for mode, fov in (("hier", False), ("hier", True), ("exact", False), ("global_z", False), ("global_dist", False)):
        cfg = api.RenderConfig(sort_mode=mode, windows=WINDOWS, key_tile=32 if fov else 16,
                               fovea_mode="bilinear" if fov else "plain")
        changed = tot = 0
        sad = 0.0
        sq = 0.0
        for ca, fv, dx, dy in steps:
            W, H = ca.width, ca.height
            cb = crop_camera(ca, dx, dy, W, H)
            fb = synth.Fovea(fv.gaze_x - dx, fv.gaze_y - dy, fv.radius_px, fv.band_px)
            a = R.render([ds], [0], [ca], [fv] if fov else None, cfg).clone()[0]
            b = R.render([ds], [0], [cb], [fb] if fov else None, cfg)[0]
            xa0, xa1 = max(dx, 0), W + min(dx, 0)
            ya0, ya1 = max(dy, 0), H + min(dy, 0)
            d = (a[:, ya0:ya1, xa0:xa1] - b[:, ya0 - dy:ya1 - dy, xa0 - dx:xa1 - dx]).abs()
            changed += int((d.amax(dim=0) > 2e-4).sum())
            tot += d.shape[1] * d.shape[2]
            sad += float(d.sum())
            sq += float((d ** 2).sum())
        R.check()
        mse = sq / (3 * tot)
        out[mode + ("_foveated" if fov else "")] = {
            "pixels_changed_over_2e-4_pct": 100.0 * changed / tot, "mean_abs": sad / (3 * tot),
            "psnr_db": float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)}
    R.close()
    out["config"] = (f"{n_steps} trajectory steps of eye 0; principal point moved by the step's image motion "
                     f"(mean |d| {np.mean([math.hypot(s[2], s[3]) for s in steps]):.1f} px); common rays compared; "
                     "plain 16x16 tiles, and foveated 32x32 with the gaze on the same ray")
    return out


def psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)


def roofline_peaks():
    """Denominators: the measured HBM copy bandwidth and BF16 GEMM throughputs of
    the GB300s (MEASURED_PEAKS.json at the repository root), else the profiling
    recipe's fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return {"hbm_gbs": float(m["hbm_gbs"]), "bf16_tflops": float(m["bf16_tflops"]),
                "bf16_tflops_sustained": float(m.get("bf16_tflops_sustained", m["bf16_tflops"])),
                "source": "of measured (MEASURED_PEAKS.json: STREAM-style copy, cuBLAS bf16 GEMM)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "of fallback (profiling recipe: 6.8 TB/s, 1.9 PFLOP/s bf16 burst, 1.7 sustained)"}


def periphery_pixels(frame, W=W_IMG, H=H_IMG) -> int:
    """Full-resolution pixels of the periphery 32x32 tiles of a stereo frame (the tiles
    whose pixel centres are all at distance >= radius + band from the gaze, Sec. 4.3):
    the pixels the composite upsamples and the network reconstructs."""
    n = 0
    for fv in frame.foveas:
        ty, tx = np.mgrid[0:(H + 31) // 32, 0:(W + 31) // 32]
        x0, y0 = tx * 32 + 0.5, ty * 32 + 0.5
        x1, y1 = np.minimum((tx + 1) * 32, W) - 0.5, np.minimum((ty + 1) * 32, H) - 0.5
        nx = np.clip(np.float32(fv.gaze_x), x0, x1) - np.float32(fv.gaze_x)
        ny = np.clip(np.float32(fv.gaze_y), y0, y1) - np.float32(fv.gaze_y)
        per = np.sqrt(nx * nx + ny * ny) >= np.float32(fv.radius_px) + np.float32(fv.band_px)
        n += int(((np.minimum((tx + 1) * 32, W) - tx * 32) * (np.minimum((ty + 1) * 32, H) - ty * 32))[per].sum())
    return n


# algorithmic bytes per unit of the HBM-bound stages (one stereo frame, V views, N
# Gaussians, K instances): the preprocess reads each Gaussian's 236 parameter bytes
# (SH degree 3) once for both eyes and writes a 96-byte record and a 4-byte tile count
# per (view, Gaussian); the scan reads the counts and writes the offsets (8 bytes per
# (view, Gaussian)); duplication writes a 12-byte (key, value) instance; the onesweep
# sort reads 8 bytes of histogram input and moves 24 bytes (key and value in and out)
# per pass per instance; the tile ranges read each 8-byte key; the composite reads a
# 12-byte half-resolution sample and writes a 12-byte pixel per periphery pixel.
PARAM_BYTES, RECORD_BYTES, COUNT_BYTES = 236, 96, 4
INSTANCE_BYTES, SORT_PASS_BYTES, SORT_HIST_BYTES = 12, 24, 8


def stage_rooflines(stages_ms, cnt, n_views, n_gauss, passes, periph_px, hbm_gbs, src):
    """Achieved algorithmic GB/s of every HBM-bound stage of the frame against the HBM peak."""
    K = cnt["instances"]
    work = {
        "preprocess": PARAM_BYTES * n_gauss + n_views * n_gauss * (RECORD_BYTES + COUNT_BYTES),
        "scan": n_views * n_gauss * 2 * COUNT_BYTES,
        "duplicate": INSTANCE_BYTES * K,
        "sort": (SORT_HIST_BYTES + passes * SORT_PASS_BYTES) * K,
        "ranges_workitems": 8 * K,
        "composite": 24 * periph_px,
    }
    out = {}
    for k, b in work.items():
        ms = stages_ms.get(k, 0.0)
        gbs = b / (ms / 1e3) / 1e9 if ms > 0 else None
        out[k] = {"bound": "hbm", "ms": ms, "algorithmic_bytes": b, "achieved": gbs, "peak": hbm_gbs,
                  "unit": "GB/s", "frac": gbs / hbm_gbs if gbs else None}
    out["note"] = (f"algorithmic bytes per stereo frame ({n_views} views, {n_gauss} Gaussians, {K:.0f} instances, "
                   f"{passes} sort passes, {periph_px} periphery pixels), stage times from CUDA events around each "
                   f"stage of eager frames; peak {src}")
    return out


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
    ap.add_argument("--backward", action="store_true", help="--ncu-case: also run the backward pass of every frame")
    ap.add_argument("--stats", action="store_true", help="--ncu-case: print the device counters of the last frame")
    ap.add_argument("--net", action="store_true", help="--ncu-case: learned periphery (network on the periphery)")
    ap.add_argument("--train", action="store_true",
                    help="--ncu-case: periphery-network training steps only (batch 8 of 256x256 crops)")
    ap.add_argument("--sort", action="store_true",
                    help="--ncu-case: the radix sort alone, on 2.47 M 46-bit (tile | depth) keys (the VR "
                         "frame's instance count), warmup + steps sorts")
    ap.add_argument("--workload", default="vr", choices=["vr", "batched", "finetune", "net"],
                    help="vr: the headline stereo frame; batched: 3 scenes x 8 poses x 2 eyes in one graph "
                         "replay; finetune: 4 views at 1280^2, render + loss + backward + Adam")
    ap.add_argument("--tune-cache", default=None, help="autotuner JSON cache for --workload batched")
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
    if args.workload == "batched":
        run_batched(args, api, torch, ws, rank, pg)
        return
    if args.workload == "finetune":
        run_finetune(args, api, torch, ws, rank, pg)
        return
    if args.workload == "net":
        run_net(args, api, torch, ws, rank, pg)
        return
    # measured denominators of the render roofline (microbenchmarks, a few ms each)
    peaks = api.measure_peaks()
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

    def timed_eager(cfg, steps, profile=False):
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

    def graphed(cfg, visible=None):
        """A frame as one CUDA-graph replay (own context), its instance workspace sized
        by the largest count over the camera path (an untimed eager pass)."""
        Rg = api.Renderer()
        most = 0
        for fr in wl.frames:
            Rg.render([ds], [0, 0], fr.cameras, fr.foveas, cfg, out=out, visible=visible)
            most = max(most, Rg.stats()["instances"])
        fr0 = wl.frames[0]
        G = api.GraphedRender(Rg, [ds], [0, 0], fr0.cameras, fr0.foveas, cfg, instances=int(most * 1.02) + 4096,
                              visible=visible)
        Rg.most_instances = most
        return Rg, G

    def timed_graph(G, Rg, steps):
        for i in range(args.warmup):
            fr = wl.frames[i % len(wl.frames)]
            G.replay(fr.cameras, fr.foveas)
        Rg.check()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            fr = wl.frames[(args.warmup + i) % len(wl.frames)]
            flush.zero_()
            ev[i][0].record()
            G.replay(fr.cameras, fr.foveas)
            ev[i][1].record()
        barrier()
        Rg.check()
        return [a.elapsed_time(b) for a, b in ev]

    # foveated frames (the headline): one graph replay per stereo frame
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    Rg, G = graphed(fov_cfg)
    kernels_per_frame = Rg.stats()["kernels"]
    with ClockSampler(gpu_index) as clk:
        t_wall = time.perf_counter()
        ms_fov = timed_graph(G, Rg, args.steps)
        t_wall = time.perf_counter() - t_wall
    total_ms = max_over_ranks(sum(ms_fov), pg)
    value = job_rate(ws, args.steps, total_ms)
    # the same frames issued eagerly (one vrs_render call each), with per-stage events
    ms_eager, stages, ncalls = timed_eager(fov_cfg, min(args.plain_steps, args.steps), profile=True)
    # the same frames as two monocular passes (one vrs_render per eye): what the fused
    # stereo pass (one preprocess reading every Gaussian once for both eyes, one sort,
    # one render launch over both eyes' work) saves
    n_mono = min(args.plain_steps, args.steps)
    for i in range(args.warmup):
        fr = wl.frames[i % len(wl.frames)]
        for e in range(2):
            R.render([ds], [0], [fr.cameras[e]], [fr.foveas[e]], fov_cfg, out=out[e:e + 1])
    R.check()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_mono)]
    for i in range(n_mono):
        fr = wl.frames[(args.warmup + i) % len(wl.frames)]
        flush.zero_()
        ev[i][0].record()
        for e in range(2):
            R.render([ds], [0], [fr.cameras[e]], [fr.foveas[e]], fov_cfg, out=out[e:e + 1])
        ev[i][1].record()
    barrier()
    R.check()
    ms_mono = [a.elapsed_time(b) for a, b in ev]
    # plain full-resolution render on the same GPU, also one graph replay per frame
    Rp, Gp = graphed(plain_cfg)
    ms_plain = timed_graph(Gp, Rp, min(args.plain_steps, args.steps))
    del Gp
    Rp.close()
    # the same foveated frames with visibility culling (Sec. 4.3) under a synthetic lens
    # mask per eye (an OpenXR hidden-area mask stands in): culled tiles hold the background
    from paper_2505_10144_gb300 import synth
    masks = [torch.from_numpy(synth.lens_mask(W_IMG, H_IMG, e)).cuda() for e in (-1, +1)]
    Rv, Gv = graphed(fov_cfg, visible=masks)
    ms_vis = timed_graph(Gv, Rv, min(args.plain_steps, args.steps))
    fr1 = wl.frames[1]
    Rv.render([ds], [0, 0], fr1.cameras, fr1.foveas, fov_cfg, out=out, visible=masks)
    inst_vis = Rv.stats()["instances"]
    Rv.render([ds], [0, 0], fr1.cameras, fr1.foveas, fov_cfg, out=out)
    inst_all = Rv.stats()["instances"]
    T = 32
    ntx, nty = (W_IMG + T - 1) // T, (H_IMG + T - 1) // T
    culled = 0
    for m in masks:
        pad = torch.zeros((nty * T, ntx * T), dtype=torch.bool, device="cuda")
        pad[:H_IMG, :W_IMG] = m != 0
        culled += int((~pad.reshape(nty, T, ntx, T).any(dim=3).any(dim=1)).sum())
    visibility = {"value": len(ms_vis) / (sum(ms_vis) / 1e3), "unit": "frames/s",
                  "ms_per_step": statistics.mean(ms_vis), "p99_ms": float(np.percentile(ms_vis, 99)),
                  "tiles_culled_pct": 100.0 * culled / (2 * ntx * nty),
                  "instances_frame1": inst_vis, "instances_frame1_unmasked": inst_all,
                  "mask": "ellipse 0.535 W x 0.555 H per eye, centre 3% towards the nose (synthetic lens)"}
    del Gv
    Rv.close()
    # the two-pass foveated baseline (Appendix A) on the same frames, eager calls like
    # the "eager" single-pass line: full-resolution centre square + half-resolution view
    n_tp = min(args.plain_steps, args.steps)
    for i in range(args.warmup):
        fr = wl.frames[i % len(wl.frames)]
        R.render_two_pass([ds], [0, 0], fr.cameras, fr.foveas, fov_cfg, out=out)
    R.check()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_tp)]
    for i in range(n_tp):
        fr = wl.frames[(args.warmup + i) % len(wl.frames)]
        flush.zero_()
        ev[i][0].record()
        R.render_two_pass([ds], [0, 0], fr.cameras, fr.foveas, fov_cfg, out=out)
        ev[i][1].record()
    barrier()
    R.check()
    ms_tp = [a.elapsed_time(b) for a, b in ev]
    fr1 = wl.frames[1]
    tp_img = R.render_two_pass([ds], [0, 0], fr1.cameras, fr1.foveas, fov_cfg, out=out).clone()
    sp_img = R.render([ds], [0, 0], fr1.cameras, fr1.foveas, fov_cfg).clone()
    # the popping global orders of 3DGS (view-space z) and Mini-Splatting (distance) on the
    # same foveated frames (graph replays), with their error against the exact per-ray order
    global_orders = {}
    exact_cfg = api.RenderConfig(**{**fov_cfg.__dict__, "sort_mode": "exact"})
    ex_img = R.render([ds], [0, 0], fr1.cameras, fr1.foveas, exact_cfg).clone()
    for gm in ("global_z", "global_dist"):
        gcfg = api.RenderConfig(**{**fov_cfg.__dict__, "sort_mode": gm})
        Rq, Gq = graphed(gcfg)
        ms_q = timed_graph(Gq, Rq, min(args.plain_steps, args.steps))
        q_img = Rq.render([ds], [0, 0], fr1.cameras, fr1.foveas, gcfg).clone()
        global_orders[gm] = {"value": len(ms_q) / (sum(ms_q) / 1e3), "unit": "frames/s",
                             "ms_per_step": statistics.mean(ms_q), "psnr_vs_exact_db": psnr(q_img, ex_img)}
        del Gq
        Rq.close()
    global_orders["popping"] = popping(api, ds, wl, fov_cfg, torch)
    global_orders["popping"]["image_flicker_on_unchanged_rays"] = grid_flicker(api, ds, wl, torch)
    global_orders["hier_4_8_16_psnr_vs_exact_db"] = psnr(R.render([ds], [0, 0], fr1.cameras, fr1.foveas, fov_cfg),
                                                          ex_img)
    two_pass = {"value": len(ms_tp) / (sum(ms_tp) / 1e3), "unit": "frames/s", "ms_per_step": statistics.mean(ms_tp),
                "p99_ms": float(np.percentile(ms_tp, 99)),
                "single_pass_eager_ms": statistics.mean(ms_eager),
                "single_pass_speedup": statistics.mean(ms_tp) / statistics.mean(ms_eager),
                "psnr_vs_single_pass_db": psnr(tp_img, sp_img),
                "config": "vrs_render_two_pass: centre square at full resolution + half-resolution view, eager"}
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
    approx = approximation_error(R, api, ds, wl.frames[1], fov_cfg, torch)
    render_ms = stages.get("render", 0.0) / max(ncalls, 1)
    flops = FLOPS_EVAL * cnt["evaluated"] + FLOPS_KEPT * cnt["kept"] + FLOPS_BLEND * cnt["blended"]
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local)
    sm_mhz = clocks["sm_mhz"] or 2070.0
    derived_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    peak_tflops = peaks["fp32_tflops"]
    achieved = flops / (render_ms / 1e3) / 1e12 if render_ms > 0 else 0.0
    exp2_rate = cnt["kept"] / (render_ms / 1e3) / 1e9 if render_ms > 0 else 0.0
    traffic, traffic_note, issue_busy, inst_pair = profiled_traffic()
    max_mhz = float(clocks.get("sm_max_mhz") or 2070.0)
    lane_peak = props.multi_processor_count * LANES_PER_SM * max_mhz * 1e6 / 1e12  # T lane-ops/s
    alu_ops = ALU_OPS_PER_PAIR * cnt["evaluated"]
    alu_achieved = alu_ops / (render_ms / 1e3) / 1e12 if render_ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": "warp_render_kernel<4,8> (hierarchical 4/8/16)",
                "achieved": alu_achieved, "peak": lane_peak, "unit": "T lane-ops/s",
                "frac": alu_achieved / lane_peak if lane_peak else None,
                "traffic": traffic, "traffic_note": traffic_note,
                "basis": f"{ALU_OPS_PER_PAIR} FP32 operations per evaluated pair (plane map and quadratic form, "
                         "exp2, t*, blend, window compares) x the evaluated pairs counted on the device, over the "
                         "launch's average CUDA-event time",
                "peak_source": f"derived: {props.multi_processor_count} SMs x 4 schedulers x 32 lanes x "
                               f"{max_mhz:.0f} MHz (maximum SM clock)",
                "issue_slots_busy_ncu": issue_busy,
                "thread_inst_per_evaluated_pair_ncu": inst_pair,
                "issue_basis_note": "ncu's thread instructions per evaluated pair against the algorithmic "
                                    f"{ALU_OPS_PER_PAIR}: the rest is window bookkeeping, staging and control",
                "fp32": {"achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops if peak_tflops else None, "flops_per_launch": flops,
                         "peak_source": "of measured: FFMA microbenchmark (vrs_measure_peaks, 64 warps per SM, "
                                        f"best of 5); derived {props.multi_processor_count} SMs x "
                                        f"{FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz = {derived_tflops:.1f}"},
                "exp2": {"achieved_gops": exp2_rate, "peak_gops": peaks["exp2_gops"],
                         "frac": exp2_rate / peaks["exp2_gops"] if peaks["exp2_gops"] else None,
                         "per_launch": cnt["kept"], "note": "one exp2f per kept pair (the pair opacity)"},
                "work_per_launch": {"evaluated_pairs": cnt["evaluated"], "kept_pairs": cnt["kept"],
                                    "blended_pairs": cnt["blended"], "alu_ops": alu_ops},
                "avg_launch_ms": render_ms}
    rp = roofline_peaks()
    stage_roof = stage_rooflines({k: v / max(ncalls, 1) for k, v in stages.items()}, cnt, 2, N_GAUSS,
                                 Rg.stats()["sort_passes"], periphery_pixels(wl.frames[args.warmup]), rp["hbm_gbs"],
                                 rp["source"])
    # end to end through the public API: camera/gaze in (pinned staging -> device inside
    # the replay), both images back to pinned host memory every frame.  Serialized: the
    # read-back follows the replay on one stream.  Pipelined, as a frame loop runs it: two
    # graphed contexts take alternate frames, and frame i's image goes device-to-host on a
    # copy stream while frame i + 1 renders.
    host = torch.empty((2, 3, H_IMG, W_IMG), dtype=torch.float32, pin_memory=True)
    n_e2e = min(40, args.steps)

    def serialized(i):
        fr = wl.frames[i % len(wl.frames)]
        host.copy_(G.replay(fr.cameras, fr.foveas), non_blocking=True)

    cur, cs = torch.cuda.current_stream(), torch.cuda.Stream()
    # a second graphed context renders every other frame into its own output buffer, so
    # a frame's device-to-host copy (copy stream) overlaps the next frame's render
    Rg2, G2 = graphed(fov_cfg)
    graphs = [G, G2]
    hosts = [host, torch.empty((2, 3, H_IMG, W_IMG), dtype=torch.float32, pin_memory=True)]
    copied = [torch.cuda.Event() for _ in range(2)]
    rendered = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]

    def pipelined(i):
        fr = wl.frames[i % len(wl.frames)]
        k = i % 2
        if used[k]:
            cur.wait_event(copied[k])  # this context's output was read out two frames ago
        img = graphs[k].replay(fr.cameras, fr.foveas)
        rendered[k].record(cur)
        cs.wait_event(rendered[k])
        with torch.cuda.stream(cs):
            hosts[k].copy_(img, non_blocking=True)
            copied[k].record(cs)
        used[k] = True

    def timed_e2e(step):
        for i in range(args.warmup):
            step(i)
        cur.wait_stream(cs)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(n_e2e):
            step(args.warmup + i)
        cur.wait_stream(cs)  # the last read-back is inside the timed region
        e1.record()
        barrier()
        Rg.check()
        return job_rate(ws, n_e2e, max_over_ranks(e0.elapsed_time(e1), pg))

    e2e_serial = timed_e2e(serialized)
    e2e_fps = timed_e2e(pipelined)
    Rg2.check()
    del G2
    Rg2.close()
    learned = learned_periphery(api, torch, min(40, args.steps), args.warmup)
    reuse = stereo_reuse(api, torch, min(30, args.steps), args.warmup)
    finetune = backward_line(api, torch, args.warmup, min(20, args.steps), peaks)
    batched = batched_line(api, torch, min(10, args.steps), args.warmup, None, quiet=True)
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
                   "timing": "CUDA events around each frame on the launching stream",
                   "frame": "one CUDA graph replay of the whole stereo frame (vrs_update_views + replay)"},
        "p50_ms": float(np.percentile(ms_fov, 50)), "p99_ms": float(np.percentile(ms_fov, 99)),
        "plain": {"value": len(ms_plain) / (sum(ms_plain) / 1e3), "unit": "frames/s",
                  "ms_per_step": statistics.mean(ms_plain), "p99_ms": float(np.percentile(ms_plain, 99)),
                  "config": "full resolution, 16x16 tiles, hierarchical 4/8/16, same pipeline"},
        "speedup_vs_plain": statistics.mean(ms_plain) / statistics.mean(ms_fov),
        "visibility_culling": visibility,
        "two_pass_baseline": two_pass,
        "global_orders": global_orders,
        "stereo_fusion": {"fused_eager_ms": statistics.mean(ms_eager), "two_monocular_passes_ms": statistics.mean(ms_mono),
                          "speedup": statistics.mean(ms_mono) / statistics.mean(ms_eager),
                          "config": "the same foveated frames, eager: one vrs_render of both eyes vs one per eye"},
        "eager": {"value": len(ms_eager) / (sum(ms_eager) / 1e3), "unit": "frames/s",
                  "ms_per_step": statistics.mean(ms_eager), "p99_ms": float(np.percentile(ms_eager, 99)),
                  "config": "one vrs_render call per frame (host reads the instance count back)"},
        "psnr_vs_plain_db": statistics.mean(ps),
        "hier_vs_exact": approx,
        "stage_ms_per_frame": {k: v / max(ncalls, 1) for k, v in stages.items()},
        "counters_per_frame": cnt,
        "roofline": roofline,
        "stage_rooflines": stage_roof,
        "learned_periphery": learned,
        "stereo_reuse": reuse,
        "finetune": finetune,
        "batched": batched,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "GraphedRender.replay (vrs_update_views + graph replay), then both eyes to pinned host "
                        "memory every frame on a copy stream; two graphed contexts take alternate frames, so a "
                        "frame's device-to-host copy overlaps the next frame's render",
                "serialized_value": e2e_serial,
                "serialized_path": "the same calls with the device-to-host copy on the render stream after each "
                                   "replay"},
        "gpu_launches": kernels_per_frame * args.steps,
        "clocks": clocks,
        "measured_peaks": peaks,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import native as on
        from paper_2505_10144_gb300 import synth
        scene64 = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in scene.arrays()], scene.sh_degree)
        whole = [oracle_whole_frame(scene64, wl.frames[i]) for i in range(3)]
        sec_band, desc_band, _ = oracle_frame_estimate(scene64, wl.frames[0], budget_s=8.0)
        line["cpu_baseline"] = {"value": 3.0 / sum(whole), "unit": "frames/s", "cores": on.num_threads(),
                                "kind": "oracle", "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
                                "sample": "FP64 oracle as it stands, hierarchical 4/8/16, foveated: 3 whole stereo "
                                          "frames of the trajectory (both eyes, every sample)",
                                "seconds_per_frame": whole,
                                "band_estimate": {"value": 1.0 / sec_band, "sample": desc_band},
                                "other_workloads": oracle_other_workloads(scene64, wl.frames[0])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
