"""Autotuner for the batched render: times CUDA-graph replays of the real workload for
each candidate and keeps the fastest one whose image stays within a quality floor,
cached as JSON keyed by (total Gaussians, width, height, views, GPU name).

Candidates: the key-tile size (32x32 as in Sec. 4.3, or 16x16: foveation classes and
sort keys on finer tiles, more instances, a better-sorted stream), the per-ray window
sizes of the hierarchical resort (Sec. 4.1), and the cap on resident render CTAs per SM
(scheduling only, never the image).  Tile and window sizes trade speed for the error of
the approximation, so every (tile, windows) pair is rendered once on one sampled view
and compared with the exact per-ray order on 32x32 tiles, the method's reference: its
PSNR and the share of pixels off by more than 2e-4 are reported beside its time, and a
candidate below the PSNR floor is not chosen.  The default floor is the PSNR of the
default configuration (32x32 tiles, windows 4/8/16) minus 0.5 dB."""
from __future__ import annotations

import dataclasses
import json
import math
import os
from pathlib import Path

import torch

from .api import GraphedRender, RenderConfig, Renderer

TILE_SIZES = [32, 16]
WINDOW_SETS = [(4, 8, 16), (4, 8, 24), (8, 16, 32)]
CTA_CAPS = [0, 1]
DEFAULT = (32, (4, 8, 16))


def cache_key(scenes, view_scene, cams) -> str:
    total = sum(scenes[v].n for v in view_scene)
    name = torch.cuda.get_device_name()
    return f"N={total}|W={cams[0].width}|H={cams[0].height}|V={len(cams)}|{name}"


def time_replays(gr: GraphedRender, reps: int) -> float:
    for _ in range(2):
        gr.replay()
    torch.cuda.synchronize()
    # CUDAGraph.replay() launches on the current stream: time on that stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        gr.graph.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def quality(renderer: Renderer, scenes, view_scene, cams, foveas, cfg: RenderConfig, ref: torch.Tensor, view: int):
    """PSNR (dB) and pixels off by more than 2e-4 (%) of one view against ref."""
    img = renderer.render([scenes[view_scene[view]]], [0], [cams[view]], [foveas[view]] if foveas else None, cfg)
    renderer.check()
    d = (img[0] - ref).abs()
    mse = float((d ** 2).mean())
    return (float("inf") if mse == 0 else 10 * math.log10(1.0 / mse),
            float((d.amax(dim=0) > 2e-4).float().mean() * 100))


def autotune(renderer: Renderer, scenes, view_scene, cams, foveas, base: RenderConfig, cache_path=None,
             reps: int = 3, window_sets=WINDOW_SETS, cta_caps=CTA_CAPS, tile_sizes=TILE_SIZES,
             psnr_floor: float | None = None, sample_view: int = 0, use_cache: bool = True):
    """-> (best config dict, list of all measured candidates).  Each candidate: key_tile,
    windows, max_ctas_per_sm, ms per replay, psnr_db and over_2e-4_pct against the exact
    order on view sample_view, and whether it met the floor."""
    key = cache_key(scenes, view_scene, cams)
    cache = {}
    if cache_path and Path(cache_path).exists():
        cache = json.loads(Path(cache_path).read_text())
        if use_cache and key in cache:
            return cache[key], cache[key].get("candidates", [])
    exact = dataclasses.replace(base, sort_mode="exact", key_tile=32)
    v = sample_view
    ref = renderer.render([scenes[view_scene[v]]], [0], [cams[v]], [foveas[v]] if foveas else None, exact)[0].clone()
    renderer.check()
    qual = {}
    for T in tile_sizes:
        for win in window_sets:
            cfg = dataclasses.replace(base, windows=tuple(win), key_tile=T)
            qual[(T, tuple(win))] = quality(renderer, scenes, view_scene, cams, foveas, cfg, ref, v)
    if psnr_floor is None:
        psnr_floor = qual.get(DEFAULT, max(qual.values()))[0] - 0.5
    results = []
    for T in tile_sizes:
        for win in window_sets:
            p, over = qual[(T, tuple(win))]
            for cap in cta_caps:
                renderer.set_tuning(cap)
                cfg = dataclasses.replace(base, windows=tuple(win), key_tile=T)
                gr = GraphedRender(renderer, scenes, view_scene, cams, foveas, cfg)
                ms = time_replays(gr, reps)
                renderer.check()
                results.append({"key_tile": T, "windows": list(win), "max_ctas_per_sm": cap, "ms": ms, "psnr_db": p,
                                "over_2e-4_pct": over, "meets_floor": p >= psnr_floor})
                del gr
    renderer.set_tuning(0)
    ok = [r for r in results if r["meets_floor"]] or results
    best = dict(min(ok, key=lambda r: r["ms"]))
    best["psnr_floor_db"] = psnr_floor
    best["reference"] = f"exact per-ray order, 32x32 key tiles, view {v}"
    best["candidates"] = results
    if cache_path:
        cache[key] = best
        Path(cache_path).parent.mkdir(parents=True, exist_ok=True)
        tmp = str(cache_path) + f".tmp{os.getpid()}"
        Path(tmp).write_text(json.dumps(cache, indent=1))
        os.replace(tmp, cache_path)
    return best, results
