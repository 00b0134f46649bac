"""Autotuner for the batched render: times CUDA-graph replays of the real workload for
each candidate (per-ray window sizes, render CTAs per SM) and keeps the fastest, cached
as JSON keyed by (total Gaussians, width, height, views, GPU name).

Window sizes trade speed for the error of the hierarchical approximation against the
exact per-ray order, so every candidate's timing is reported with its windows; the CTA
cap changes scheduling only, never the image."""
from __future__ import annotations

import dataclasses
import json
import os
from pathlib import Path

import torch

from .api import GraphedRender, RenderConfig, Renderer

WINDOW_SETS = [(4, 8, 16), (4, 8, 24), (8, 16, 32)]
CTA_CAPS = [0, 1]


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


def autotune(renderer: Renderer, scenes, view_scene, cams, foveas, base: RenderConfig, cache_path=None,
             reps: int = 3, window_sets=WINDOW_SETS, cta_caps=CTA_CAPS, use_cache: bool = True):
    """-> (best config dict, list of all measured candidates)."""
    key = cache_key(scenes, view_scene, cams)
    cache = {}
    if cache_path and Path(cache_path).exists():
        cache = json.loads(Path(cache_path).read_text())
        if use_cache and key in cache:
            return cache[key], cache[key].get("candidates", [])
    results = []
    for win in window_sets:
        for cap in cta_caps:
            renderer.set_tuning(cap)
            cfg = dataclasses.replace(base, windows=tuple(win))
            gr = GraphedRender(renderer, scenes, view_scene, cams, foveas, cfg)
            ms = time_replays(gr, reps)
            renderer.check()
            results.append({"windows": list(win), "max_ctas_per_sm": cap, "ms": ms})
            del gr
    renderer.set_tuning(0)
    best = dict(min(results, key=lambda r: r["ms"]))
    best["candidates"] = results
    if cache_path:
        cache[key] = best
        Path(cache_path).parent.mkdir(parents=True, exist_ok=True)
        tmp = str(cache_path) + f".tmp{os.getpid()}"
        Path(tmp).write_text(json.dumps(cache, indent=1))
        os.replace(tmp, cache_path)
    return best, results
