"""Batched persistent launch in a captured CUDA graph, and the autotuner."""
import json

import numpy as np
import pytest
import torch

import outcomes as oc

from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2505_10144_gb300 import api, build
    build.build()
    R = api.Renderer()
    scenes = [api.DeviceScene.from_host(synth.shell_scene(n, synth.rng_for(2, salt=k), sh_degree=3))
              for k, n in enumerate([3000, 8000])]
    W, H = 256, 192
    poses = [synth.batched_poses(2, synth.rng_for(2, salt=10 + k), W, H) for k in range(2)]
    cams, fovs, vs = [], [], []
    for s_idx, frames in enumerate(poses):
        for fr in frames:
            cams += fr.cameras
            fovs += [synth.fovea_for(W, (f.gaze_x, f.gaze_y), radius_frac=0.25) for f in fr.foveas]
            vs += [s_idx, s_idx]
    cfg = api.RenderConfig(sort_mode="hier", windows=(4, 8, 16), key_tile=32, fovea_mode="bilinear")
    yield api, R, scenes, vs, cams, fovs, cfg
    R.close()


def test_graph_replay_equals_eager_render(setup):
    api, R, scenes, vs, cams, fovs, cfg = setup
    gr = api.GraphedRender(R, scenes, vs, cams, fovs, cfg)
    out = gr.replay().clone()
    R.check()
    eager = R.render(scenes, vs, cams, fovs, cfg)
    R.check()
    assert torch.equal(out, eager)
    # new poses and gaze through vrs_update_views, then replay
    cams2 = [synth.Camera(c.world_to_cam, c.fx, c.fy, c.cx, c.cy, c.width, c.height, c.near_z) for c in cams]
    rot = synth.head_rotation(0.15)
    for c in cams2:
        R3 = c.world_to_cam[:, :3].astype(np.float64) @ rot.T
        c.world_to_cam = np.ascontiguousarray(np.concatenate([R3, c.world_to_cam[:, 3:]], 1), dtype=np.float32)
    fovs2 = [synth.Fovea(f.gaze_x + 17.0, f.gaze_y - 9.0, f.radius_px, f.band_px) for f in fovs]
    out2 = gr.replay(cams2, fovs2).clone()
    R.check()
    eager2 = R.render(scenes, vs, cams2, fovs2, cfg)
    R.check()
    assert torch.equal(out2, eager2)
    assert not torch.equal(out2, out)


def test_autotuner_picks_a_candidate_and_caches_it(setup, tmp_path):
    from paper_2505_10144_gb300 import autotune
    api, R, scenes, vs, cams, fovs, cfg = setup
    path = tmp_path / "tune.json"
    best, res = autotune.autotune(R, scenes, vs, cams, fovs, cfg, cache_path=path, reps=2,
                                  window_sets=[(4, 8, 16), (8, 16, 32)], cta_caps=[0, 1], tile_sizes=[32, 16])
    assert len(res) == 8
    # every candidate carries its quality against the exact order; the choice is the
    # fastest of those at or above the floor
    ok = [r for r in res if r["meets_floor"]]
    assert ok and all(r["meets_floor"] == (r["psnr_db"] >= best["psnr_floor_db"]) for r in res)
    assert best["ms"] == min(r["ms"] for r in ok) and best["psnr_db"] >= best["psnr_floor_db"]
    assert all(0.0 <= r["over_2e-4_pct"] <= 100.0 and r["psnr_db"] > 20.0 for r in res)
    # larger windows approach the exact order: never less accurate on the same tiles
    for T in (32, 16):
        q = {tuple(r["windows"]): r["psnr_db"] for r in res if r["key_tile"] == T}
        assert q[(8, 16, 32)] >= q[(4, 8, 16)] - 0.05
    # with a floor that some candidates miss, the choice is the fastest of the others, and
    # with none meeting it, the fastest overall
    b3, r3 = autotune.autotune(R, scenes, vs, cams, fovs, cfg, reps=1, window_sets=[(4, 8, 16)], cta_caps=[0],
                               tile_sizes=[32, 16], psnr_floor=max(r["psnr_db"] for r in res) + 1.0, use_cache=False)
    met = [r for r in r3 if r["meets_floor"]]
    assert b3["ms"] == min(r["ms"] for r in (met or r3))
    cache = json.loads(path.read_text())
    assert autotune.cache_key(scenes, vs, cams) in cache
    best2, _ = autotune.autotune(R, scenes, vs, cams, fovs, cfg, cache_path=path)
    assert best2["windows"] == best["windows"] and best2["max_ctas_per_sm"] == best["max_ctas_per_sm"]
    assert best2["key_tile"] == best["key_tile"]
    # the CTA cap is scheduling only: same image
    R.set_tuning(1)
    a = R.render(scenes, vs, cams, fovs, cfg).clone()
    R.set_tuning(0)
    b = R.render(scenes, vs, cams, fovs, cfg)
    assert torch.equal(a, b)


def test_full_size_batched_views_sampled_crops():
    """The batched workload at full size, as the benchmark launches it: scenes of 200k, 1M
    and 3M Gaussians x 8 head poses x 2 eyes = 48 views of 2064x2208, foveated, hierarchical
    4/8/16, in one captured graph.  Crops of one view per scene (32-aligned, at the gaze
    point and in the periphery) against oracle renders of the same rays, interior pixels."""
    from oracle import native as on
    from paper_2505_10144_gb300 import api, build
    build.build()
    W, H = 2064, 2208
    hosts = [synth.shell_scene(n, synth.rng_for(2, salt=k), sh_degree=3)
             for k, n in enumerate([200_000, 1_000_000, 3_000_000])]
    cams, fovs, vs = [], [], []
    for k in range(3):
        for fr in synth.batched_poses(8, synth.rng_for(2, salt=10 + k), W, H):
            cams += fr.cameras
            fovs += fr.foveas
            vs += [k, k]
    R = api.Renderer()
    try:
        scenes = [api.DeviceScene.from_host(h) for h in hosts]
        cfg = api.RenderConfig(sort_mode="hier", windows=(4, 8, 16), key_tile=32, fovea_mode="bilinear")
        gr = api.GraphedRender(R, scenes, vs, cams, fovs, cfg)
        out = gr.replay()
        R.check()
        checked = 0
        for k in range(3):
            v = 16 * k + 2 * (3 + k) + (k & 1)  # pose 3 + k, left or right eye
            cam, fv = cams[v], fovs[v]
            for sx, sy in [(fv.gaze_x, fv.gaze_y), (300.0 + 500.0 * k, 1900.0 - 400.0 * k)]:
                x0 = int(min(max(sx - 32, 0), W - 64)) // 32 * 32
                y0 = int(min(max(sy - 32, 0), H - 64)) // 32 * 32
                ref = oc.crop_reference(hosts[k], cam, x0, y0, 64, 64, "hier", fovea=fv, windows=(4, 8, 16),
                                        key_tile=32)
                sub = out[v][:, y0:y0 + 64, x0:x0 + 64].cpu().numpy().astype(np.float64)
                oc.check(sub, ref, "hier", label=f"batched scene {k} view {v} at ({x0},{y0})")
                checked += 1
            if k == 0:
                # the exact order on one view of this scene, through an eager render
                ex = R.render([scenes[k]], [0], [cam], [fv], api.RenderConfig(sort_mode="exact", key_tile=32,
                                                                               fovea_mode="bilinear"))
                R.check()
                x0 = int(min(max(fv.gaze_x - 32, 0), W - 64)) // 32 * 32
                y0 = int(min(max(fv.gaze_y - 32, 0), H - 64)) // 32 * 32
                ref = oc.crop_reference(hosts[k], cam, x0, y0, 64, 64, "exact", fovea=fv, key_tile=32)
                oc.check(ex[0][:, y0:y0 + 64, x0:x0 + 64].cpu().numpy().astype(np.float64), ref, "exact",
                         label=f"batched scene {k} view {v} exact")
        assert checked == 6
    finally:
        R.close()
