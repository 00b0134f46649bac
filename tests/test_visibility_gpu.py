"""Visibility culling (Sec. 4.3): a headset mask removes the key tiles without a visible
pixel from the instance lists and from the render.  GPU against the FP64 oracle with
the same mask, through the C ABI; the parity rule is the one of the render tests."""
import numpy as np
import pytest
import torch

import outcomes as oc

from oracle import grad as og
from oracle import native as on
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-4
BG = (0.2, 0.35, 0.5)


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    r = api.Renderer()
    yield r
    r.close()


@pytest.fixture(scope="module")
def vr_masked():
    scene = synth.shell_scene(30_000, synth.rng_for(1), sh_degree=3)
    W, H = 320, 256
    cams = synth.stereo_cameras((0.02, -0.01, 0.05), 0.3, W, H, 110.0)
    fov = [synth.fovea_for(W, (150.0, 120.0), radius_frac=0.2), synth.fovea_for(W, (170.0, 110.0), radius_frac=0.2)]
    masks = [synth.lens_mask(W, H, -1, 0.48, 0.5), synth.lens_mask(W, H, +1, 0.48, 0.5)]
    return scene, cams, fov, masks


def tiles_invisible(mask, T):
    H, W = mask.shape
    ntx, nty = (W + T - 1) // T, (H + T - 1) // T
    pad = np.zeros((nty * T, ntx * T), bool)
    pad[:H, :W] = mask != 0
    return ~pad.reshape(nty, T, ntx, T).any(axis=(1, 3))


def render(R, scene, cams, fov, masks, **cfg):
    from paper_2505_10144_gb300 import api
    ds = api.DeviceScene.from_host(scene)
    vis = None if masks is None else [torch.from_numpy(np.ascontiguousarray(m)).cuda() for m in masks]
    out = R.render([ds], [0] * len(cams), cams, fov, api.RenderConfig(**cfg), visible=vis)
    R.check()
    return out.cpu().numpy().astype(np.float64), R.stats()


@pytest.mark.parametrize("mode,win", [("exact", (0, 0, 0)), ("hier", (4, 8, 16))])
def test_visibility_foveated_stereo_matches_oracle(R, vr_masked, mode, win):
    scene, cams, fov, masks = vr_masked
    T = 32
    gpu, st = render(R, scene, cams, fov, masks, sort_mode=mode, windows=win, key_tile=T, fovea_mode="bilinear", bg=BG)
    _, st0 = render(R, scene, cams, fov, None, sort_mode=mode, windows=win, key_tile=T, fovea_mode="bilinear", bg=BG)
    assert st["instances"] < st0["instances"]
    for v in range(2):
        inv = tiles_invisible(masks[v], T)
        assert inv.sum() >= 4
        ref = oc.reference(scene, cams[v], mode, windows=win, key_tile=T, fovea=fov[v], bg=BG, visible=masks[v])
        assert np.array_equal(ref["tile_class"] >= 4, inv)
        oc.check(gpu[v], ref, mode, label=f"visibility foveated {mode} eye {v}")
        pix = np.repeat(np.repeat(inv, T, 0), T, 1)[:256, :320]
        for ch in range(3):
            assert np.all(gpu[v][ch][pix] == np.float32(BG[ch]))


@pytest.mark.parametrize("mode", ["exact", "hier"])
def test_visibility_plain_matches_oracle(R, vr_masked, mode):
    scene, cams, _, masks = vr_masked
    gpu, _ = render(R, scene, cams, None, masks, sort_mode=mode, key_tile=16, bg=BG)
    for v in range(2):
        ref = oc.reference(scene, cams[v], mode, key_tile=16, bg=BG, visible=masks[v])
        oc.check(gpu[v], ref, mode, label=f"visibility plain {mode} eye {v}")


def test_visibility_lists_are_the_unmasked_lists_of_visible_tiles(R, vr_masked):
    """The masked instance lists are exactly the unmasked ones with the invisible tiles
    emptied (integer work: bit-exact)."""
    from paper_2505_10144_gb300 import api
    scene, cams, fov, masks = vr_masked
    ds = api.DeviceScene.from_host(scene)
    cfg = api.RenderConfig(sort_mode="hier", key_tile=32, fovea_mode="bilinear")
    lists = []
    for vis in (None, [torch.from_numpy(m).cuda() for m in masks]):
        R.render([ds], [0, 0], cams, fov, cfg, visible=vis)
        R.check()
        tpv = ((320 + 31) // 32) * ((256 + 31) // 32)
        k, v, rg = R.instances(2, tpv)
        lists.append((k.cpu().numpy(), v.cpu().numpy(), rg.cpu().numpy()))
    (k0, v0, r0), (k1, v1, r1) = lists
    inv = np.concatenate([tiles_invisible(m, 32).ravel() for m in masks])
    for t in range(len(inv)):
        a0, b0 = r0[t]
        a1, b1 = r1[t]
        if inv[t]:
            assert b1 == a1
        else:
            assert np.array_equal(k1[a1:b1], k0[a0:b0]) and np.array_equal(v1[a1:b1], v0[a0:b0])


def test_visibility_all_visible_is_no_mask(R, vr_masked):
    scene, cams, fov, _ = vr_masked
    ones = [np.ones((256, 320), np.uint8)] * 2
    a, _ = render(R, scene, cams, fov, None, sort_mode="hier", key_tile=32, fovea_mode="bilinear", bg=BG)
    b, _ = render(R, scene, cams, fov, ones, sort_mode="hier", key_tile=32, fovea_mode="bilinear", bg=BG)
    assert np.array_equal(a, b)


def test_visibility_graph_replay(R, vr_masked):
    """Masks are fixed per eye across replays; a replay equals the eager render, and a
    replay cannot add or drop masks."""
    from paper_2505_10144_gb300 import api
    scene, cams, fov, masks = vr_masked
    ds = api.DeviceScene.from_host(scene)
    cfg = api.RenderConfig(sort_mode="hier", key_tile=32, fovea_mode="bilinear", bg=BG)
    vis = [torch.from_numpy(m).cuda() for m in masks]
    R2 = api.Renderer()
    try:
        G = api.GraphedRender(R2, [ds], [0, 0], cams, fov, cfg, visible=vis)
        cams2 = synth.stereo_cameras((0.03, 0.0, 0.04), 0.33, 320, 256, 110.0)
        got = G.replay(cams2, fov).clone()
        R2.check()
        want = R.render([ds], [0, 0], cams2, fov, cfg, visible=vis)
        R.check()
        assert torch.equal(got, want)
        with pytest.raises(RuntimeError):
            R2.update_views(cams2, fov, cfg)  # no masks: differs from the captured render
    finally:
        R2.close()


def test_visibility_backward_matches_oracle(R):
    """Fine-tuning under a mask: pixels of invisible tiles are a constant background and
    pass no gradient; the rest matches the oracle gradient."""
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(41)
    scene = synth.shell_scene(6000, synth.rng_for(3), sh_degree=3)
    W, H = 128, 96
    cams = synth.stereo_cameras((0.01, 0.0, 0.02), 0.25, W, H, 110.0)
    fov = [synth.fovea_for(W, (60.0, 50.0), radius_frac=0.25), synth.fovea_for(W, (70.0, 44.0), radius_frac=0.25)]
    masks = [synth.lens_mask(W, H, -1, 0.45, 0.5), synth.lens_mask(W, H, +1, 0.45, 0.5)]
    masks[0][:, :32] = 0  # the outer tile column of each eye
    masks[1][:, W - 32:] = 0
    cfg = api.RenderConfig(sort_mode="hier", key_tile=32, fovea_mode="bilinear")
    dimg = np.zeros((2, 3, H, W))
    g_ref = None
    for v in range(2):
        ref = on.render(scene, cams[v], "hier", key_tile=32, fovea=fov[v], want_orders=True, visible=masks[v])
        assert (ref["tile_class"] >= 4).any()
        m = ref["marginal"].copy()
        for dy in (-2, -1, 1, 2):
            m |= np.roll(ref["marginal"], dy, 0)
        for dx in (-2, -1, 1, 2):
            m |= np.roll(m, dx, 1)
        dimg[v] = rng.normal(size=(3, H, W)) * ~m[None]
        gv = og.image_grad(scene, cams[v], ref["orders"], dimg[v], ref["tile_class"], fov[v])
        g_ref = gv if g_ref is None else {k: g_ref[k] + gv[k] for k in gv}
    ds = api.DeviceScene.from_host(scene)
    vis = [torch.from_numpy(mm).cuda() for mm in masks]
    R.render([ds], [0, 0], cams, fov, cfg, save=True, visible=vis)
    g = ds.zeros_like()
    R.backward([ds], [0, 0], cams, fov, cfg, torch.tensor(dimg, dtype=torch.float32).cuda(), [g], visible=vis)
    R.check()
    names = ["mean", "log_scale", "quat", "opacity_logit", "sh"]
    got = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(names, g.tensors())}
    for k in g_ref:
        err = np.linalg.norm(got[k] - g_ref[k]) / max(np.linalg.norm(g_ref[k]), 1e-30)
        assert err < 1e-4, (k, err)
