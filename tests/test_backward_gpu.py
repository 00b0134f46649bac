"""Backward pass (fine-tuning through the rasterizer) and the loss / optimiser kernels
against the float64 oracle gradient (autograd of the restated forward with the oracle's
blend orders; itself pinned to central finite differences in the CPU tests).

Gradients are compared as relative L2 error per parameter group.  The image weights
dL/dimage are zero on pixels the oracle flags as marginal, so a legitimate FP32 flip of
a threshold or an order cannot move the comparison."""
import numpy as np
import pytest
import torch

from oracle import grad as og
from oracle import loss as ol
from oracle import native as on
from paper_2505_10144_gb300 import synth
from scenes import random_scene

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-4


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    r = api.Renderer()
    yield r
    r.close()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def gpu_grads(R, scene, cams, foveas, cfg, dimg):
    from paper_2505_10144_gb300 import api
    ds = api.DeviceScene.from_host(scene)
    R.render([ds], [0] * len(cams), cams, foveas, cfg, save=True)
    g = ds.zeros_like()
    R.backward([ds], [0] * len(cams), cams, foveas, cfg, torch.tensor(dimg, dtype=torch.float32).cuda(), [g])
    R.check()
    names = ["mean", "log_scale", "quat", "opacity_logit", "sh"]
    return {k: t.cpu().numpy().astype(np.float64) for k, t in zip(names, g.tensors())}


@pytest.mark.parametrize("mode,win", [("exact", (0, 0, 0)), ("window", (0, 0, 16)), ("hier", (4, 8, 16)),
                                      ("global_z", (0, 0, 0))])
def test_backward_plain_matches_oracle(R, mode, win):
    """1k Gaussians, 64x64, 110 deg FOV, SH degree 3 (the fine-tuning gradient subset)."""
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(31)
    scene = random_scene(1000, rng, sh_degree=3, z=(1.0, 3.0), xy=2.0, ls_mu=-2.6, ls_sd=0.4)
    cam = synth.identity_camera(64, 64, 110.0)
    ref = on.render(scene, cam, mode, windows=win, key_tile=16, want_orders=True)
    dimg = rng.normal(size=(1, 3, 64, 64)) * ~ref["marginal"][None, None]
    g_ref = og.image_grad(scene, cam, ref["orders"], dimg[0])
    cfg = api.RenderConfig(sort_mode=mode, windows=win, key_tile=16)
    g = gpu_grads(R, scene, [cam], None, cfg, dimg)
    for k in g_ref:
        assert rel_l2(g[k], g_ref[k]) < GRAD_RTOL, (k, rel_l2(g[k], g_ref[k]))


@pytest.mark.parametrize("mode,win", [("exact", (0, 0, 0)), ("hier", (4, 8, 16)), ("hier", (4, 8, 24)),
                                      ("window", (0, 0, 24))])
def test_backward_large_gaussians_matches_oracle(R, mode, win):
    """400 Gaussians much larger than a tile, some just beyond the near plane, 96x80: a
    pixel blends about 40 of them, so thousands of lanes add into the same Gaussian's
    gradient.  Per-sample windows of 16 (tree) and 24 (ring) replay in the backward as in
    the forward."""
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(78)
    scene = random_scene(400, rng, sh_degree=1, z=(0.25, 3.0), xy=1.5, ls_mu=-1.6, ls_sd=0.5)
    cam = synth.identity_camera(96, 80, 90.0)
    ref = on.render(scene, cam, mode, windows=win, key_tile=16, want_orders=True)
    assert len(ref["orders"][0]) > 30 * 96 * 80
    dimg = rng.normal(size=(1, 3, 80, 96)) * ~ref["marginal"][None, None]
    g_ref = og.image_grad(scene, cam, ref["orders"], dimg[0])
    g = gpu_grads(R, scene, [cam], None, api.RenderConfig(sort_mode=mode, windows=win, key_tile=16), dimg)
    errs = {k: rel_l2(g[k], g_ref[k]) for k in g_ref}
    assert max(errs.values()) < GRAD_RTOL, errs


@pytest.mark.parametrize("mode,win", [("exact", (0, 0, 0)), ("hier", (4, 8, 16))])
def test_backward_foveated_stereo_matches_oracle(R, mode, win):
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(32)
    scene = synth.shell_scene(6000, synth.rng_for(3), sh_degree=3)
    W, H = 128, 96
    cams = synth.stereo_cameras((0.01, 0.0, 0.02), 0.25, W, H, 110.0)
    fov = [synth.fovea_for(W, (60.0, 50.0), radius_frac=0.25), synth.fovea_for(W, (70.0, 44.0), radius_frac=0.25)]
    cfg = api.RenderConfig(sort_mode=mode, windows=win, key_tile=32, fovea_mode="bilinear")
    dimg = np.zeros((2, 3, H, W))
    g_ref = None
    for v in range(2):
        ref = on.render(scene, cams[v], mode, windows=win, key_tile=32, fovea=fov[v], want_orders=True)
        assert (ref["tile_class"] == 2).any() and (ref["tile_class"] != 2).any()
        # bilinear periphery pixels also read neighbouring samples: mask a pixel when any
        # sample of its 4x4 neighbourhood is marginal
        m = ref["marginal"].copy()
        for dy in (-2, -1, 1, 2):
            m |= np.roll(ref["marginal"], dy, 0)
        for dx in (-2, -1, 1, 2):
            m |= np.roll(m, dx, 1)
        dimg[v] = rng.normal(size=(3, H, W)) * ~m[None]
        gv = og.image_grad(scene, cams[v], ref["orders"], dimg[v], ref["tile_class"], fov[v])
        g_ref = gv if g_ref is None else {k: g_ref[k] + gv[k] for k in gv}
    g = gpu_grads(R, scene, cams, fov, cfg, dimg)
    for k in g_ref:
        assert rel_l2(g[k], g_ref[k]) < GRAD_RTOL, (k, rel_l2(g[k], g_ref[k]))


def test_autograd_function_and_loss(R):
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(33)
    scene = random_scene(500, rng, sh_degree=1, z=(1.0, 3.0), xy=2.0, ls_mu=-2.5)
    cams = [synth.identity_camera(48, 40, 100.0), synth.camera_from_pose(synth.head_rotation(0.2), (0.1, 0, 0), 48, 40,
                                                                         synth.focal_for_hfov(48, 100.0))]
    params = {k: torch.tensor(np.asarray(v), device="cuda", requires_grad=True)
              for k, v in zip(["mean", "log_scale", "quat", "opacity_logit", "sh"], scene.arrays())}
    cfg = api.RenderConfig(sort_mode="hier", key_tile=16)
    img = api.render_differentiable(R, params, 1, cams, None, cfg)
    target = torch.rand_like(img)
    loss = api.l1_ssim_loss(R, img, target)
    loss.backward()
    # the loss against its float64 definition
    L_ref, dimg_ref = ol.loss_and_grad(img.detach().cpu().numpy(), target.cpu().numpy())
    assert abs(loss.item() - L_ref) < 1e-5 * max(1.0, abs(L_ref))
    _, dimg = R.loss(img.detach(), target)
    assert rel_l2(dimg.cpu().numpy(), dimg_ref) < 1e-4
    # autograd path == explicit backward with the loss gradient
    ds = api.DeviceScene(*[p.detach() for p in params.values()], 1)
    R.render([ds], [0, 0], cams, None, cfg, save=True)
    g = ds.zeros_like()
    R.backward([ds], [0, 0], cams, None, cfg, dimg, [g])
    for p, t in zip(params.values(), g.tensors()):
        assert torch.allclose(p.grad, t, rtol=1e-5, atol=1e-9)


def test_backward_of_a_superseded_render_raises(R):
    """Two differentiable renders on one Renderer: the backward of the second is that
    render's gradient; the backward of the first, whose saved lists the second render
    replaced, raises instead of returning the second render's gradient."""
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(36)
    scene = random_scene(300, rng, sh_degree=0, z=(1.0, 3.0), xy=2.0, ls_mu=-2.5)
    params = {k: torch.tensor(np.asarray(v), device="cuda", requires_grad=True)
              for k, v in zip(["mean", "log_scale", "quat", "opacity_logit", "sh"], scene.arrays())}
    cfg = api.RenderConfig(sort_mode="hier", key_tile=16)
    cam_a = synth.identity_camera(40, 32, 90.0)
    cam_b = synth.camera_from_pose(synth.head_rotation(0.1), (0.05, 0, 0), 40, 32, synth.focal_for_hfov(40, 90.0))
    img_a = api.render_differentiable(R, params, 0, [cam_a], None, cfg)
    img_b = api.render_differentiable(R, params, 0, [cam_b], None, cfg)
    img_b.sum().backward()
    assert float(params["mean"].grad.abs().sum()) > 0
    with pytest.raises(RuntimeError, match="rendered again"):
        img_a.sum().backward()


def test_loss_kernel_matches_oracle_on_several_images(R):
    rng = np.random.default_rng(34)
    x = rng.uniform(size=(3, 3, 37, 53)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1).astype(np.float32)
    L_ref, g_ref = ol.loss_and_grad(x.astype(np.float64), y.astype(np.float64))
    loss, grad = R.loss(torch.tensor(x).cuda(), torch.tensor(y).cuda())
    assert abs(float(loss.item()) - L_ref) < 1e-5
    assert rel_l2(grad.cpu().numpy(), g_ref) < 1e-4


def test_adam_step_matches_its_definition(R):
    from paper_2505_10144_gb300 import api
    rng = np.random.default_rng(35)
    p0 = rng.normal(size=1000).astype(np.float32)
    p, m, v = (torch.tensor(a).cuda() for a in (p0.copy(), np.zeros(1000, np.float32), np.zeros(1000, np.float32)))
    pm, mm, vm = p0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t in range(1, 4):
        g = rng.normal(size=1000).astype(np.float32)
        api.adam_step(p, torch.tensor(g).cuda(), m, v, 1e-3, t, 0.9, 0.999, 1e-8)
        mm = 0.9 * mm + 0.1 * g
        vm = 0.999 * vm + 0.001 * g.astype(np.float64) ** 2
        pm = pm - 1e-3 * (mm / (1 - 0.9 ** t)) / (np.sqrt(vm / (1 - 0.999 ** t)) + 1e-8)
    torch.cuda.synchronize()
    assert np.abs(p.cpu().numpy() - pm).max() < 1e-5
