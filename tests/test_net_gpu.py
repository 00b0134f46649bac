"""Periphery network kernels against the float64 oracle (oracle/net.py), the fused
tensor-core inference against the training forward, and what training buys over the
bilinear fallback on held-out crops.

Tolerance: activations are BF16 on both sides, rounded at the same three points; a
hidden value whose FP32 (GPU) and FP64 (oracle) pre-activation fall on opposite sides
of a BF16 rounding boundary moves by one BF16 ulp (2^-8 relative).  Such flips are rare
(the FP32 accumulation error is ~1e-6 of a value, a BF16 ulp ~4e-3), so the bound is a
small absolute error on almost every output plus a larger one on a few outputs."""
import numpy as np
import pytest
import torch

from oracle import net as onet
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import api, build
    build.build()
    r = api.Renderer()
    yield r
    r.close()


def oracle_forward(net, x):
    y, _ = onet.forward(torch.tensor(x, dtype=torch.float64), net.numpy_weights())
    return y.numpy()


def test_net_forward_matches_oracle(R):
    from paper_2505_10144_gb300 import periphery
    net = periphery.PeripheryNet(R, seed=1, last_scale=1.0)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, size=(2, 3, 37, 45)).astype(np.float32)
    y, acts = net.forward(torch.tensor(x).cuda())
    yr = oracle_forward(net, x)
    d = np.abs(y.cpu().numpy() - yr)
    assert np.quantile(d, 0.99) < 1e-3 and d.max() < 3e-2, (np.quantile(d, 0.99), d.max())


def test_net_backward_matches_oracle(R):
    from paper_2505_10144_gb300 import periphery
    net = periphery.PeripheryNet(R, seed=2, last_scale=1.0)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, size=(2, 3, 24, 33)).astype(np.float32)
    dy = rng.normal(size=x.shape).astype(np.float32)
    xt = torch.tensor(x).cuda()
    _, acts = net.forward(xt)
    net.backward(xt, acts, torch.tensor(dy).cuda())
    g = net.grad.cpu().numpy().astype(np.float64)
    gr = onet.grads(x.astype(np.float64), net.numpy_weights(), dy.astype(np.float64))
    for k, (o, shape) in periphery.OFF.items():
        a, b = g[o:o + int(np.prod(shape))], gr[k].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel < 2e-2, (k, rel)


def test_mse_kernel(R):
    from paper_2505_10144_gb300 import periphery
    net = periphery.PeripheryNet(R)
    rng = np.random.default_rng(3)
    y, t = rng.normal(size=(3, 1000)).astype(np.float32), rng.normal(size=(3, 1000)).astype(np.float32)
    loss, dy = net.mse(torch.tensor(y).cuda(), torch.tensor(t).cuda())
    assert abs(loss.item() - float(((y.astype(np.float64) - t) ** 2).mean())) < 1e-5
    assert np.allclose(dy.cpu().numpy(), 2 * (y - t) / y.size, rtol=1e-6, atol=1e-9)


@pytest.fixture(scope="module")
def vr_frame(R):
    from paper_2505_10144_gb300 import api
    scene = api.DeviceScene.from_host(synth.shell_scene(60_000, synth.rng_for(4), sh_degree=3))
    W, H = 320, 288
    cams = synth.stereo_cameras((0.02, 0.0, 0.0), 0.35, W, H, 110.0)
    fov = [synth.fovea_for(W, (150.0, 130.0), radius_frac=0.2), synth.fovea_for(W, (170.0, 140.0), radius_frac=0.2)]
    return scene, cams, fov, W, H


def test_fused_periphery_kernel_matches_training_forward(R, vr_frame):
    """Every tile in the periphery: the render's output is then bilinear(low) everywhere,
    the exact input of the network, so the fused tensor-core kernel must agree with the
    training forward (and the oracle) on the whole frame."""
    from paper_2505_10144_gb300 import api, periphery
    scene, cams, _, W, H = vr_frame
    allp = [periphery.ALL_PERIPHERY] * 2
    net = periphery.PeripheryNet(R, seed=4, last_scale=1.0)
    x = R.render([scene], [0, 0], cams, allp, api.RenderConfig(key_tile=32, fovea_mode="bilinear")).clone()
    low = torch.empty((2, 3, H // 2, W // 2), device="cuda")
    out = R.render([scene], [0, 0], cams, allp, api.RenderConfig(key_tile=32, fovea_mode="net"), low=low)
    net.apply_periphery(low, out)
    R.check()
    y, _ = net.forward(x, save=False)
    d = (out - y).abs()
    assert float(torch.quantile(d.flatten(), 0.99)) < 1e-3 and float(d.max()) < 3e-2
    yr = oracle_forward(net, x.cpu().numpy().astype(np.float64))
    dr = np.abs(out.cpu().numpy() - yr)
    assert np.quantile(dr, 0.99) < 1e-3 and dr.max() < 3e-2


def test_network_leaves_focus_and_hybrid_pixels_alone(R, vr_frame):
    from paper_2505_10144_gb300 import api, periphery
    scene, cams, fov, W, H = vr_frame
    net = periphery.PeripheryNet(R, seed=4, last_scale=1.0)
    bil = R.render([scene], [0, 0], cams, fov, api.RenderConfig(key_tile=32, fovea_mode="bilinear")).clone()
    low = torch.empty((2, 3, H // 2, W // 2), device="cuda")
    out = R.render([scene], [0, 0], cams, fov, api.RenderConfig(key_tile=32, fovea_mode="net"), low=low)
    net.apply_periphery(low, out)
    mask = periphery.periphery_mask(synth.Frame(cams, fov), W, H).cuda()
    assert mask.any() and (~mask).any()
    assert torch.equal(out.permute(1, 0, 2, 3)[:, ~mask], bil.permute(1, 0, 2, 3)[:, ~mask])
    assert float((out - bil).permute(1, 0, 2, 3)[:, mask].abs().max()) > 1e-3  # the network did act


def test_zero_last_layer_is_the_bilinear_fallback(R, vr_frame):
    from paper_2505_10144_gb300 import api, periphery
    scene, cams, fov, W, H = vr_frame
    net = periphery.PeripheryNet(R, seed=5, zero_last=True)
    bil = R.render([scene], [0, 0], cams, fov, api.RenderConfig(key_tile=32, fovea_mode="bilinear")).clone()
    low = torch.empty((2, 3, H // 2, W // 2), device="cuda")
    out = R.render([scene], [0, 0], cams, fov, api.RenderConfig(key_tile=32, fovea_mode="net"), low=low)
    net.apply_periphery(low, out)
    assert float((out - bil).abs().max()) < 1e-6


def test_training_beats_bilinear_on_held_out_crops(R):
    """Trained on the GPU by the library's own kernels, the network must reconstruct
    held-out periphery crops better than its bilinear fallback (the untrained network with
    a zero last layer is exactly the fallback)."""
    from paper_2505_10144_gb300 import api, periphery
    scene = api.DeviceScene.from_host(synth.shell_scene(100_000, synth.rng_for(4, salt=1), sh_degree=3))
    xs, ts = periphery.make_pairs(R, scene, 128, np.random.default_rng(10), crop=128)
    xv, tv = periphery.make_pairs(R, scene, 32, np.random.default_rng(11), crop=128)
    net = periphery.PeripheryNet(R, seed=6, zero_last=True)
    before = float(((xv - tv) ** 2).mean())
    losses = periphery.train(net, xs, ts, steps=400, batch=8, lr=1e-3)
    y, _ = net.forward(xv, save=False)
    after = float(((y - tv) ** 2).mean())
    assert losses[-40:].mean() < losses[:40].mean()
    assert after < 0.99 * before, (after, before)


def test_full_size_vr_frame_network_sampled_crops(R):
    """1M Gaussians, stereo 2064x2208, foveated with the network (the learned-periphery
    workload's frame): the fused tensor-core kernel runs once over every periphery tile of
    both eyes.  Crops of its output against the float64 network applied to the float64
    bilinear upsample of the GPU's half-resolution image (the network's input): the top-left
    and bottom-right corners (zero padding, the ragged last tile column) and an interior
    crop, each compared where the crop's 3-pixel halo is complete."""
    from oracle import grad as ograd
    from paper_2505_10144_gb300 import api, periphery
    W, H = 2064, 2208
    scene = api.DeviceScene.from_host(synth.shell_scene(1_000_000, synth.rng_for(4), sh_degree=3))
    fr = synth.vr_trajectory(3, synth.rng_for(4, salt=200), W, H).frames[2]
    net = periphery.PeripheryNet(R, seed=4, last_scale=1.0)
    low = torch.empty((2, 3, H // 2, W // 2), device="cuda")
    cfg = api.RenderConfig(sort_mode="hier", windows=(4, 8, 16), key_tile=32, fovea_mode="net")
    out = R.render([scene], [0, 0], fr.cameras, fr.foveas, cfg, low=low)
    net.apply_periphery(low, out)
    R.check()
    mask = periphery.periphery_mask(fr, W, H).numpy()
    outs = out.cpu().numpy().astype(np.float64)
    lows = low.cpu().numpy().astype(np.float64)
    checked = 0
    for v in range(2):
        x = ograd.bilinear_up2(torch.tensor(lows[v]))  # [3, H, W]
        # (crop origin, input window origin): outputs [y0, y0 + 64) x [x0, x0 + 64)
        for y0, x0 in [(0, 0), (64, W - 128), (H - 64, W - 64)]:
            wy0, wx0 = max(y0 - 3, 0), max(x0 - 3, 0)
            wy1, wx1 = min(y0 + 67, H), min(x0 + 67, W)
            assert mask[v, y0:y0 + 64, x0:x0 + 64].all()
            y, _ = onet.forward(x[None, :, wy0:wy1, wx0:wx1], net.numpy_weights())
            ref = y[0, :, y0 - wy0:y0 - wy0 + 64, x0 - wx0:x0 - wx0 + 64].numpy()
            d = np.abs(outs[v][:, y0:y0 + 64, x0:x0 + 64] - ref)
            assert np.quantile(d, 0.99) < 1e-3 and d.max() < 3e-2, (v, y0, x0, np.quantile(d, 0.99), d.max())
            assert np.abs(ref - x[:, y0:y0 + 64, x0:x0 + 64].numpy()).max() > 1e-3  # the network acts here
            checked += 1
    assert checked == 6
