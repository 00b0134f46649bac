"""Periphery network kernels against the float64 oracle (oracle/net.py), and what
training buys over the bilinear fallback on held-out crops.

Tolerance, derived per output (oracle.net.forward_bound): the GPU accumulates in FP32
(its tensor-core kernel in the MMA's accumulation order) and rounds to BF16 at the same
three points as the oracle.  A sum of n products carries at most gamma_n sum |w a| of
accumulation error (unit roundoff 2^-23 here: one bit of slack for the order); a hidden
activation then rounds to the same BF16 value unless its pre-rounding value lies within
that reach of a rounding boundary, and it moves by at most the rounding of the reach's
ends otherwise; an output moves by its own accumulation error plus |w3| times the moves
of the activations it reads.  Every test asserts |GPU - oracle| <= that bound on every
output and prints the largest error and the bound's quantiles.

The training backward is mixed precision (dy and the hidden gradients rounded to BF16
where they enter a tensor-core contraction); it is compared with the oracle's gradients
rounded at the same places (oracle.net.grads_mixed), within the bound that function
derives the same way: accumulation error, rounding flips near BF16 boundaries, and the
forward's activation moves.

Inputs are seeded: random images, and for the fused kernel seeded half-resolution images
handed to vrs_net_periphery (its d_low argument), so neither side reads the other's
values."""
import numpy as np
import pytest
import torch

from oracle import grad as ograd
from oracle import net as onet
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu

U_ACC = 2.0 ** -23


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import api, build
    build.build()
    r = api.Renderer()
    yield r
    r.close()


def within_bound(gpu, x, net, label, x_err=0.0):
    """gpu: [B, 3, H, W] GPU outputs for the float64 network input x."""
    y, b = onet.forward_bound(torch.as_tensor(x, dtype=torch.float64), net.numpy_weights(), x_err=x_err, u=U_ACC)
    d = (torch.as_tensor(np.asarray(gpu, dtype=np.float64)) - y).abs()
    print(f"[net {label}] {d.numel()} outputs: max |d| {float(d.max()):.3g}, q99 {float(torch.quantile(d.flatten()[:2**24], 0.99)):.3g}; "
          f"bound q50 {float(torch.quantile(b.flatten()[:2**24], 0.5)):.3g}, max {float(b.max()):.3g}; "
          f"max |d| / bound {float((d / b).max()):.3f}")
    bad = d > b + 1e-7
    assert not bool(bad.any()), f"{label}: {int(bad.sum())} outputs beyond the derived bound (worst {float((d - b).max()):.3g})"
    return y


def test_net_forward_matches_oracle(R):
    from paper_2505_10144_gb300 import periphery
    net = periphery.PeripheryNet(R, seed=1, last_scale=1.0)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, size=(2, 3, 37, 45)).astype(np.float32)
    y, acts = net.forward(torch.tensor(x).cuda())
    within_bound(y.cpu().numpy(), x.astype(np.float64), net, "training forward")


def _net_case(R, seed, signed, shape):
    """A network and gradient case: random signs, or weights, biases, input and dy all
    >= 0 (no cancellation: the derived bound is then a small fraction of every gradient)."""
    from paper_2505_10144_gb300 import periphery
    net = periphery.PeripheryNet(R, seed=seed, last_scale=1.0)
    rng = np.random.default_rng(seed)
    if not signed:
        p = net.params.abs()
        for k in ("b1", "b2", "b3"):
            o, sh = periphery.OFF[k]
            p[o:o + int(np.prod(sh))] = torch.tensor(np.abs(rng.normal(0, 0.1, size=sh)), dtype=torch.float32)
        net.params.copy_(p)
    x = rng.uniform(0, 1, size=shape).astype(np.float32)
    dy = (rng.normal(size=shape) if signed else rng.uniform(0, 1, size=shape)).astype(np.float32)
    return net, x, dy


@pytest.mark.parametrize("signed,shape", [(True, (2, 3, 24, 33)), (False, (2, 3, 100, 130)), (True, (3, 3, 64, 128)),
                                          (False, (3, 3, 64, 128))])
def test_net_backward_matches_oracle(R, signed, shape):
    """Parameter gradients of the tensor-core backward against the oracle's mixed-
    precision gradients (oracle.net.grads_mixed: dy, dz2 and dz1 rounded to BF16 where
    they enter a contraction), every value within the derived bound: FP32 accumulation,
    BF16 rounding flips and the forward's activation moves.  Shapes span ragged 32 x 12
    convolution tiles and 64-pixel weight-gradient chunks, with widths that take the
    scalar (W % 8 != 0) and the 16-byte (W % 8 == 0) load paths.  The distance of the
    mixed-precision gradients from the straight-through float64 ones is printed."""
    from paper_2505_10144_gb300 import periphery
    net, x, dy = _net_case(R, 2, signed, shape)
    xt = torch.tensor(x).cuda()
    _, acts = net.forward(xt)
    net.grad.zero_()
    net.backward(xt, acts, torch.tensor(dy).cuda())
    R.check()
    g = net.grad.cpu().numpy().astype(np.float64)
    w = net.numpy_weights()
    gm, bnd = onet.grads_mixed(x.astype(np.float64), w, dy.astype(np.float64), bound=True, u=U_ACC)
    ex = onet.grads(x.astype(np.float64), w, dy.astype(np.float64))
    worst, worst_mix = 0.0, 0.0
    for k, (o, sh) in periphery.OFF.items():
        a = g[o:o + int(np.prod(sh))].reshape(sh)
        d = np.abs(a - gm[k])
        worst = max(worst, float((d / np.maximum(bnd[k], 1e-300)).max()))
        worst_mix = max(worst_mix, float(np.linalg.norm(gm[k] - ex[k]) / max(np.linalg.norm(ex[k]), 1e-30)))
        assert (d <= bnd[k]).all(), (k, float(d.max()), float(bnd[k][d > bnd[k]].min()))
        if not signed:  # tight: the accumulation term 2 gamma_n plus under 1% for the rest
            gn = onet._gamma(shape[0] * shape[2] * shape[3], U_ACC)
            assert (bnd[k] <= (1e-2 + 2 * gn) * np.abs(gm[k])).all(), k
    print(f"[net backward {'signed' if signed else 'sign-free'} {shape}] max |GPU - mixed| / bound {worst:.3f}; "
          f"mixed vs straight-through float64: relative L2 {worst_mix:.3g}")


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


def seeded_low(rng, shape):
    """A seeded half-resolution image with structure at every scale: a smooth gradient,
    blobs and pixel noise in [0, 1]."""
    V, C, H2, W2 = shape
    yy, xx = np.mgrid[0:H2, 0:W2] / max(H2, W2)
    img = 0.3 + 0.3 * np.sin(6 * xx + 3 * yy)[None, None] + 0.25 * rng.uniform(0, 1, size=shape)
    return np.clip(img, 0, 1).astype(np.float32)


def fused_periphery(R, scene, cams, fov, net, low_img):
    """A foveated render sets the tile classes; the fused kernel then reconstructs every
    periphery tile from low_img (handed to it in place of the render's own)."""
    from paper_2505_10144_gb300 import api
    W, H = cams[0].width, cams[0].height
    low = torch.empty((len(cams), 3, H // 2, W // 2), device="cuda")
    out = R.render([scene], [0] * len(cams), cams, fov, api.RenderConfig(key_tile=32, fovea_mode="net"), low=low)
    low.copy_(torch.from_numpy(low_img))
    net.apply_periphery(low, out)
    R.check()
    return out.cpu().numpy().astype(np.float64)


def test_fused_periphery_kernel_matches_oracle(R, vr_frame):
    """Every tile in the periphery: the fused tensor-core kernel's output on the whole
    frame against the float64 network on the float64 bilinear upsample of the same
    half-resolution image (the kernel upsamples in FP32: input error <= 4 ulp)."""
    from paper_2505_10144_gb300 import periphery
    scene, cams, _, W, H = vr_frame
    allp = [periphery.ALL_PERIPHERY] * 2
    net = periphery.PeripheryNet(R, seed=4, last_scale=1.0)
    low = seeded_low(np.random.default_rng(21), (2, 3, H // 2, W // 2))
    out = fused_periphery(R, scene, cams, allp, net, low)
    x = np.stack([ograd.bilinear_up2(torch.tensor(low[v].astype(np.float64))).numpy() for v in range(2)])
    within_bound(out, x, net, "fused kernel, whole frame", x_err=4 * 2.0 ** -24)


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
    """Stereo 2064x2208, foveated with the network (the learned-periphery frame's shape):
    the fused tensor-core kernel runs once over every periphery tile of both eyes, here
    from a seeded half-resolution image.  Crops of its output against the float64 network
    on the float64 bilinear upsample of that image: the top-left and bottom-right corners
    (zero padding, the ragged last tile column) and an interior crop, each where the
    crop's 3-pixel halo is complete, within the derived bound."""
    from paper_2505_10144_gb300 import api, periphery
    W, H = 2064, 2208
    scene = api.DeviceScene.from_host(synth.shell_scene(200_000, synth.rng_for(4), sh_degree=3))
    fr = synth.vr_trajectory(3, synth.rng_for(4, salt=200), W, H).frames[2]
    net = periphery.PeripheryNet(R, seed=4, last_scale=1.0)
    low = seeded_low(np.random.default_rng(22), (2, 3, H // 2, W // 2))
    outs = fused_periphery(R, scene, fr.cameras, fr.foveas, net, low)
    mask = periphery.periphery_mask(fr, W, H).numpy()
    checked = 0
    for v in range(2):
        x = ograd.bilinear_up2(torch.tensor(low[v].astype(np.float64)))  # [3, H, W]
        for y0, x0 in [(0, 0), (64, W - 128), (H - 64, W - 64)]:
            wy0, wx0 = max(y0 - 3, 0), max(x0 - 3, 0)
            wy1, wx1 = min(y0 + 67, H), min(x0 + 67, W)
            assert mask[v, y0:y0 + 64, x0:x0 + 64].all()
            xin = x[None, :, wy0:wy1, wx0:wx1]
            y, b = onet.forward_bound(xin, net.numpy_weights(), x_err=4 * 2.0 ** -24, u=U_ACC)
            sl = (slice(None), slice(None), slice(y0 - wy0, y0 - wy0 + 64), slice(x0 - wx0, x0 - wx0 + 64))
            d = np.abs(outs[v][None, :, y0:y0 + 64, x0:x0 + 64] - y[sl].numpy())
            bb = b[sl].numpy()
            print(f"[net full-size eye {v} at ({x0},{y0})] max |d| {d.max():.3g}, bound q50 {np.median(bb):.3g}, "
                  f"max |d| / bound {(d / bb).max():.3f}")
            assert (d <= bb + 1e-7).all(), (v, y0, x0, float((d - bb).max()))
            assert np.abs(y[sl].numpy() - xin[sl].numpy()).max() > 1e-3  # the network acts here
            checked += 1
    assert checked == 6
