"""Stereo reuse of distant content (Sec. 7's future work, vrs_render_stereo_reuse) on the
GPU against its oracle composition (oracle/reuse.py): near layer per eye, far layer
rendered once from the cyclopean eye, C_near + T_near (C_far + T_far bg).  Same parity
rule as the render tests (tests/outcomes.py), with the outcome sets of both layers."""
import numpy as np
import pytest
import torch

import outcomes as oc
from oracle import reuse as oreuse
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu

FAR = 92.0  # metres: 0.25 px of eye-to-cyclopean disparity at f = 722.6, IPD 64 mm


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    r = api.Renderer()
    yield r
    r.close()


@pytest.fixture(scope="module")
def landscape():
    scene = synth.open_room_with_landscape(30_000, 20_000, synth.rng_for(5), sh_degree=3)
    cams = synth.stereo_cameras((0.02, -0.01, 0.05), 0.25, 320, 256, 110.0, pitch=-0.15)
    return scene, cams


@pytest.mark.parametrize("mode,win", [("exact", (0, 0, 0)), ("hier", (4, 8, 16))])
def test_stereo_reuse_matches_oracle(R, landscape, mode, win):
    from paper_2505_10144_gb300 import api
    scene, cams = landscape
    bg = (0.05, 0.1, 0.2)
    ds = api.DeviceScene.from_host(scene)
    cfg = api.RenderConfig(sort_mode=mode, windows=win, key_tile=16, bg=bg)
    gpu = R.render_stereo_reuse(ds, cams, FAR, cfg)
    R.check()
    gpu = gpu.cpu().numpy().astype(np.float64)
    ref = oreuse.render(scene, cams, FAR, mode, windows=win, key_tile=16, bg=bg, outcomes=True)
    far_t = ref["far"]["full"][3]
    assert (far_t < 0.99).mean() > 0.05 and ref["far"]["stats"]["valid"] > 1000  # the far layer is in view
    for e in range(2):
        oc.check(gpu[e], {"image": ref["images"][e], "alt": ref["alt"][e], "unchecked": ref["unchecked"][e]}, mode,
                 label=f"stereo reuse {mode} eye {e}")


def test_stereo_reuse_without_far_layer_equals_the_fused_stereo_render(R, landscape):
    from paper_2505_10144_gb300 import api
    scene, cams = landscape
    ds = api.DeviceScene.from_host(scene)
    cfg = api.RenderConfig(sort_mode="hier", key_tile=16, bg=(0.3, 0.2, 0.1))
    a = R.render_stereo_reuse(ds, cams, 1e30, cfg).clone()
    b = R.render([ds], [0, 0], cams, None, cfg)
    R.check()
    assert torch.equal(a, b)


def test_stereo_reuse_rejects_bad_arguments(R, landscape):
    from paper_2505_10144_gb300 import api
    scene, cams = landscape
    ds = api.DeviceScene.from_host(scene)
    cfg = api.RenderConfig(sort_mode="hier", key_tile=16)
    other = synth.stereo_cameras((0.0, 0.0, 0.0), 0.5, 320, 256, 110.0)
    with pytest.raises(api.VrsError, match="INVALID"):  # the eyes' rotations differ
        R.render_stereo_reuse(ds, [cams[0], other[1]], FAR, cfg)
    with pytest.raises(api.VrsError, match="INVALID"):
        R.render_stereo_reuse(ds, cams, -1.0, cfg)
    with pytest.raises(api.VrsError, match="INVALID"):
        R.render_stereo_reuse(ds, cams, FAR, api.RenderConfig(sort_mode="global_z", key_tile=16))
