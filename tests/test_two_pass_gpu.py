"""The two-pass foveated baseline (Appendix A) on the GPU against its oracle
composition: full-resolution centre square, half-resolution view, bilinear upsample and
w-blend.  Same parity rule as the render tests (tests/outcomes.py)."""
import numpy as np
import pytest

import outcomes as oc

from oracle import twopass as otp
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    r = api.Renderer()
    yield r
    r.close()


@pytest.mark.parametrize("mode,win", [("exact", (0, 0, 0)), ("hier", (4, 8, 16))])
def test_two_pass_matches_oracle(R, mode, win):
    from paper_2505_10144_gb300 import api
    scene = synth.shell_scene(30_000, synth.rng_for(1), sh_degree=3)
    W, H = 320, 256
    cams = synth.stereo_cameras((0.02, -0.01, 0.05), 0.3, W, H, 110.0)
    # one gaze near the border: the centre square is moved inside the image
    fov = [synth.fovea_for(W, (150.0, 120.0), radius_frac=0.2), synth.fovea_for(W, (300.0, 20.0), radius_frac=0.2)]
    bg = (0.1, 0.2, 0.3)
    ds = api.DeviceScene.from_host(scene)
    cfg = api.RenderConfig(sort_mode=mode, windows=win, fovea_mode="bilinear", bg=bg)
    gpu = R.render_two_pass([ds], [0, 0], cams, fov, cfg)
    R.check()
    gpu = gpu.cpu().numpy().astype(np.float64)
    for v in range(2):
        ref = otp.render(scene, cams[v], fov[v], mode, windows=win, bg=bg, outcomes=True)
        oc.check(gpu[v], ref, mode, label=f"two-pass {mode} eye {v}")


def test_two_pass_rejects_bad_arguments(R):
    from paper_2505_10144_gb300 import api
    scene = synth.shell_scene(1000, synth.rng_for(1), sh_degree=0)
    ds = api.DeviceScene.from_host(scene)
    cams = synth.stereo_cameras((0.0, 0.0, 0.0), 0.0, 65, 64, 110.0)  # odd width
    fov = [synth.fovea_for(65, (30.0, 30.0))] * 2
    with pytest.raises(RuntimeError):
        R.render_two_pass([ds], [0, 0], cams, fov, api.RenderConfig(fovea_mode="bilinear"))
    cams = synth.stereo_cameras((0.0, 0.0, 0.0), 0.0, 64, 64, 110.0)
    with pytest.raises(RuntimeError):  # plain fovea mode
        R.render_two_pass([ds], [0, 0], cams, [synth.fovea_for(64, (30.0, 30.0))] * 2, api.RenderConfig())
