"""Failure detection without a GPU fault: each bounded device wait of the library is run
against a flag that nothing sets.  The wait gives up after its limit, the kernel raises
the timeout status and returns; the host reads VRS_ERR_TIMEOUT at the next status check,
and the same context then renders normally."""
import numpy as np
import pytest

import outcomes as oc

from oracle import native as on
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    r = api.Renderer()
    yield r
    r.close()


@pytest.mark.parametrize("which", [0, 1], ids=["sort_lookback", "network_mbarrier"])
def test_bounded_wait_times_out_and_the_context_stays_usable(R, which):
    from paper_2505_10144_gb300 import _lib, api
    R.check()
    R.test_bounded_wait(which)
    with pytest.raises(_lib.VrsError) as e:
        R.check()
    assert e.value.status == 4  # VRS_ERR_TIMEOUT
    R.check()  # the status was cleared
    scene = synth.tiny_scene(2000, synth.rng_for(0))
    cam = synth.identity_camera(96, 64, 90.0)
    out = R.render([api.DeviceScene.from_host(scene)], [0], [cam], None, api.RenderConfig(sort_mode="exact"))
    R.check()
    oc.check(out.cpu().numpy()[0], oc.reference(scene, cam, "exact"), "exact", label="after a timeout")


def test_bounded_wait_rejects_unknown_waits(R):
    from paper_2505_10144_gb300 import _lib
    with pytest.raises(_lib.VrsError):
        R.test_bounded_wait(7)
