"""vrs_probe_orders: the front-to-back blend order of single rays, GPU against the FP64
oracle's per-sample orders (index work: the Gaussian sequences must agree exactly,
except where the oracle flags the pixel as marginal or two pairs are tied to within
FP32 reach of their order key)."""
import numpy as np
import pytest
import torch

from oracle import native as on
from paper_2505_10144_gb300 import synth

pytestmark = pytest.mark.gpu

W, H = 160, 128
TIE_REL = 1e-5  # FP32 reach of an order key computed in a few dependent operations


@pytest.fixture(scope="module")
def R():
    from paper_2505_10144_gb300 import build
    build.build()
    from paper_2505_10144_gb300 import api
    r = api.Renderer()
    yield r
    r.close()


@pytest.fixture(scope="module")
def view():
    scene = synth.shell_scene(20_000, synth.rng_for(1), sh_degree=3)
    cam = synth.stereo_cameras((0.02, 0.0, 0.03), 0.4, W, H, 110.0)[0]
    return scene, cam


def pixel_probes(view_index=0, step=1):
    ys, xs = np.mgrid[0:H:step, 0:W:step]
    p = np.stack([np.full(xs.size, view_index, np.float32), xs.ravel() + 0.5, ys.ravel() + 0.5], 1)
    return torch.tensor(p, dtype=torch.float32).cuda(), ys.ravel(), xs.ravel()


def order_key(scene, cam, mode):
    """Per-Gaussian global order key (FP64) of the global modes."""
    Rw = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    mu = np.asarray(scene.mean, np.float64)
    pc = Rw[:, :3] @ mu + Rw[:, 3:4]
    return pc[2] if mode == "global_z" else np.linalg.norm(pc, axis=0)


def inverted_pairs(a, b):
    """Pairs (i, j) ordered i before j in a and j before i in b (common elements only)."""
    pos = {g: k for k, g in enumerate(b)}
    common = [g for g in a if g in pos]
    out = []
    for x in range(len(common)):
        for y in range(x + 1, len(common)):
            if pos[common[x]] > pos[common[y]]:
                out.append((common[x], common[y]))
    return out


def run(R, scene, cam, mode, max_len=512):
    from paper_2505_10144_gb300 import api
    ds = api.DeviceScene.from_host(scene)
    R.render([ds], [0], [cam], None, api.RenderConfig(sort_mode=mode, key_tile=16))
    R.check()
    probes, ys, xs = pixel_probes()
    ids, depth, length = R.probe_orders(probes, max_len)
    R.check()
    return ids.cpu().numpy(), depth.cpu().numpy(), length.cpu().numpy(), ys, xs


@pytest.mark.parametrize("mode", ["exact", "global_z", "global_dist"])
def test_probe_orders_match_oracle(R, view, mode):
    scene, cam = view
    ids, depth, length, ys, xs = run(R, scene, cam, mode)
    assert length.max() < ids.shape[1]
    ref = on.render(scene, cam, mode, key_tile=16, want_orders=True)
    order, off = ref["orders"]
    marg = ref["marginal"]
    gkey = None if mode == "exact" else order_key(scene, cam, mode)
    unexplained, near_tie, compared, blended = 0, 0, 0, 0
    for k in range(len(ys)):
        y, x = ys[k], xs[k]
        if marg[y, x]:
            continue
        want = order[off[y * W + x]:off[y * W + x + 1]]
        got = ids[k, :length[k]]
        compared += 1
        blended += len(want)
        if np.array_equal(got, want):
            continue
        tgot = dict(zip(got.tolist(), depth[k, :length[k]].tolist()))
        ok = set(got.tolist()) == set(want.tolist())
        for i, j in inverted_pairs(want.tolist(), got.tolist()):
            if gkey is None:
                ki, kj = tgot[i], tgot[j]
            else:
                ki, kj = gkey[i], gkey[j]
            ok &= abs(ki - kj) <= TIE_REL * max(abs(ki), abs(kj))
        if ok:
            near_tie += 1
        else:
            unexplained += 1
    assert unexplained == 0, f"{unexplained} non-marginal rays blend another order ({near_tie} near ties)"
    assert near_tie <= 0.005 * compared
    assert compared > 0.9 * len(ys) and blended > 5 * compared


def test_probe_exact_order_is_ascending_depth(R, view):
    scene, cam = view
    ids, depth, length, _, _ = run(R, scene, cam, "exact")
    for k in range(0, len(length), 7):
        d, g = depth[k, :length[k]], ids[k, :length[k]]
        assert np.all((d[1:] > d[:-1]) | ((d[1:] == d[:-1]) & (g[1:] > g[:-1])))


def test_probe_truncation_and_bounds(R, view):
    from paper_2505_10144_gb300 import api
    scene, cam = view
    ids, _, length, ys, xs = run(R, scene, cam, "exact")
    k = int(np.argmax(length))
    probes = torch.tensor([[0, xs[k] + 0.5, ys[k] + 0.5], [0, -1.0, 3.0], [0, W + 0.5, 3.0], [1, 5.5, 5.5],
                           [0.5, 5.5, 5.5]], dtype=torch.float32).cuda()
    i4, _, l4 = R.probe_orders(probes, 4)
    R.check()
    l4 = l4.cpu().numpy()
    assert l4[0] == length[k] and l4[0] > 4
    assert np.array_equal(i4[0].cpu().numpy(), ids[k, :4])
    assert list(l4[1:]) == [-1, -1, -1, -1]
    R.render([api.DeviceScene.from_host(scene)], [0], [cam], None, api.RenderConfig(sort_mode="hier", key_tile=16))
    with pytest.raises(RuntimeError):
        R.probe_orders(probes, 4)
