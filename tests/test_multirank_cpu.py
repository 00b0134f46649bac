"""The benchmark's multi-rank logic on CPU with gloo, world size 2: every rank renders its
own trajectory of the same scene, the job's time is the slowest rank's (all-reduce max)
and the job's rate counts every rank's frames.  The render shards by view with no
exchange (replicas); fine-tuning is data-parallel over views, and its one exchange, the
all-reduce that averages the flat gradient buffer, is checked here with gloo ranks."""
import json
import os
import socket
import sys
from pathlib import Path

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank))
    import torch.distributed as dist
    sys.path.insert(0, str(ROOT))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        rate = bench.job_rate(ws, 120, slowest)
        wl = bench.rank_trajectory(4, rank)
        cam = wl.frames[2].cameras[0]
        rec = {"ws": bench.dist_setup()[0], "rank": bench.dist_setup()[1], "slowest": slowest, "rate": rate,
               "w2c": np.asarray(cam.world_to_cam).tolist(), "gaze": [wl.frames[2].foveas[0].gaze_x,
                                                                    wl.frames[2].foveas[0].gaze_y]}
        Path(out_dir, f"rank{rank}.json").write_text(json.dumps(rec))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark(tmp_path):
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    r0, r1 = (json.loads(Path(tmp_path, f"rank{r}.json").read_text()) for r in range(ws))
    assert (r0["ws"], r0["rank"], r1["rank"]) == (2, 0, 1)
    assert r0["slowest"] == r1["slowest"] == 15.0  # the max over ranks, on every rank
    assert r0["rate"] == r1["rate"] == pytest.approx(2 * 120 / 0.015)
    # weak scaling: the ranks render different frames of the trajectory's distribution
    assert r0["w2c"] != r1["w2c"] or r0["gaze"] != r1["gaze"]


def test_single_process_needs_no_group():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_rate(1, 30, 1500.0) == pytest.approx(20.0)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, str(ROOT))
    import bench

    class Args:
        steps, warmup, gpus = 1, 3, 2

    assert bench.run_reference(Args(), 2, 1) is None
    assert capsys.readouterr().out == ""


def _grad_worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank))
    import torch
    import torch.distributed as dist
    sys.path.insert(0, str(ROOT))
    from paper_2505_10144_gb300 import api, synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        scene = api.DeviceScene.from_host(synth.shell_scene(1000, synth.rng_for(3), sh_degree=3), device="cpu")
        grads, flat = scene.flat_zeros_like()
        g = torch.Generator().manual_seed(100 + rank)
        for t in grads.tensors():  # this rank's gradients, written through the views
            t.copy_(torch.randn(t.shape, generator=g))
        mine = [t.clone() for t in grads.tensors()]
        api.average_gradients(flat, dist)
        torch.save({"mine": mine, "avg": [t.clone() for t in grads.tensors()]}, Path(out_dir, f"g{rank}.pt"))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_flat_gradient_buffer_is_one_allocation_of_aligned_views():
    import torch
    sys.path.insert(0, str(ROOT))
    from paper_2505_10144_gb300 import api, synth
    scene = api.DeviceScene.from_host(synth.shell_scene(1001, synth.rng_for(3), sh_degree=3), device="cpu")
    grads, flat = scene.flat_zeros_like()
    base = flat.data_ptr()
    for t, p in zip(grads.tensors(), scene.tensors()):
        assert t.shape == p.shape and t.is_contiguous() and t.dtype == torch.float32
        off = (t.data_ptr() - base) // 4
        assert off % 64 == 0 and off + t.numel() <= flat.numel()
        t.fill_(1.0)
    assert float(flat.sum()) == sum(p.numel() for p in scene.tensors())  # parts are disjoint
    flat.zero_()
    assert all(float(t.abs().sum()) == 0.0 for t in grads.tensors())
    api.average_gradients(flat, None)  # no group: nothing to do


def test_two_gloo_ranks_average_the_flat_gradient_buffer(tmp_path):
    import torch
    ws = 2
    mp.start_processes(_grad_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    r = [torch.load(Path(tmp_path, f"g{k}.pt")) for k in range(ws)]
    for i in range(5):
        want = (r[0]["mine"][i] + r[1]["mine"][i]) / 2
        assert torch.allclose(r[0]["avg"][i], want, rtol=1e-6, atol=1e-7)
        assert torch.equal(r[0]["avg"][i], r[1]["avg"][i])  # every rank takes the same step
