"""The benchmark's multi-rank logic on CPU with gloo, world size 2: every rank renders its
own trajectory of the same scene, the job's time is the slowest rank's (all-reduce max)
and the job's rate counts every rank's frames.  The GPU path is replicas only (the render
shards by view with no exchange), so this host logic is all there is to the N > 1 path."""
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
