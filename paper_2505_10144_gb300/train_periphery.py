"""Trains the periphery network of the learned-periphery frame and writes its weights.

  python -m paper_2505_10144_gb300.train_periphery [--pairs 2000] [--steps 80000]
      [--batch 8] [--lr 1e-3] [--seed 0] [--order exact|hier] [--out weights/periphery_1m.npy]

Workload: 1M Gaussians in the 6 m room shell (SH degree 3), 2064x2208 eyes at 110 deg.
Pairs: seeded random head poses, 256x256 crops, input = the all-periphery foveated render
(half-resolution group samples, bilinear upsample), target = the plain full-resolution
render of the same rays, both in the exact per-ray order by default, so that the target
differs from the input only by what reconstruction from half resolution loses.  The
network is evaluated on 200 held-out trajectory frames against the plain render, in the
exact order and in the hierarchical order the timed frame uses.
Learning rate: Adam at 1e-3 (10% linear warm-up, cosine decay) learns on every seed
tried; at 2e-3 most runs stall near the bilinear error (the batch-sampling seed decides
whether a run escapes), so the schedule is 1e-3 over 80k steps.
Every numeric step runs in libvrsplat kernels: the renders of the pairs, the network's
forward and backward, the loss and Adam.  The weights (11,011 float32: w1, b1, w2, b2,
w3, b3 in the layout of ``periphery.OFF``) go to a .npy file next to this module, which
``bench.py`` loads for the learned-periphery line.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "periphery_1m.npy")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=80000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0, help="seed of the batch sampling")
    ap.add_argument("--order", default="exact", choices=["exact", "hier"],
                    help="per-ray order of the training renders")
    ap.add_argument("--eval-frames", type=int, default=200)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args(argv)
    import torch

    from . import api, build, periphery, synth
    build.build()
    R = api.Renderer()
    scene = api.DeviceScene.from_host(synth.shell_scene(1_000_000, synth.rng_for(4), sh_degree=3))
    t0 = time.perf_counter()
    xs, ts = periphery.make_pairs(R, scene, args.pairs, np.random.default_rng(synth.BASE_SEED + 4), crop=256,
                                  sort_mode=args.order)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = periphery.PeripheryNet(R, seed=4, zero_last=True)
    t0 = time.perf_counter()
    losses = periphery.train(net, xs, ts, steps=args.steps, batch=args.batch, lr=args.lr, seed=args.seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del xs, ts
    frames = synth.vr_trajectory(args.eval_frames, synth.rng_for(4, salt=200)).frames
    t0 = time.perf_counter()
    ev = {f"exact_{k}": v for k, v in periphery.evaluate_frames(R, net, scene, frames, sort_mode="exact").items()}
    t_eval_exact = time.perf_counter() - t0
    ev.update({f"hier_{k}": v for k, v in periphery.evaluate_frames(R, net, scene, frames, sort_mode="hier").items()})
    ev["eval_exact_s"] = t_eval_exact
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, net.params.cpu().numpy())
    meta = {"weights": os.path.basename(args.out), "pairs": args.pairs, "steps": args.steps, "batch": args.batch,
            "lr": args.lr, "seed": args.seed, "order": args.order, "pairs_s": t_pairs, "train_s": t_train,
            "loss_first": float(losses[:50].mean()), "loss_last": float(losses[-50:].mean()),
            "eval_frames": len(frames), **ev}
    with open(args.out[:-4] + ".json", "w") as fh:
        json.dump(meta, fh, indent=1)
    print(json.dumps(meta), flush=True)
    R.close()


if __name__ == "__main__":
    main()
