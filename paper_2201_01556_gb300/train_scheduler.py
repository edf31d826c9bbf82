"""Training recipe of the learned block-pair scheduler's committed weights.

    python -m paper_2201_01556_gb300.train_scheduler [--out PATH]

Collects outcomes of unpruned k-way rounds (batched, which gives the plain
round's outcome) on seeded instances of the k-way ring generator (2 +
Zipf(2.5) pins capped at 10,000, window 4,096, k contiguous arcs with 5 % of
the vertices moved to a neighbouring block), then trains the perceptron with
full-batch Adam on the GPU (hfp_mlp_train).  A pair's label is 1 when its
FlowCutter run found Delta_exp > 0.  The instances: n in {200,000, 500,000}
(m = 1.5 n), k in {16, 32, 64}, seeds 1-4, eight rounds each (the later
rounds, where most pairs no longer improve, are where pruning pays);
held-out evaluation uses seeds from 1001 on (eval_scheduler).  The weights,
the recipe and the training statistics are written to one .npz file; the
default path is the file bench.py and eval_scheduler load.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "scheduler_params.npz")
RECIPE = dict(n=[200_000, 500_000], k=[16, 32, 64], seeds=[1, 2, 3, 4], rounds=8, steps=3000,
              lr=3e-3, init_seed=0)


def collect_instances(hfp, scheduler, ctx, recipe, log=print):
    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    import synth
    S = scheduler.Samples()
    for n in recipe["n"]:
        inst = None
        for seed in recipe["seeds"]:
            inst = synth.instance("ring_n8M_zipf_k64", seed, n=n, m=n * 3 // 2)
            H = inst["H"]
            hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
            for k in recipe["k"]:
                part = inst["part"] if k == 64 else synth.kway_partition(n, k, 50_000, seed)
                t0 = time.perf_counter()
                before = len(S.y)
                scheduler.collect(hg, torch.from_numpy(part.copy()).cuda(), k,
                                  rounds=recipe["rounds"], samples=S)
                got = sum(len(y) for y in S.y[before:])
                log(f"n={n} seed={seed} k={k}: {got} samples in {time.perf_counter() - t0:.1f} s")
            hg.close()
    return S


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    from . import hfp, scheduler
    hfp.load()
    ctx = hfp.ctx_create(0)
    t0 = time.perf_counter()
    S = collect_instances(hfp, scheduler, ctx, RECIPE)
    X, y, pins = S.arrays()
    t1 = time.perf_counter()
    params, losses = scheduler.train(ctx, X, y, steps=RECIPE["steps"], lr=RECIPE["lr"],
                                     seed=RECIPE["init_seed"])
    t2 = time.perf_counter()
    info = dict(recipe=RECIPE, samples=int(len(y)), positive_rate=float(y.mean()),
                loss_first=float(losses[0]), loss_last=float(losses[-1]),
                collect_seconds=round(t1 - t0, 1), train_seconds=round(t2 - t1, 2))
    np.savez(args.out, params=params.cpu().numpy(), info=json.dumps(info))
    print(json.dumps(info))
    ctx.close()


def load_params(path: str = DEFAULT_OUT):
    """(float32[HFP_MLP_PARAMS] weights, recipe/statistics dict) or None."""
    if not os.path.exists(path):
        return None
    z = np.load(path)
    return z["params"].astype(np.float32), json.loads(str(z["info"]))


if __name__ == "__main__":
    main()
