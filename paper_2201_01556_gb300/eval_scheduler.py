"""Plain vs batched vs batched + learned k-way refinement on held-out seeds.

    python -m paper_2201_01556_gb300.eval_scheduler [--n 200000] [--k 16,32,64]
        [--seeds 1001,1002,1003] [--rounds 10] [--threshold 0.5] [--no-plain]

Every arm starts from the same partition and runs up to `rounds` rounds
(stopping at a round without gain): the plain round (hfp_refine_round, one
FlowCutter problem at a time), the batched round (hfp_refine_round_batched,
identical outcome), the batched round pruned by the learned scheduler with
the committed weights (train_scheduler), and batched rounds under the
paper's active block scheduling (scheduler.refine_active).  Prints one JSON object with
per-arm totals: wall seconds, pairs refined, final (lambda - 1), and the
relative (lambda - 1) difference of the learned arm to the unpruned one.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def compare(hfp, scheduler, ctx, H, part, k, rounds, mlp_params, threshold=0.5, plain=True):
    """The three arms on one instance -> dict of per-arm results."""
    import torch
    hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
    out = {}
    arms = [("batched", True, None), ("learned", True, mlp_params)]
    if plain:
        arms.insert(0, ("plain", False, None))
    finals = {}
    for name, batched, mp in arms:
        pd = torch.from_numpy(part.copy()).cuda()
        r = scheduler.refine(hg, pd, k, rounds, mlp_params=mp, threshold=threshold,
                             batched=batched)
        finals[name] = pd.cpu().numpy()
        out[name] = r
    # the paper's active block scheduling (batched rounds)
    pd = torch.from_numpy(part.copy()).cuda()
    out["active"] = scheduler.refine_active(hg, pd, k, rounds)
    if plain:
        # the batched round is the plain round run differently: same partition
        out["plain"]["identical_to_batched"] = bool(np.array_equal(finals["plain"],
                                                                   finals["batched"]))
    hg.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--k", default="16,32,64")
    ap.add_argument("--seeds", default="1001,1002,1003")
    ap.add_argument("--rounds", type=int, default=10)
    ap.add_argument("--threshold", type=float, default=0.5)
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    import torch
    import synth
    from . import hfp, scheduler, train_scheduler
    hfp.load()
    loaded = train_scheduler.load_params()
    if loaded is None:
        raise SystemExit("no committed scheduler weights: run train_scheduler first")
    params = torch.from_numpy(loaded[0]).cuda()
    ctx = hfp.ctx_create(0)
    tot = {a: dict(seconds=0.0, pairs=0, connectivity=0)
           for a in ("plain", "batched", "learned", "active")}
    rows = []
    for seed in [int(s) for s in args.seeds.split(",")]:
        inst = synth.instance("ring_n8M_zipf_k64", seed, n=args.n, m=args.n * 3 // 2)
        for k in [int(x) for x in args.k.split(",")]:
            part = inst["part"] if k == 64 else synth.kway_partition(args.n, k, 50_000, seed)
            r = compare(hfp, scheduler, ctx, inst["H"], part, k, args.rounds, params,
                        args.threshold, plain=not args.no_plain)
            rows.append(dict(seed=seed, k=k, **{a: dict(seconds=round(v["seconds"], 3),
                                                          pairs=v["pairs"],
                                                          connectivity=v["connectivity"][-1],
                                                          rounds=len(v["connectivity"]))
                                                 for a, v in r.items()}))
            if "plain" in r:
                rows[-1]["plain_identical_to_batched"] = r["plain"]["identical_to_batched"]
            for a, v in r.items():
                tot[a]["seconds"] += v["seconds"]
                tot[a]["pairs"] += v["pairs"]
                tot[a]["connectivity"] += v["connectivity"][-1]
    res = dict(n=args.n, rounds=args.rounds, threshold=args.threshold, per_instance=rows,
               totals={a: v for a, v in tot.items() if v["pairs"]},
               learned_vs_unpruned=(tot["learned"]["connectivity"] / tot["batched"]["connectivity"]
                                    - 1.0) if tot["batched"]["connectivity"] else None)
    print(json.dumps(res))
    ctx.close()
    return res


if __name__ == "__main__":
    main()
