"""Learned block-pair scheduler around hfp_refine_round.

The paper's rounds refine every edge of the quotient graph (Section 5).  This
module adds a small perceptron (hfp_mlp_*) that scores each edge before the
round; pairs scoring below a threshold are skipped.  Everything numeric runs
in libhfp's kernels; this file only sequences the calls:

  collect()   runs plain (unpruned) rounds and records, per refined pair,
              its 16 features and the label "the pair's flow refinement
              found an improvement" (status OK and Delta_exp > 0);
  train()     full-batch Adam on those samples (hfp_mlp_train);
  refine()    rounds with or without the scheduler, returning the
              connectivity trajectory and the wall time; a pruned round
              without gain is repeated unpruned before refinement stops.

The paper's own pruning, active block scheduling (Section 5, "Parallel
Active Block Scheduling"), is here too: refine_active() refines every pair
in the first round and afterwards only the pairs with a block that an
applied move set of the previous round improved, and stops when no block is
active or a round improves (lambda - 1) by less than 0.1 %.  Its rounds are
synchronous; the paper interleaves the rounds' pairs in one queue.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import hfp


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform hidden layers, a small output layer, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (64, 16)) * np.sqrt(6 / 16) * 0.25
    W2 = rng.uniform(-1, 1, (64, 64)) * np.sqrt(6 / 64)
    w3 = rng.uniform(-1, 1, 64) * np.sqrt(6 / 128)
    z = np.zeros
    return np.concatenate([W1.reshape(-1), z(64), W2.reshape(-1), z(64), w3, z(1)]).astype(
        np.float32)


def _prev_from(results, k: int) -> np.ndarray:
    prev = -np.ones((k, k), np.int64)
    for r in results:
        prev[r.bi, r.bj] = r.gain if r.applied else 0
    return prev


@dataclass
class Samples:
    x: list = field(default_factory=list)      # float32[P, 16] per round
    y: list = field(default_factory=list)      # float32[P]
    pins: list = field(default_factory=list)   # int64[P]: network pins (cost proxy)

    def arrays(self):
        return (np.concatenate(self.x).astype(np.float32), np.concatenate(self.y).astype(np.float32),
                np.concatenate(self.pins))


def _round(hg, part_dev, k, params, scores=None, threshold=0.5, batched=True):
    if batched:
        stats, res, _ = hfp.refine_round_batched(hg, part_dev, k, params, pair_scores=scores,
                                                 min_score=threshold)
    else:
        stats, res = hfp.refine_round(hg, part_dev, k, params, pair_scores=scores,
                                      min_score=threshold)
    return stats, res


def collect(hg, part_dev, k: int, rounds: int = 2, params=None, samples: Samples | None = None,
            batched: bool = True):
    """Unpruned rounds on part_dev (updated); appends features and labels.
    The batched round gives the plain round's outcome, faster."""
    params = params or hfp.refine_params()
    samples = samples if samples is not None else Samples()
    prev = None
    for _ in range(rounds):
        pairs, feat = hfp.pair_features(hg, part_dev, k, params.eps_pct, prev)
        pairs = pairs.cpu().numpy()
        stats, res = _round(hg, part_dev, k, params, batched=batched)
        by = {(r.bi, r.bj): r for r in res}
        y = np.zeros(len(pairs), np.float32)
        pins = np.zeros(len(pairs), np.int64)
        for t, (i, j) in enumerate(pairs):
            r = by[(int(i), int(j))]
            y[t] = 1.0 if (r.status == hfp.OK and r.delta_exp > 0) else 0.0
            pins[t] = r.pins
        samples.x.append(feat.cpu().numpy())
        samples.y.append(y)
        samples.pins.append(pins)
        prev = _prev_from(res, k)
    return samples


def train(ctx, x: np.ndarray, y: np.ndarray, steps: int = 2000, lr: float = 3e-3, seed: int = 0):
    """Adam on (x, y) from init_params(seed) -> (params CUDA tensor, losses)."""
    import torch
    st = hfp.MlpState(torch.from_numpy(init_params(seed)).cuda())
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()
    losses = hfp.mlp_train(ctx, st, xd, yd, steps, lr=lr)
    return st.params, losses.cpu().numpy()


def refine(hg, part_dev, k: int, rounds: int, params=None, mlp_params=None,
           threshold: float = 0.5, batched: bool = True):
    """rounds of refinement (stopping early at a round without gain), pruned
    by the scheduler when mlp_params is given -> dict with the connectivity
    after each round, pairs refined and skipped, and the wall time."""
    import torch
    params = params or hfp.refine_params()
    prev = None
    conn, refined, skipped = [], 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fallbacks = 0
    for _ in range(rounds):
        scores = None
        if mlp_params is not None:
            scores = hfp.pair_scores(hg, part_dev, k, mlp_params, params.eps_pct, prev)
        stats, res = _round(hg, part_dev, k, params, scores, threshold, batched)
        refined += stats.pairs
        skipped += stats.pairs_skipped
        if stats.gain == 0 and scores is not None and stats.pairs_skipped > 0:
            # the unpruned schedule is the fallback: a pruned round without
            # gain is repeated with every pair before refinement stops
            fallbacks += 1
            stats, res = _round(hg, part_dev, k, params, None, threshold, batched)
            refined += stats.pairs
        conn.append(int(stats.connectivity_after))
        prev = _prev_from(res, k)
        if stats.gain == 0:
            break
    torch.cuda.synchronize()
    return dict(connectivity=conn, pairs=refined, skipped=skipped, fallbacks=fallbacks,
                seconds=time.perf_counter() - t0)


def active_blocks(results, k: int) -> np.ndarray:
    """Blocks of the pairs whose move set was applied with a positive gain."""
    act = np.zeros(k, bool)
    for r in results:
        if r.applied and r.gain > 0:
            act[r.bi] = act[r.bj] = True
    return act


def active_scores(active: np.ndarray) -> np.ndarray:
    """Pair scores selecting the pairs with an active block (1) over the
    others (0), for a round's min_score of 0.5."""
    a = active.astype(np.float32)
    return np.maximum(a[:, None], a[None, :]).astype(np.float32)


def refine_active(hg, part_dev, k: int, rounds: int, params=None, min_rel_gain: float = 0.001,
                  batched: bool = True):
    """Rounds under active block scheduling (see the module docstring) ->
    dict with the connectivity after each round, pairs refined and skipped,
    and the wall time."""
    import torch
    params = params or hfp.refine_params()
    conn, refined, skipped = [], 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    scores = None
    for _ in range(rounds):
        stats, res = _round(hg, part_dev, k, params, scores, 0.5, batched)
        refined += stats.pairs
        skipped += stats.pairs_skipped
        conn.append(int(stats.connectivity_after))
        act = active_blocks(res, k)
        before = int(stats.connectivity_before)
        if not act.any() or stats.gain < min_rel_gain * max(before, 1):
            break
        scores = active_scores(act)
    torch.cuda.synchronize()
    return dict(connectivity=conn, pairs=refined, skipped=skipped, fallbacks=0,
                seconds=time.perf_counter() - t0)
