"""The k-way round with its block pairs split across processes, one GPU each.

Algorithm 1 refines every block pair of a round against the same partition
and applies the move sets only afterwards (Section 5, "Parallel Scheduling"
and "Apply Moves").  The pairs are therefore independent problems.  Each
rank refines its share in one batched launch (hfp_refine_pairs_batched).
The ranks then exchange results and moves once (an all-gather), and every
rank applies all of them in the same deterministic order (hfp_apply_moves:
descending Delta_exp, ties ascending (i, j)).  The partitions stay identical
on all ranks without further communication, and the outcome is the
single-process round's whatever the split.

round_sharded() is the rank logic, independent of where the pairs are
refined; refine_round_sharded() runs it on the library.
"""
from __future__ import annotations

import numpy as np

from . import hfp


def assign_pairs(sizes, world: int) -> np.ndarray:
    """Longest-processing-time split: pairs in descending size (ties:
    ascending index) each go to the rank with the smallest total so far
    (ties: lowest rank).  Returns the owning rank of every pair."""
    sizes = np.asarray(sizes, np.int64)
    owner = np.zeros(len(sizes), np.int32)
    load = np.zeros(max(world, 1), np.int64)
    for t in sorted(range(len(sizes)), key=lambda t: (-int(sizes[t]), t)):
        r = int(np.argmin(load))
        owner[t] = r
        load[r] += max(int(sizes[t]), 1)
    return owner


def _rank_world(group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def gather(obj, group=None) -> list:
    """Every rank's obj, in rank order (one process: [obj])."""
    rank, world = _rank_world(group)
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, obj, group=group)
    return out


def round_sharded(pairs, sizes, refine, apply, group=None):
    """One round over `pairs` ((i, j) list, the same on every rank) split by
    assign_pairs(sizes).  refine(my_pairs) returns one record per pair with
    attributes or keys bi, bj; apply(all_records) applies them and returns
    the round's statistics.  Returns (statistics, records in pair order)."""
    rank, world = _rank_world(group)
    owner = assign_pairs(sizes, world)
    mine = [(int(p[0]), int(p[1])) for t, p in enumerate(pairs) if owner[t] == rank]
    recs = refine(mine)
    everyone = [r for part in gather(recs, group) for r in part]

    def key(r):
        return (r["bi"], r["bj"]) if isinstance(r, dict) else (r.bi, r.bj)
    everyone.sort(key=key)
    if [key(r) for r in everyone] != sorted((int(i), int(j)) for i, j in pairs):
        raise RuntimeError("the ranks' results do not cover the round's pairs")
    return apply(everyone), everyone


def _result_dict(r) -> dict:
    return {name: getattr(r, name) for name, _ in hfp.PairResult._fields_}


def refine_round_sharded(hg, part_dev, k: int, params=None, group_ctas: int = 0, group=None,
                         pair_scores=None, min_score: float = 0.0):
    """One k-way round of the library with the block pairs split across the
    ranks of `group` (torch.distributed; one process without it).  part_dev
    (this rank's device copy of the partition, identical on all ranks) is
    updated in place on every rank.  Returns (RoundStats, [PairResult])."""
    params = params or hfp.refine_params()
    pairs, nets, _ = hfp.round_pairs(hg, part_dev, k, pair_scores, min_score)

    def refine(mine):
        if not mine:
            return []
        res, moves, off, _ = hfp.refine_pairs_batched(hg, part_dev, k, mine, params, group_ctas)
        return [{"bi": r.bi, "bj": r.bj, "result": _result_dict(r),
                 "moves": moves[off[t]:off[t + 1]].copy()} for t, r in enumerate(res)]

    def apply(recs):
        results = [hfp.PairResult(**r["result"]) for r in recs]
        moves = [r["moves"] for r in recs]
        off = np.zeros(len(recs) + 1, np.int64)
        off[1:] = np.cumsum([len(m) for m in moves])
        allm = np.concatenate(moves) if moves else np.zeros((0, 3), np.int32)
        return hfp.apply_moves(hg, part_dev, k, results, allm, off, params)

    (stats, results), _ = round_sharded(pairs, nets, refine, apply, group)
    return stats, results
