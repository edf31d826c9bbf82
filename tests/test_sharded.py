"""The rank-sharded k-way round (paper_2201_01556_gb300.sharded) on CPU:
two gloo ranks split the block pairs of a round, refine their share with
the oracle (Algorithm 1's pair refinement), exchange the results with one
all-gather and apply them; both ranks must end with the partition and gain
of the single-process oracle round, for several splits."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth
from paper_2201_01556_gb300 import sharded

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, K, SEED = 6000, 16, 5


def _instance():
    inst = synth.instance("ring_n8M_zipf_k64", SEED, n=N, m=N * 3 // 2)
    return inst["H"], synth.kway_partition(N, K, 50_000, SEED)


def _oracle_round(H, part, pairs, sizes, group):
    part = np.array(part, np.int32)

    def refine(mine):
        return [oracle.refine_block_pair(H, part, K, i, j, seed=3) for i, j in mine]

    def apply(recs):
        return oracle.apply_round(H, part, K, recs)

    (total, gains), recs = sharded.round_sharded(pairs, sizes, refine, apply, group)
    return part, total, recs


def _worker(rank, world, port, sizes_kind, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        H, part = _instance()
        qn, _ = oracle.quotient(H, part, K)
        pairs = [(i, j) for i in range(K) for j in range(i + 1, K) if qn[i, j] > 0]
        sizes = [int(qn[i, j]) for i, j in pairs] if sizes_kind == "nets" else [1] * len(pairs)
        newp, total, recs = _oracle_round(H, part, pairs, sizes, None)
        owner = sharded.assign_pairs(sizes, world)
        q.put((rank, newp, total, [(r.bi, r.bj) for r in recs], int((owner == rank).sum())))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("sizes_kind", ["nets", "uniform"])
def test_two_gloo_ranks_match_the_single_process_round(sizes_kind):
    pytest.importorskip("torch")
    H, part = _instance()
    want_part, want_total, res, _ = oracle.refine_round(H, part, K, seed=3)
    assert want_total > 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes_kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = 0
    for rank, newp, total, keys, mine in out:
        assert np.array_equal(newp, want_part), f"rank {rank}: partition differs"
        assert total == want_total
        assert keys == [(r.bi, r.bj) for r in res]
        assert 0 < mine < len(res)
        shares += mine
    assert shares == len(res)


def test_one_process_round_equals_the_oracle_round():
    H, part = _instance()
    want_part, want_total, _, _ = oracle.refine_round(H, part, K, seed=3)
    qn, _ = oracle.quotient(H, part, K)
    pairs = [(i, j) for i in range(K) for j in range(i + 1, K) if qn[i, j] > 0]
    newp, total, _ = _oracle_round(H, part, pairs, [1] * len(pairs), None)
    assert np.array_equal(newp, want_part) and total == want_total


def test_assign_pairs_is_a_balanced_deterministic_split():
    rng = np.random.default_rng(1)
    sizes = rng.integers(1, 1000, 200)
    for world in (1, 2, 3, 8):
        owner = sharded.assign_pairs(sizes, world)
        assert np.array_equal(owner, sharded.assign_pairs(sizes, world))
        assert set(owner.tolist()) <= set(range(world))
        loads = np.bincount(owner, weights=sizes, minlength=world)
        # greedy LPT: no rank exceeds the mean by more than the largest job
        assert loads.max() <= sizes.sum() / world + sizes.max()
    assert sharded.assign_pairs([], 4).tolist() == []
