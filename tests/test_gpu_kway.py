"""Parity of the CUDA k-way refinement with the oracle (bit-exact): block
pair results (region size, cut, flow, Delta_exp, moves) and whole rounds
(final partition, gain, applied move sets)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_01556_gb300 import hfp
    hfp.load()
    ctx = hfp.ctx_create(0)
    yield torch, hfp, ctx


def _setup(env, seed, n, m, k=64):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n8M_zipf_k64", seed, n=n, m=m)
    H, part = inst["H"], inst["part"]
    if k != 64:
        part = synth.kway_partition(n, k, 50_000, seed)
    hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
    pd = torch.from_numpy(part.copy()).cuda()
    return H, part, hg, pd


@pytest.mark.parametrize("seed,n,m", [(1, 16000, 24000), (2, 64000, 96000)])
def test_pairs_match_oracle(env, seed, n, m):
    torch, hfp, ctx = env
    H, part, hg, pd = _setup(env, seed, n, m)
    assert hfp.connectivity(hg, pd, 64) == oracle.connectivity(H, part, 64)
    qn, _ = oracle.quotient(H, part, 64)
    pairs = [(i, j) for i in range(64) for j in range(i + 1, 64) if qn[i, j] > 0]
    rng = np.random.default_rng(seed)
    pick = [pairs[t] for t in rng.choice(len(pairs), min(16, len(pairs)), replace=False)]
    for i, j in pick:
        o = oracle.refine_block_pair(H, part, 64, i, j, seed=7)
        g, mv = hfp.refine_block_pair(hg, pd, 64, i, j, hfp.refine_params(seed=7))
        assert (g.status, g.region_size, g.original_cut) == (o.status, o.region_size,
                                                             o.original_cut), (i, j)
        assert g.pins == o.pins
        if o.status == oracle.OK:
            assert g.flow == o.flow and g.delta_exp == o.delta_exp
            assert np.array_equal(mv, o.moves)


@pytest.mark.parametrize("seed,n,m,k", [(3, 16000, 24000, 64), (4, 40000, 60000, 16)])
def test_round_matches_oracle(env, seed, n, m, k):
    torch, hfp, ctx = env
    H, part, hg, pd = _setup(env, seed, n, m, k)
    newp, total, res, gains = oracle.refine_round(H, part, k, seed=5)
    stats, pres = hfp.refine_round(hg, pd, k, hfp.refine_params(seed=5))
    got = pd.cpu().numpy()
    assert stats.gain == total
    assert stats.connectivity_before == oracle.connectivity(H, part, k)
    assert stats.connectivity_after == oracle.connectivity(H, newp, k)
    assert np.array_equal(got, newp)
    assert len(pres) == len(res)
    for g, o in zip(pres, res):
        assert (g.bi, g.bj, g.status, g.delta_exp, g.n_moves) == (o.bi, o.bj, o.status,
                                                                  o.delta_exp, len(o.moves))
        key = (o.bi, o.bj)
        if key in gains:
            assert (g.gain, g.applied, g.valid_moves) == gains[key]


def test_round_skips_low_scores(env):
    torch, hfp, ctx = env
    H, part, hg, pd = _setup(env, 6, 16000, 24000)
    scores = np.zeros((64, 64), np.float32)
    scores[0, 1] = scores[1, 2] = 1.0
    stats, pres = hfp.refine_round(hg, pd, 64, hfp.refine_params(), pair_scores=scores,
                                   min_score=0.5)
    assert {(p.bi, p.bj) for p in pres} <= {(0, 1), (1, 2)}
    assert stats.pairs_skipped > 0
    newp, total, _, _ = oracle.refine_round(H, part, 64, pairs=[(p.bi, p.bj) for p in pres])
    assert np.array_equal(pd.cpu().numpy(), newp) and stats.gain == total


def _km1_host(H, part):
    """(lambda - 1) recomputed from scratch on the host (Section 2): one
    64-bit block mask per net, its population count minus one, times w(e)."""
    bits = np.left_shift(np.uint64(1), part[H.pins].astype(np.uint64))
    off = H.net_off.astype(np.int64)
    masks = np.bitwise_or.reduceat(bits, off[:-1])
    masks[off[1:] == off[:-1]] = 0
    lam = np.array([bin(int(x)).count("1") for x in masks], np.int64) if masks.size < 10 \
        else np.unpackbits(masks.view(np.uint8).reshape(-1, 8), axis=1).sum(1).astype(np.int64)
    return int((np.maximum(lam - 1, 0) * H.net_w.astype(np.int64)).sum())


def test_round_certificate_1M(env):
    """A batched round at n = 1,000,000, k = 64 (too large for the oracle's
    round): the returned partition's (lambda - 1), recomputed on the host,
    equals connectivity_after and connectivity_before - gain; every applied
    move set has a non-negative actual gain (Section 5, "Apply Moves")."""
    torch, hfp, ctx = env
    n = 1_000_000
    H, part, hg, pd = _setup(env, 1, n, n * 3 // 2)
    before = _km1_host(H, part)
    stats, pres, _ = hfp.refine_round_batched(hg, pd, 64, group_ctas=4)
    after = _km1_host(H, pd.cpu().numpy())
    assert stats.connectivity_before == before
    assert stats.connectivity_after == after
    assert after == before - stats.gain
    assert stats.gain > 0
    applied = [p for p in pres if p.applied]
    assert applied and all(p.gain >= 0 for p in applied)
    assert sum(p.gain for p in applied) == stats.gain
    hg.close()


def _with_construction(hfp, ctx, mode):
    t = hfp.ctx_get_tuning(ctx)
    hfp.ctx_set_tuning(ctx, construction=mode)
    return t


@pytest.mark.parametrize("seed,n,m,k", [(7, 16000, 24000, 64), (8, 30000, 12000, 16)])
def test_sorted_construction_matches_oracle(env, seed, n, m, k):
    """The second construction algorithm (Section 6: the region's incidences
    sorted by net) gives the networks of the first: every refined pair's
    region, pin count, original cut, flow and moves equal the oracle's (whose
    construction is the first algorithm's), and so does a whole round.  The
    second case is a sparse hypergraph (|E| < |V| / 2), where the automatic
    choice takes the sorted construction."""
    torch, hfp, ctx = env
    H, part, hg, pd = _setup(env, seed, n, m, k)
    qn, _ = oracle.quotient(H, part, k)
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if qn[i, j] > 0]
    rng = np.random.default_rng(seed)
    pick = [pairs[t] for t in rng.choice(len(pairs), min(12, len(pairs)), replace=False)]
    base = _with_construction(hfp, ctx, 2)
    try:
        for i, j in pick:
            o = oracle.refine_block_pair(H, part, k, i, j, seed=7)
            g, mv = hfp.refine_block_pair(hg, pd, k, i, j, hfp.refine_params(seed=7))
            assert (g.status, g.region_size, g.original_cut, g.pins) == (
                o.status, o.region_size, o.original_cut, o.pins), (i, j)
            if o.status == oracle.OK:
                assert g.flow == o.flow and g.delta_exp == o.delta_exp
                assert np.array_equal(mv, o.moves)
        newp, total, _, _ = oracle.refine_round(H, part, k, seed=5)
        for mode in (0, 2):
            hfp.ctx_set_tuning(ctx, construction=mode)
            pd2 = torch.from_numpy(part.copy()).cuda()
            stats, _, _ = hfp.refine_round_batched(hg, pd2, k, hfp.refine_params(seed=5),
                                                   group_ctas=4)
            assert stats.gain == total
            assert np.array_equal(pd2.cpu().numpy(), newp)
    finally:
        hfp.ctx_set_tuning(ctx, **base)


def test_active_block_rounds_match_oracle(env):
    """Two rounds of active block scheduling (Section 5): the first refines
    every pair, the second only the pairs with a block that an applied move
    set improved; partition and connectivity equal the oracle's rounds on
    the same pair sets."""
    torch, hfp, ctx = env
    from paper_2201_01556_gb300 import scheduler
    H, part, hg, pd = _setup(env, 9, 16000, 24000)
    p1, _, _, gains1 = oracle.refine_round(H, part, 64)
    act = set()
    for (i, j), (gain, applied, _) in gains1.items():
        if applied and gain > 0:
            act |= {i, j}
    assert act
    qn, _ = oracle.quotient(H, p1, 64)
    pairs2 = [(i, j) for i in range(64) for j in range(i + 1, 64)
              if qn[i, j] > 0 and (i in act or j in act)]
    p2, _, _, _ = oracle.refine_round(H, p1, 64, pairs=pairs2)
    r = scheduler.refine_active(hg, pd, 64, rounds=2, min_rel_gain=0.0)
    assert r["connectivity"] == [oracle.connectivity(H, p1, 64), oracle.connectivity(H, p2, 64)]
    assert np.array_equal(pd.cpu().numpy(), p2)
    qn0, _ = oracle.quotient(H, part, 64)
    assert r["pairs"] == int((np.triu(qn0, 1) > 0).sum()) + len(pairs2)


def test_engine_autotuner_keeps_outcomes(env):
    """hfp_autotune_round_engine times the batched launch over its knob list
    (speed only) and keeps the fastest setting for the hypergraph; a batched
    round afterwards still equals the oracle's round."""
    torch, hfp, ctx = env
    H, part, hg, pd = _setup(env, 10, 16000, 24000)
    chosen, ms = hfp.autotune_round_engine(hg, pd, 64, group_ctas=4)
    assert len(ms) == 11 and (ms > 0).all()
    assert chosen["batch_gr_work_x100"] in (100, 200, 400)
    assert chosen["batch_stall_rounds_pierce"] in (0, 30, 100)
    assert (chosen["tail_enter"], chosen["tail_exit"]) in ((64, 192), (16, 64), (256, 768))
    assert chosen["batch_fused_rounds"] in (0, 1)
    assert np.array_equal(pd.cpu().numpy(), part)
    newp, total, _, _ = oracle.refine_round(H, part, 64, seed=5)
    stats, _, _ = hfp.refine_round_batched(hg, pd, 64, hfp.refine_params(seed=5), group_ctas=4)
    assert stats.gain == total
    assert np.array_equal(pd.cpu().numpy(), newp)


@pytest.mark.parametrize("streams,construction", [(1, 1), (3, 1), (16, 1), (5, 2)])
def test_prepare_streams_match_oracle(env, streams, construction):
    """Pair preparation on several host threads (each with a stream and
    region scratch of its own; pairs that share a block are prepared at the
    same time) gives the oracle's round: the same final partition and gain,
    and the same per-pair results, for the one-thread path, thread counts
    that do not divide the pair count, more threads than a round needs, and
    the second construction algorithm."""
    torch, hfp, ctx = env
    H, part, hg, pd = _setup(env, 11, 24000, 36000, 32)
    newp, total, res, _ = oracle.refine_round(H, part, 32, seed=5)
    base = hfp.ctx_get_tuning(ctx)
    try:
        hfp.ctx_set_tuning(ctx, prep_streams=streams, construction=construction)
        stats, pres, _ = hfp.refine_round_batched(hg, pd, 32, hfp.refine_params(seed=5),
                                                  group_ctas=4)
    finally:
        hfp.ctx_set_tuning(ctx, **base)
    assert stats.gain == total
    assert np.array_equal(pd.cpu().numpy(), newp)
    assert [(g.bi, g.bj, g.status, g.region_size, g.delta_exp, g.n_moves) for g in pres] == [
        (o.bi, o.bj, o.status, o.region_size, o.delta_exp, len(o.moves)) for o in res]
