"""The round in three calls (hfp_round_pairs, hfp_refine_pairs_batched,
hfp_apply_moves) on the GPU: any split of the pairs, refined separately and
applied together in any order, gives hfp_refine_round_batched's outcome
(and through it the oracle round's)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2201_01556_gb300 import hfp
    hfp.load()
    ctx = hfp.ctx_create(0)
    yield torch, hfp, ctx
    ctx.close()


def _setup(env, seed, n, k):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n8M_zipf_k64", seed, n=n, m=n * 3 // 2)
    H = inst["H"]
    part = inst["part"] if k == 64 else synth.kway_partition(n, k, 50_000, seed)
    hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
    return H, part, hg


FIELDS = ("bi", "bj", "status", "region_size", "pins", "original_cut", "flow", "delta_exp",
          "n_moves", "iterations", "applied", "valid_moves", "gain")


@pytest.mark.parametrize("seed,n,k,world", [(5, 6000, 16, 2), (3, 16000, 64, 3),
                                            (4, 40000, 16, 2)])
def test_split_rounds_equal_the_batched_round(env, seed, n, k, world):
    torch, hfp, ctx = env
    from paper_2201_01556_gb300 import sharded
    H, part, hg = _setup(env, seed, n, k)
    prm = hfp.refine_params(seed=5)
    p1 = torch.from_numpy(part.copy()).cuda()
    s1, r1, _ = hfp.refine_round_batched(hg, p1, k, prm, group_ctas=4)

    p2 = torch.from_numpy(part.copy()).cuda()
    pairs, nets, conn = hfp.round_pairs(hg, p2, k)
    assert conn == s1.connectivity_before and len(pairs) == s1.pairs
    assert [tuple(p) for p in pairs.tolist()] == [(r.bi, r.bj) for r in r1]
    qn, _ = oracle.quotient(H, part, k)
    assert nets.tolist() == [int(qn[i, j]) for i, j in pairs.tolist()]
    owner = sharded.assign_pairs(nets, world)
    results, moves = [], []
    for r in range(world):          # the ranks' shares, one after another
        mine = pairs[owner == r]
        res, mv, off, _ = hfp.refine_pairs_batched(hg, p2, k, mine, prm, group_ctas=4)
        assert off[-1] == len(mv)
        for t, x in enumerate(res):
            results.append(x)
            moves.append(mv[off[t]:off[t + 1]])
    # gathered in rank order, applied in the round's own order
    perm = np.random.default_rng(seed).permutation(len(results))
    results = [results[i] for i in perm]
    moves = [moves[i] for i in perm]
    off = np.zeros(len(results) + 1, np.int64)
    off[1:] = np.cumsum([len(m) for m in moves])
    s2, r2 = hfp.apply_moves(hg, p2, k, results, np.concatenate(moves), off, prm)
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    for f in ("connectivity_before", "connectivity_after", "gain", "moves_applied", "pairs",
              "pairs_improved", "pairs_applied"):
        assert getattr(s1, f) == getattr(s2, f), f
    got = {(x.bi, x.bj): x for x in r2}
    for a in r1:
        b = got[(a.bi, a.bj)]
        for f in FIELDS:
            assert getattr(a, f) == getattr(b, f), f
    hg.close()


def test_sharded_module_in_one_process(env):
    torch, hfp, ctx = env
    from paper_2201_01556_gb300 import sharded
    H, part, hg = _setup(env, 6, 30000, 16)
    p1 = torch.from_numpy(part.copy()).cuda()
    p2 = torch.from_numpy(part.copy()).cuda()
    s1, r1, _ = hfp.refine_round_batched(hg, p1, 16, hfp.refine_params(seed=2), group_ctas=4)
    s2, r2 = sharded.refine_round_sharded(hg, p2, 16, hfp.refine_params(seed=2), group_ctas=4)
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    assert s1.gain == s2.gain and s1.connectivity_after == s2.connectivity_after
    newp, total, _, _ = oracle.refine_round(H, part, 16, seed=2)
    assert np.array_equal(p2.cpu().numpy(), newp) and s2.gain == total
    hg.close()


def test_apply_moves_rejects_inconsistent_input(env):
    torch, hfp, ctx = env
    H, part, hg = _setup(env, 5, 6000, 16)
    pd = torch.from_numpy(part.copy()).cuda()
    pairs, _, _ = hfp.round_pairs(hg, pd, 16)
    res, mv, off, _ = hfp.refine_pairs_batched(hg, pd, 16, pairs)
    t = int(np.argmax([r.n_moves for r in res]))
    assert res[t].n_moves > 0
    bad_off = off.copy()
    bad_off[t + 1:] += 1                     # one move more than the result says
    padded = np.concatenate([mv, np.zeros((1, 3), np.int32)])
    with pytest.raises(hfp.HfpError) as e:
        hfp.apply_moves(hg, pd, 16, res, padded, bad_off)
    assert e.value.status == hfp.ERR_INVALID
    bad = mv.copy()
    bad[off[t], 2] = next(b for b in range(16) if b not in (res[t].bi, res[t].bj))
    with pytest.raises(hfp.HfpError):
        hfp.apply_moves(hg, pd, 16, res, bad, off)
    with pytest.raises(hfp.HfpError):
        hfp.refine_pairs_batched(hg, pd, 16, [[3, 3]])
    with pytest.raises(hfp.HfpError):
        hfp.refine_pairs_batched(hg, pd, 16, [[0, 1], [0, 1]])
    # nothing was applied by the rejected calls
    assert np.array_equal(pd.cpu().numpy(), part)
    hg.close()
