"""Pins of the oracle's k-way pieces (CPU only): connectivity, quotient
graph, region growing, apply-moves rules, refine_block_pair and the round
(Section 4 Algorithm 1, Section 5, Section 6)."""
import numpy as np

import oracle
import synth
from tests.helpers import hypergraph_from_lists


def _small_kway():
    # 9 vertices in 3 blocks: {0,1,2} {3,4,5} {6,7,8}
    nets = [[0, 1], [1, 3], [2, 4, 6], [5, 7], [7, 8], [0, 8], [3, 4, 5]]
    w = [1, 2, 3, 4, 5, 6, 7]
    H = hypergraph_from_lists(9, nets, w)
    part = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2], np.int32)
    return H, part


def test_connectivity_hand_example():
    H, part = _small_kway()
    # lambda - 1 per net: [0, 1, 2, 1, 0, 1, 0] -> 2 + 2*3 + 4 + 6 = 18
    assert oracle.connectivity(H, part, 3) == 18


def test_connectivity_k2_is_the_hypergraph_cut():
    """For k = 2, (lambda - 1) is the cut weight (Section 2)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(5, 40))
        nets = [sorted(rng.choice(n, int(rng.integers(2, 6)), replace=False).tolist())
                for _ in range(int(rng.integers(3, 60)))]
        H = hypergraph_from_lists(n, nets, rng.integers(1, 9, len(nets)))
        part = rng.integers(0, 2, n).astype(np.int32)
        net = oracle.build_network(H, part, np.arange(n, dtype=np.int32))
        assert oracle.connectivity(H, part, 2) == oracle.cut_weight(net, np.r_[True, False, part == 0])


def test_quotient_hand_example():
    H, part = _small_kway()
    qn, qw = oracle.quotient(H, part, 3)
    # pairs: (0,1): nets 1, 2 -> 2 nets, weight 5; (0,2): nets 2, 5 -> 9; (1,2): nets 2, 3 -> 7
    assert (qn[0, 1], qw[0, 1]) == (2, 5)
    assert (qn[0, 2], qw[0, 2]) == (2, 9)
    assert (qn[1, 2], qw[1, 2]) == (2, 7)


def test_grow_region_hand_example():
    H, part = _small_kway()
    region, dist = oracle.grow_region(H, part, 0, 1, alpha_eps_pct=48, delta=2)
    # cut nets of (0,1): {1,3}, {2,4,6}: block 0 pins 1, 2 (dist 1), block 1 pins 3, 4 (dist 1);
    # bound per side: floor(1.48 * 3) - 3 = 1 -> only the first vertex of each side fits
    assert region.tolist() == [1, 3]
    assert dist.tolist() == [1, 1]
    region, dist = oracle.grow_region(H, part, 0, 1, alpha_eps_pct=300, delta=2)
    # bound 4*3 - 3 = 9: all of level 1, then level 2: 0 (via {0,1}) and 5 (via {3,4,5})
    assert region.tolist() == [0, 1, 2, 3, 4, 5]
    assert dist.tolist() == [2, 1, 1, 1, 1, 2]


def test_grow_region_properties():
    inst = synth.instance("ring_n8M_zipf_k64", 2, n=16000, m=24000)
    H, part = inst["H"], inst["part"]
    W = {b: int(H.node_w[part == b].sum()) for b in range(64)}
    for bi, bj in [(0, 1), (5, 6), (10, 11), (63, 0)]:
        i, j = min(bi, bj), max(bi, bj)
        region, dist = oracle.grow_region(H, part, i, j, 48, 2)
        assert np.all(np.diff(region) > 0)
        assert set(np.unique(part[region])) <= {i, j}
        assert dist.min() >= 1 and dist.max() <= 2
        lim = (148 * ((W[i] + W[j] + 1) // 2)) // 100
        for b, o in ((i, j), (j, i)):
            assert int(H.node_w[region[part[region] == b]].sum()) <= max(0, lim - W[o])


def test_apply_moves_rules():
    H, part = _small_kway()
    L = 4
    p = part.copy()
    # moving 1 to block 1 and 4 to block 0: net {1,3} stops being cut (+2),
    # net {2,4,6} keeps blocks 0 and 2 but loses block 1 (+3), net {0,1} becomes
    # cut (-1), net {3,4,5} becomes cut (-7): 18 -> 23, so it is reverted
    g, applied, nv = oracle.apply_moves(H, p, 3, L, np.array([[1, 0, 1], [4, 1, 0]], np.int32))
    assert (g, applied, nv) == (0, 0, 2)
    assert np.array_equal(p, part)
    # a stale move (vertex not in its expected block) is dropped
    g, applied, nv = oracle.apply_moves(H, p, 3, L, np.array([[3, 0, 1], [2, 0, 1]], np.int32))
    # 2 -> block 1: net {2,4,6} goes from blocks {0,1,2} to {1,2}: gain w = 3
    assert nv == 1 and applied == 1 and g == 3
    assert p[2] == 1
    # balance: block 1 already has 4 vertices, one more exceeds L = 4
    g, applied, nv = oracle.apply_moves(H, p, 3, L, np.array([[0, 0, 1]], np.int32))
    assert applied == 0 and p[0] == 0


def test_pair_gain_equals_connectivity_change():
    """Delta_exp of a pair is exactly the change of (lambda - 1) when its moves
    are applied alone: the pair network keeps every net whose cut status
    between the two blocks can change (Sections 5 and 6)."""
    checked = 0
    for seed in (1, 2, 3):
        inst = synth.instance("ring_n8M_zipf_k64", seed, n=16000, m=24000)
        H, part = inst["H"], inst["part"]
        c0 = oracle.connectivity(H, part, 64)
        qn, _ = oracle.quotient(H, part, 64)
        pairs = [(i, j) for i in range(64) for j in range(i + 1, 64) if qn[i, j] > 0][:12]
        L = oracle.max_block_weight(int(H.node_w.sum()), 64, 3)
        for i, j in pairs:
            r = oracle.refine_block_pair(H, part, 64, i, j)
            if r.status != oracle.OK or len(r.moves) == 0:
                continue
            p = part.copy()
            p[r.moves[:, 0]] = r.moves[:, 2]
            assert c0 - oracle.connectivity(H, p, 64) == r.delta_exp
            w = np.bincount(p, weights=H.node_w.astype(np.float64), minlength=64)
            assert w[i] <= L and w[j] <= L
            checked += 1
    assert checked >= 10


def test_round_gain_bookkeeping():
    inst = synth.instance("ring_n8M_zipf_k64", 4, n=16000, m=24000)
    H, part = inst["H"], inst["part"]
    c0 = oracle.connectivity(H, part, 64)
    newp, total, res, gains = oracle.refine_round(H, part, 64)
    assert total > 0
    assert oracle.connectivity(H, newp, 64) == c0 - total
    assert all(g >= 0 for g, _, _ in gains.values())
    L = oracle.max_block_weight(int(H.node_w.sum()), 64, 3)
    w0 = np.bincount(part, weights=H.node_w.astype(np.float64), minlength=64)
    w1 = np.bincount(newp, weights=H.node_w.astype(np.float64), minlength=64)
    assert np.all(w1 <= np.maximum(w0, L))       # no block grew beyond the bound
