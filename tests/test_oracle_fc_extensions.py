"""The oracle's FlowCutter extensions of Section 7 pinned against brute force
and a hand-worked case (CPU only).

Bulk piercing ("Bulk Piercing"): replayed step by step on small networks
with unit vertex weights.  The replay recomputes, without any flow
algorithm, the minimum cut and the minimal sides of every step (the
min-cut lattice, as in test_oracle_fc_replay), and re-derives from the
definitions of the reading (per-side geometric goal with carried
remainder, average growth per pierced node, warm-up, far from balance)
how many nodes each iteration must pierce; every pierced node must be a
legal candidate, a single path-free one whenever one exists.

Most balanced cut ("Most Balanced Cut"): the result is balanced, its cut
equals the flow (it is a minimum cut), it is at least as balanced as the
core algorithm's first balanced bipartition, and the flow is the core's;
plus the hand-worked case in tests/golden/most_balanced.json.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import hypergraph_from_lists, load_golden, random_instance
from tests.test_oracle_fc_replay import Enumerated, _candidates


def _replay_bulk(net, L, r, beta, warmup):
    E = Enumerated(net)
    W = int(E.w.sum())
    S = np.zeros(net.n_nodes, bool)
    T = np.zeros(net.n_nodes, bool)
    S[0] = True
    T[1] = True
    w = E.w
    base = [beta * (W - 2 * int(w[0])) // 200, beta * (W - 2 * int(w[1])) // 200]
    carry, added_w, added_n, grown = [0, 0], [0, 0], [0, 0], [0, 0]
    pending = [None, None]
    k_used = 0
    steps = 0
    bulk_steps = 0
    while True:
        steps += 1
        lam, Sr, Tr = E.sides(S, T)
        wS, wT = int(w[Sr].sum()), int(w[Tr].sum())
        for x in (0, 1):
            if pending[x] is not None:
                grew = (wS if x == 0 else wT) - pending[x]
                goal = base[x] + carry[x]
                added_w[x] += grew
                carry[x] = max(goal - grew, 0)
                base[x] = base[x] * beta // 100
                grown[x] += 1
                pending[x] = None
        balS = wS <= L and W - wS <= L
        balT = wT <= L and W - wT <= L
        if balS or balT:
            assert r.status == oracle.OK and k_used == len(r.pierce_node)
            assert r.flow == lam and r.iterations == steps
            return "balanced", bulk_steps
        grow_s = wS <= wT
        x = 0 if grow_s else 1
        R, O, Ro = (Sr, T, Tr) if grow_s else (Tr, S, Sr)
        wR = wS if grow_s else wT
        cand = _candidates(net, R, O, wR, L)
        if not cand.any():
            assert r.status == oracle.NO_BALANCED_CUT and k_used == len(r.pierce_node)
            return "none", bulk_steps
        path_free = (cand & ~Ro).any()
        k = 1
        goal = base[x] + carry[x]
        if not path_free and 2 * (wR + goal) <= W and grown[x] >= warmup and added_n[x] > 0:
            avg = max(added_w[x] // added_n[x], 1)
            k = max(-(-goal // avg), 1)
        # unit weights: the iteration takes min(k, candidates, room below L) nodes
        take = int(min(k, cand.sum(), L - wR))
        got = r.pierce_node[k_used:k_used + take]
        assert len(got) == take, "the oracle pierced fewer nodes than the rule asks"
        assert (r.pierce_side[k_used:k_used + take] == x).all()
        assert len(set(got.tolist())) == take
        for p in got:
            assert cand[p], "pierced node is not a candidate"
        if path_free:
            assert take == 1 and not Ro[got[0]], "a path-free candidate existed"
        bulk_steps += take > 1
        k_used += take
        X = (Sr if grow_s else Tr).copy()
        X[got] = True
        if grow_s:
            S = X
        else:
            T = X
        pending[x] = wR
        added_n[x] += take


@pytest.mark.parametrize("beta,warmup", [(55, 1), (55, 2), (70, 1)])
def test_bulk_piercing_replayed_by_brute_force(beta, warmup):
    rng = np.random.default_rng(1000 + beta + warmup)
    outcomes = {"balanced": 0, "none": 0}
    bulk = 0
    for _ in range(800):
        n = int(rng.integers(10, 17))
        H, side, region = random_instance(rng, n, int(rng.integers(10, 30)), max_size=5,
                                          region_frac=0.9, w_max=4, c_max=1)
        net = oracle.build_network(H, side, region)
        if net.n_nodes - 2 > 14 or net.m_nets == 0:
            continue
        W = int(net.node_w.sum())
        L = oracle.max_block_weight(W, 2, int(rng.choice([3, 10])))
        dist = oracle.dist_from_cut(H, side, region)
        orig, d, gid = oracle.node_arrays(net, side, region, dist)
        r = oracle.flowcutter(net, L, orig, d, gid, seed=int(rng.integers(0, 1 << 31)),
                              bulk_beta_pct=beta, bulk_warmup=warmup)
        how, b = _replay_bulk(net, L, r, beta, warmup)
        outcomes[how] += 1
        bulk += b
        assert r.bulk_steps == b
    assert outcomes["balanced"] > 100
    assert bulk > 20, "the sample rarely pierced in bulk"


def test_bulk_piercing_off_is_the_core_algorithm():
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(6, 30))
        H, side, region = random_instance(rng, n, int(rng.integers(4, 40)), max_size=5,
                                          region_frac=0.8, w_max=5, c_max=3)
        net = oracle.build_network(H, side, region)
        if net.m_nets == 0:
            continue
        L = oracle.max_block_weight(int(net.node_w.sum()), 2, 3)
        dist = oracle.dist_from_cut(H, side, region)
        orig, d, gid = oracle.node_arrays(net, side, region, dist)
        a = oracle.flowcutter(net, L, orig, d, gid, seed=9)
        b = oracle.flowcutter(net, L, orig, d, gid, seed=9, bulk_beta_pct=55, bulk_warmup=10**6)
        assert (a.status, a.flow, a.iterations) == (b.status, b.flow, b.iterations)
        assert np.array_equal(a.pierce_node, b.pierce_node)
        assert np.array_equal(a.final_side, b.final_side)


def test_most_balanced_hand_case():
    c = load_golden("most_balanced.json")
    H = hypergraph_from_lists(6, c["nets"], c["net_w"], c["node_w"])
    side = np.array(c["side"], np.int32)
    region = np.array(c["region"], np.int32)
    net = oracle.build_network(H, side, region)
    orig, d, gid = oracle.node_arrays(net, side, region, np.array(c["dist"], np.int32))
    r0 = oracle.flowcutter(net, c["max_block_weight"], orig, d, gid, seed=c["seed"])
    e0 = c["expected_core"]
    assert (r0.final_side.tolist(), r0.flow, r0.source_weight, r0.result_side) == \
        (e0["final_side"], e0["flow"], e0["source_weight"], e0["result_side"])
    e = c["expected"]
    r = oracle.flowcutter(net, c["max_block_weight"], orig, d, gid, seed=c["seed"],
                          mb_reps=e["mb_reps"])
    assert (r.final_side.tolist(), r.flow, r.source_weight, r.result_side, r.mb_steps) == \
        (e["final_side"], e["flow"], e["source_weight"], e["result_side"], e["mb_steps"])
    # the two path-free piercings: y2 (hypernode 4) into S, then y1 (3) into T
    assert r.pierce_side.tolist() == [2, 3] and r.pierce_node.tolist() == [4, 3]


def _replay_most_balanced(net, L, a, b, reps):
    """The path-free piercings after the core run: from the first balanced
    terminal sets, each recorded node must be a path-free candidate of the
    lighter reachable side, and a repetition ends exactly when none exists."""
    E = Enumerated(net)
    W = int(E.w.sum())
    # terminal sets of the first balanced state, rebuilt from the core record
    S = np.zeros(net.n_nodes, bool)
    T = np.zeros(net.n_nodes, bool)
    S[0] = True
    T[1] = True
    for side, p in zip(a.pierce_side, a.pierce_node):
        _, Sr, Tr = E.sides(S, T)
        if side == 0:
            S = Sr.copy()
            S[p] = True
        else:
            T = Tr.copy()
            T[p] = True
    S0, T0 = S.copy(), T.copy()
    rec = list(zip(b.pierce_side[len(a.pierce_node):].tolist(),
                   b.pierce_node[len(a.pierce_node):].tolist()))
    k = 0
    for _ in range(reps):
        S, T = S0.copy(), T0.copy()
        while True:
            lam, Sr, Tr = E.sides(S, T)
            assert lam == a.flow, "a path-free piercing changed the flow"
            wS, wT = int(E.w[Sr].sum()), int(E.w[Tr].sum())
            grow_s = wS <= wT
            R, O, Ro = (Sr, T, Tr) if grow_s else (Tr, S, Sr)
            cand = _candidates(net, R, O, wS if grow_s else wT, L) & ~Ro
            if not cand.any():
                break
            assert k < len(rec), "stopped although a path-free candidate exists"
            side, p = rec[k]
            k += 1
            assert side == (2 if grow_s else 3) and cand[p]
            X = (Sr if grow_s else Tr).copy()
            X[p] = True
            if grow_s:
                S = X
            else:
                T = X
    assert k == len(rec)
    return k


def test_most_balanced_is_a_more_balanced_minimum_cut():
    rng = np.random.default_rng(77)
    improved = steps = 0
    for _ in range(400):
        n = int(rng.integers(6, 15))
        H, side, region = random_instance(rng, n, int(rng.integers(4, 22)), max_size=4,
                                          region_frac=0.8, w_max=5, c_max=4)
        net = oracle.build_network(H, side, region)
        if net.n_nodes - 2 > 12 or net.m_nets == 0:
            continue
        W = int(net.node_w.sum())
        L = oracle.max_block_weight(W, 2, int(rng.choice([3, 10, 25])))
        dist = oracle.dist_from_cut(H, side, region)
        orig, d, gid = oracle.node_arrays(net, side, region, dist)
        seed = int(rng.integers(0, 1 << 31))
        a = oracle.flowcutter(net, L, orig, d, gid, seed=seed)
        b = oracle.flowcutter(net, L, orig, d, gid, seed=seed, mb_reps=3)
        assert b.status == a.status and b.flow == a.flow
        if a.status != oracle.OK:
            continue
        side_h = b.final_side.astype(bool)           # True: block 1
        w0 = int(net.node_w[~side_h].sum())
        assert w0 == b.source_weight
        assert w0 <= L and W - w0 <= L, "not balanced"
        assert oracle.cut_weight(net, ~side_h) == b.flow, "not a minimum cut"
        assert max(w0, W - w0) <= max(a.source_weight, W - a.source_weight)
        improved += max(w0, W - w0) < max(a.source_weight, W - a.source_weight)
        steps += _replay_most_balanced(net, L, a, b, 3)
    assert improved > 5 and steps > 50
