"""FlowCutter (Algorithm 2, Section 7) replayed against brute force.

For small networks every bipartition of the region is enumerated.  Starting
from S = {s}, T = {t}, each step recomputes, without any flow algorithm:
the minimum cut between the current terminal sets, the minimal source side
S_r (the intersection of all minimising source sets) and the minimal sink
side T_r (the complement of their union), as the min-cut lattice fixes them
(Picard-Queyranne).  The oracle's recorded piercing sequence is then checked
step by step against the rules of Algorithm 2 and Section 7 "Piercing":

* it stops exactly when (S_r, V \\ S_r) or (V \\ T_r, T_r) is balanced, with
  that bipartition and a flow equal to the brute-force minimum cut;
* otherwise it grows the lighter side (S iff c(S_r) <= c(T_r));
* the pierced node is a pin of a net touching the growing side's reachable
  set, outside both terminal sides' reachable sets, keeps the growing side
  within L, and avoids an augmenting path (lies outside the other side's
  reachable set) whenever any candidate does;
* it reports no balanced cut exactly when no candidate exists;
* the new terminal set is the reachable set plus the pierced node.

The tie-breaking order among equally good candidates (distance from the
original cut, then a hash) is the oracle's reading and is not re-derived
here."""
import numpy as np

import oracle
from tests.helpers import random_instance


class Enumerated:
    """All bipartitions of a flow network's region (hypernode 0 = s on the
    source side, 1 = t on the sink side, region vertex i <-> bit i)."""

    def __init__(self, net):
        nh = net.n_nodes
        self.r = nh - 2
        self.masks = np.arange(1 << self.r, dtype=np.int64)
        cut = np.zeros(len(self.masks), np.int64)
        for e in range(net.m_nets):
            ps = net.pins[net.net_off[e]:net.net_off[e + 1]]
            bits = 0
            for p in ps:
                if p >= 2:
                    bits |= 1 << (int(p) - 2)
            has_s, has_t = bool((ps == 0).any()), bool((ps == 1).any())
            inside = has_s | ((self.masks & bits) != 0)
            outside = has_t | ((self.masks & bits) != bits)
            cut += np.where(inside & outside, int(net.net_w[e]), 0)
        self.cut = cut
        self.w = np.asarray(net.node_w, np.int64)

    def bits(self, nodes):
        b = 0
        for h in np.nonzero(nodes)[0]:
            if h >= 2:
                b |= 1 << (int(h) - 2)
        return b

    def sides(self, S, T):
        """Minimum cut, minimal source side and minimal sink side (boolean
        arrays over hypernodes) for terminal sets S (contains s), T (contains
        t)."""
        sb, tb = self.bits(S), self.bits(T)
        ok = ((self.masks & sb) == sb) & ((self.masks & tb) == 0)
        lam = int(self.cut[ok].min())
        mins = self.masks[ok & (self.cut == lam)]
        and_m = int(np.bitwise_and.reduce(mins))
        or_m = int(np.bitwise_or.reduce(mins))
        nh = self.r + 2
        Sr = np.zeros(nh, bool)
        Tr = np.zeros(nh, bool)
        Sr[0] = True
        Tr[1] = True
        for i in range(self.r):
            Sr[i + 2] = bool(and_m >> i & 1)
            Tr[i + 2] = not (or_m >> i & 1)
        return lam, Sr, Tr


def _candidates(net, R, O, wR, L):
    """Pins of nets with a pin in R, outside R and O, that keep R within L."""
    cand = np.zeros(net.n_nodes, bool)
    for e in range(net.m_nets):
        ps = net.pins[net.net_off[e]:net.net_off[e + 1]]
        if R[ps].any():
            cand[ps] = True
    cand &= ~R & ~O
    cand &= wR + np.asarray(net.node_w, np.int64) <= L
    return cand


def _replay(net, L, r):
    E = Enumerated(net)
    W = int(E.w.sum())
    S = np.zeros(net.n_nodes, bool)
    T = np.zeros(net.n_nodes, bool)
    S[0] = True
    T[1] = True
    k = 0
    steps = 0
    while True:
        steps += 1
        lam, Sr, Tr = E.sides(S, T)
        wS, wT = int(E.w[Sr].sum()), int(E.w[Tr].sum())
        balS = wS <= L and W - wS <= L
        balT = wT <= L and W - wT <= L
        if balS or balT:
            assert r.status == oracle.OK and k == len(r.pierce_node)
            assert r.flow == lam and r.iterations == steps
            if balS and balT:
                use_t = max(wT, W - wT) < max(wS, W - wS)
            else:
                use_t = not balS
            want = Tr.astype(np.uint8) if use_t else (~Sr).astype(np.uint8)
            assert r.result_side == int(use_t)
            assert np.array_equal(r.final_side, want)
            return "balanced"
        grow_s = wS <= wT
        R, O, Ro = (Sr, T, Tr) if grow_s else (Tr, S, Sr)
        cand = _candidates(net, R, O, wS if grow_s else wT, L)
        if not cand.any():
            assert r.status == oracle.NO_BALANCED_CUT and k == len(r.pierce_node)
            return "none"
        assert k < len(r.pierce_node), "the oracle stopped early"
        p = int(r.pierce_node[k])
        assert int(r.pierce_side[k]) == (0 if grow_s else 1)
        assert cand[p], "pierced node is not a candidate"
        if (cand & ~Ro).any():
            assert not Ro[p], "an augmenting path was taken although a path-free candidate exists"
        k += 1
        if grow_s:
            S = Sr.copy()
            S[p] = True
        else:
            T = Tr.copy()
            T[p] = True


def test_flowcutter_replayed_by_brute_force():
    rng = np.random.default_rng(2201)
    outcomes = {"balanced": 0, "none": 0}
    pierced = 0
    multi = 0
    for _ in range(600):
        n = int(rng.integers(6, 15))
        H, side, region = random_instance(rng, n, int(rng.integers(4, 22)), max_size=4,
                                          region_frac=0.8, w_max=5, c_max=4)
        net = oracle.build_network(H, side, region)
        if net.n_nodes - 2 > 12 or net.m_nets == 0:
            continue
        W = int(net.node_w.sum())
        # the loop is the same for any bound; looser ones reach balance more often
        L = oracle.max_block_weight(W, 2, int(rng.choice([3, 10, 25])))
        dist = oracle.dist_from_cut(H, side, region)
        orig, d, gid = oracle.node_arrays(net, side, region, dist)
        r = oracle.flowcutter(net, L, orig, d, gid, seed=int(rng.integers(0, 1 << 31)))
        outcomes[_replay(net, L, r)] += 1
        pierced += len(r.pierce_node)
        multi += len(r.pierce_node) > 1
    # the sample exercises both endings and multi-step piercing sequences
    assert outcomes["balanced"] > 200 and outcomes["none"] > 100
    assert pierced > 800 and multi > 150


def test_replay_detects_a_wrong_piercing():
    """The replay is strict: the oracle's own piercing sequence with every
    side flipped is rejected."""
    rng = np.random.default_rng(7)
    rejected = 0
    for _ in range(300):
        n = int(rng.integers(8, 15))
        H, side, region = random_instance(rng, n, int(rng.integers(6, 22)), max_size=4,
                                          region_frac=0.8, w_max=5, c_max=4)
        net = oracle.build_network(H, side, region)
        if net.n_nodes - 2 > 12 or net.m_nets == 0:
            continue
        L = oracle.max_block_weight(int(net.node_w.sum()), 2, 3)
        dist = oracle.dist_from_cut(H, side, region)
        orig, d, gid = oracle.node_arrays(net, side, region, dist)
        r = oracle.flowcutter(net, L, orig, d, gid, seed=3)
        if len(r.pierce_node) == 0:
            continue
        bad = oracle.FlowCutterResult(r.status, r.flow, r.iterations, r.final_side,
                                      1 - r.pierce_side, r.pierce_node, r.result_side,
                                      r.source_weight)
        try:
            _replay(net, L, bad)
        except AssertionError:
            rejected += 1
        else:
            raise AssertionError("a flipped piercing side was accepted")
    assert rejected > 20
