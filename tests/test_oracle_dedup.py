"""The oracle's identical net removal (Section 6, "Identical Net Removal")
pinned against a hand-worked case and against what merging must preserve
(CPU only): every cut of the flow hypergraph keeps its weight (brute force
over all bipartitions of small regions), so the maximum flow, the minimal
cut sides over the hypernodes and FlowCutter's outcome are unchanged; no two
kept nets have the same pin set; weights are conserved."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import hypergraph_from_lists, load_golden, random_instance


def _nets(net):
    return [net.pins[net.net_off[e]:net.net_off[e + 1]].tolist() for e in range(net.m_nets)]


def test_hand_case():
    g = load_golden("identical_nets.json")
    side = np.array(g["side"], np.int32)
    region = np.array(g["region"], np.int32)
    H = hypergraph_from_lists(g["n"], g["nets"], g["net_w"])
    d = oracle.dedup_network(oracle.build_network(H, side, region))
    assert _nets(d) == g["expected_nets"]
    assert d.net_w.tolist() == g["expected_net_w"]
    assert d.net_gid.tolist() == g["expected_net_gid"]
    c = g["collision"]
    H = hypergraph_from_lists(g["n"], c["nets"], c["net_w"])
    d = oracle.dedup_network(oracle.build_network(H, side, region))
    assert _nets(d) == c["expected_nets"]
    assert d.net_w.tolist() == c["expected_net_w"]
    assert d.net_gid.tolist() == c["expected_net_gid"]


def _dup_instance(rng):
    """Random small instance with many nets that coincide after contraction."""
    n = int(rng.integers(6, 13))
    H, side, region = random_instance(rng, n, int(rng.integers(6, 30)), max_size=3,
                                      region_frac=0.6, w_max=5, c_max=3)
    return H, side, region


def test_every_cut_keeps_its_weight():
    rng = np.random.default_rng(31)
    merged = 0
    for _ in range(300):
        H, side, region = _dup_instance(rng)
        net = oracle.build_network(H, side, region)
        d = oracle.dedup_network(net)
        merged += net.m_nets - d.m_nets
        assert int(d.net_w.sum()) == int(net.net_w.sum())
        r = net.n_nodes - 2
        if r > 10:
            continue
        for mask in range(1 << r):
            src = np.zeros(net.n_nodes, bool)
            src[0] = True
            for i in range(r):
                src[2 + i] = bool(mask >> i & 1)
            assert oracle.cut_weight(d, src) == oracle.cut_weight(net, src)
    assert merged > 100


def test_kept_nets_are_distinct_sets():
    rng = np.random.default_rng(32)
    for _ in range(200):
        H, side, region = _dup_instance(rng)
        d = oracle.dedup_network(oracle.build_network(H, side, region))
        sets = [frozenset(x) for x in _nets(d)]
        assert len(set(sets)) == len(sets), "identical nets kept"


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_flow_cuts_and_flowcutter_unchanged(seed):
    inst = synth.instance("ring_n500k_zipf_fc", seed, n=20000, m=30000, radius=2000)
    H, side, region = inst["H"], inst["part"], inst["region"]
    net = oracle.build_network(H, side, region)
    d = oracle.dedup_network(net)
    assert d.m_nets < net.m_nets
    a = oracle.max_flow_min_cut(net)
    b = oracle.max_flow_min_cut(d)
    nh = net.n_nodes
    assert a.flow == b.flow
    assert np.array_equal(a.source_side[:nh], b.source_side[:nh])
    assert np.array_equal(a.sink_side[:nh], b.sink_side[:nh])
    L = oracle.max_block_weight(int(net.node_w.sum()), 2, 3)
    dist = oracle.dist_from_cut(H, side, region)
    orig, dd, gid = oracle.node_arrays(net, side, region, dist)
    fa = oracle.flowcutter(net, L, orig, dd, gid, seed=seed)
    fb = oracle.flowcutter(d, L, orig, dd, gid, seed=seed)
    assert (fa.status, fa.flow, fa.iterations) == (fb.status, fb.flow, fb.iterations)
    assert np.array_equal(fa.pierce_node, fb.pierce_node)
    assert np.array_equal(fa.final_side, fb.final_side)
