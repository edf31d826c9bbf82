"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks the oracle against a value or property that the paper or
the mathematics fixes: hand-worked fixtures (tests/golden), brute force over
all cuts, independent library routines on a differently built model (scipy's
maximum_flow on a Lawler graph assembled here, networkx's minimum_cut on the
plain graph of 2-pin nets), feasibility of the flow, and invariants of the
construction and of Algorithm 2.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import hypergraph_from_lists, load_golden, random_instance


def _lawler_names(net, mask):
    nh, m = net.n_nodes, net.m_nets
    out = set()
    for x in np.nonzero(mask)[0]:
        x = int(x)
        if x < nh:
            out.add(f"h{x}")
        elif x < nh + m:
            out.add(f"in{x - nh}")
        else:
            out.add(f"out{x - nh - m}")
    return out


def _fixture():
    g = load_golden("lawler_hand_example.json")
    h = g["hypergraph"]
    H = hypergraph_from_lists(h["n"], h["nets"], h["net_w"], h["node_w"])
    return g, H, np.array(g["side"], np.int32), np.array(g["region"], np.int32)


def test_hand_fixture_network():
    g, H, side, region = _fixture()
    net = oracle.build_network(H, side, region)
    ex = g["expected_network"]
    assert net.n_nodes == ex["n_nodes"]
    got = [net.pins[net.net_off[e]:net.net_off[e + 1]].tolist() for e in range(net.m_nets)]
    assert got == ex["nets"]
    assert net.net_w.tolist() == ex["net_w"]
    assert net.net_gid.tolist() == ex["net_gid"]
    assert net.node_w.tolist() == ex["node_w"]


@pytest.mark.parametrize("algo", ["dinic", "ek"])
def test_hand_fixture_flow_and_cuts(algo):
    g, H, side, region = _fixture()
    net = oracle.build_network(H, side, region)
    mc = oracle.max_flow_min_cut(net, algo)
    assert mc.flow == g["expected_flow"]
    assert _lawler_names(net, mc.source_side) == set(g["expected_source_side_lawler"])
    assert _lawler_names(net, mc.sink_side) == set(g["expected_sink_side_lawler"])
    hs = np.nonzero(mc.source_side[: net.n_nodes])[0].tolist()
    assert hs == g["expected_source_side_hypernodes"]


def test_hand_fixture_dist():
    g, H, side, region = _fixture()
    assert oracle.dist_from_cut(H, side, region).tolist() == g["expected_dist_from_cut"]


def test_hand_fixture_flowcutter():
    g, H, side, region = _fixture()
    fc = g["flowcutter"]
    net = oracle.build_network(H, side, region)
    dist = oracle.dist_from_cut(H, side, region)
    orig, d, gid = oracle.node_arrays(net, side, region, dist)
    r = oracle.flowcutter(net, fc["max_block_weight"], orig, d, gid, seed=0)
    assert r.status == oracle.OK
    assert r.pierce_side.tolist() == fc["expected_pierce_side"]
    assert r.pierce_node.tolist() == fc["expected_pierce_node"]
    assert r.final_side.tolist() == fc["expected_final_side"]
    assert r.flow == fc["expected_cut"]
    assert r.iterations == fc["expected_iterations"]


def test_max_block_weight():
    # Section 2: L_max = (1 + eps) * ceil(c(V) / k); eps = 0.03
    assert oracle.max_block_weight(4096, 2, 3) == 2109       # 1.03 * 2048 = 2109.44
    assert oracle.max_block_weight(6, 2, 3) == 3
    assert oracle.max_block_weight(101, 2, 3) == 52           # ceil = 51, 1.03 * 51 = 52.53
    assert oracle.max_block_weight(8_000_000, 64, 3) == 128750


def _random_nets(seed, count, n_lo=4, n_hi=14, m_hi=18, c_max=1):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        m = int(rng.integers(1, m_hi + 1))
        H, side, region = random_instance(rng, n, m, max_size=4, region_frac=0.7, w_max=6,
                                          c_max=c_max)
        yield H, side, region, oracle.build_network(H, side, region)


def test_bruteforce_agreement():
    """Max-flow = min-cut (Section 2) and the minimal cut sides: S_r is the
    intersection of all minimum source sets, T_r's complement their union."""
    checked = 0
    for H, side, region, net in _random_nets(11, 250):
        if net.n_nodes - 2 > 14:
            continue
        mc = oracle.max_flow_min_cut(net)
        bf = oracle.bruteforce(net)
        assert mc.flow == bf["min_cut"]
        r = net.n_nodes - 2
        s_mask = sum(1 << i for i in range(r) if mc.source_side[2 + i])
        not_t_mask = sum(1 << i for i in range(r) if not mc.sink_side[2 + i])
        assert s_mask == bf["and_mask"]
        assert not_t_mask == bf["or_mask"]
        assert mc.source_side[0] == 1 and mc.sink_side[0] == 0
        assert mc.sink_side[1] == 1 and mc.source_side[1] == 0
        checked += 1
    assert checked > 150


def _scipy_lawler_value(net):
    """Maximum flow of the Lawler expansion with scipy (an independent
    implementation, on a graph assembled here from the definition)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_flow
    nh, m = net.n_nodes, net.m_nets
    N = nh + 2 * m
    inf = int(net.net_w.sum()) + 1
    rows, cols, caps = [], [], []
    for e in range(m):
        ein, eout = nh + e, nh + m + e
        for u in net.pins[net.net_off[e]:net.net_off[e + 1]]:
            rows += [int(u), eout]
            cols += [ein, int(u)]
            caps += [inf, inf]
        rows.append(ein); cols.append(eout); caps.append(int(net.net_w[e]))
    A = csr_matrix((np.array(caps, np.int32), (rows, cols)), shape=(N, N))
    return maximum_flow(A, 0, 1).flow_value


def test_scipy_maxflow_agreement():
    for H, side, region, net in _random_nets(5, 120, n_hi=40, m_hi=60):
        assert oracle.max_flow_min_cut(net).flow == _scipy_lawler_value(net)


def test_scipy_ring4096():
    I = synth.instance("ring_n4096_geom", 3)
    net = oracle.build_network(I["H"], I["part"], I["region"])
    assert oracle.max_flow_min_cut(net).flow == _scipy_lawler_value(net)


def test_dinic_vs_edmonds_karp():
    """Two independent textbook routines reach the same (unique) value and
    cut sides; 4096-vertex ring instances and random ones."""
    nets = [oracle.build_network(I["H"], I["part"], I["region"])
            for I in (synth.instance("ring_n4096_geom", s) for s in (1, 2))]
    nets += [n for *_, n in _random_nets(3, 40, n_hi=60, m_hi=90)]
    for net in nets:
        a = oracle.max_flow_min_cut(net, "dinic")
        b = oracle.max_flow_min_cut(net, "ek")
        assert a.flow == b.flow
        assert np.array_equal(a.source_side, b.source_side)
        assert np.array_equal(a.sink_side, b.sink_side)


def test_flow_feasibility_and_cut_capacity():
    """Capacity, skew symmetry and conservation (Section 2), and the cut
    between S_r and the rest carrying exactly the flow value."""
    for H, side, region, net in _random_nets(9, 60, n_hi=50, m_hi=80):
        mc = oracle.max_flow_min_cut(net)
        tail, head, cap, flow = mc.lawler.arcs()
        assert np.all(flow <= cap)
        # reverse arcs come in pairs: total flow over all arcs cancels
        N = mc.lawler.N
        net_out = np.zeros(N, np.int64)
        np.add.at(net_out, tail, flow)
        assert np.all(net_out[2:] == 0)          # conservation except at s and t
        assert net_out[0] == mc.flow and net_out[1] == -mc.flow
        S = mc.source_side.astype(bool)
        crossing = S[tail] & ~S[head]
        assert int(cap[crossing].sum()) == mc.flow
        assert int(flow[crossing].sum()) == mc.flow


def test_two_pin_nets_graph_mincut():
    """With only 2-pin nets the hypergraph is a graph; its minimum s-t cut by
    networkx equals the Lawler max flow."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(21)
    for _ in range(40):
        n = int(rng.integers(6, 30))
        m = int(rng.integers(5, 60))
        nets = [sorted(rng.choice(n, 2, replace=False).tolist()) for _ in range(m)]
        w = rng.integers(1, 9, m)
        H = hypergraph_from_lists(n, nets, w)
        side = rng.integers(0, 2, n).astype(np.int32)
        region = np.sort(rng.choice(n, n // 2, replace=False)).astype(np.int32)
        net = oracle.build_network(H, side, region)
        G = nx.DiGraph()
        G.add_nodes_from(range(net.n_nodes))
        for e in range(net.m_nets):
            a, b = net.pins[net.net_off[e]:net.net_off[e + 1]]
            for x, y in ((a, b), (b, a)):
                c = G[x][y]["capacity"] if G.has_edge(x, y) else 0
                G.add_edge(int(x), int(y), capacity=c + int(net.net_w[e]))
        val = nx.minimum_cut_value(G, 0, 1) if net.m_nets else 0
        assert oracle.max_flow_min_cut(net).flow == val


def test_path_lightest_net():
    """A path s - v1 - ... - vk - t of 2-pin nets: the flow is its lightest net."""
    w = [7, 3, 9, 4, 6]
    nets = [[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]]
    H = hypergraph_from_lists(6, nets, w)
    side = np.array([0, 0, 0, 1, 1, 1], np.int32)
    net = oracle.build_network(H, side, np.array([1, 2, 3, 4], np.int32))
    mc = oracle.max_flow_min_cut(net)
    assert mc.flow == 3
    # minimal source side: s and v1 only (the lightest net is the second)
    assert np.nonzero(mc.source_side[: net.n_nodes])[0].tolist() == [0, 2]


def test_net_with_s_and_t_is_dropped():
    """Section 6: a net holding both s and t can never leave the cut and is
    discarded, so the flow through the region is 0."""
    H = hypergraph_from_lists(4, [[0, 1, 3]], [5])
    side = np.array([0, 0, 1, 1], np.int32)
    net = oracle.build_network(H, side, np.array([1], np.int32))
    assert net.m_nets == 0
    assert oracle.max_flow_min_cut(net).flow == 0
    # single-pin remainder is discarded too
    H2 = hypergraph_from_lists(3, [[0, 1]], [5])
    net2 = oracle.build_network(H2, np.array([0, 0, 1], np.int32), np.array([1], np.int32))
    assert net2.m_nets == 1        # {v1, s}: two pins, kept
    net3 = oracle.build_network(H2, np.array([0, 0, 1], np.int32), np.array([2], np.int32))
    assert net3.m_nets == 0        # only s remains: discarded


def test_construction_preserves_cuts():
    """For every bipartition X of the region, the cut of the flow hypergraph
    plus the weight of the discarded s-t nets equals the cut of H under
    V_1 \\ B + X versus the rest (the contraction of Section 6)."""
    rng = np.random.default_rng(4)
    for H, side, region, net in _random_nets(13, 60, n_hi=30, m_hi=40):
        in_b = np.zeros(H.n, bool)
        in_b[region] = True
        st = 0
        for e in range(H.m):
            ps = H.pins[H.net_off[e]:H.net_off[e + 1]]
            outside = ps[~in_b[ps]]
            if (side[outside] == 0).any() and (side[outside] == 1).any():
                st += int(H.net_w[e])
        for _ in range(8):
            x = rng.integers(0, 2, len(region)).astype(bool)
            blk = side.copy()
            blk[region] = np.where(x, 0, 1)
            cut_h = 0
            for e in range(H.m):
                b = blk[H.pins[H.net_off[e]:H.net_off[e + 1]]]
                b = b[b >= 0]
                if (b == 0).any() and (b == 1).any():
                    cut_h += int(H.net_w[e])
            in_src = np.zeros(net.n_nodes, bool)
            in_src[0] = True
            in_src[2:] = x
            assert oracle.cut_weight(net, in_src) + st == cut_h


def test_dist_from_cut_bfs_properties():
    """Distance 1 exactly for region pins of cut nets; every larger distance
    has a region neighbour (sharing a net) one closer and none closer still."""
    rng = np.random.default_rng(8)
    for _ in range(40):
        n = int(rng.integers(10, 60))
        H, side, region = random_instance(rng, n, int(rng.integers(5, 60)), max_size=4,
                                          region_frac=0.6)
        dist = oracle.dist_from_cut(H, side, region)
        pos = {int(v): i for i, v in enumerate(region)}
        nbrs = {i: set() for i in range(len(region))}
        cutpin = set()
        for e in range(H.m):
            ps = H.pins[H.net_off[e]:H.net_off[e + 1]].tolist()
            sides = {int(side[v]) for v in ps}
            r = [pos[v] for v in ps if v in pos]
            if 0 in sides and 1 in sides:
                cutpin.update(r)
            for a in r:
                nbrs[a].update(r)
        for i in range(len(region)):
            d = int(dist[i])
            if i in cutpin:
                assert d == 1
            elif d == oracle.DIST_FAR:
                assert all(dist[j] == oracle.DIST_FAR for j in nbrs[i] if j not in cutpin) \
                    and not (nbrs[i] & cutpin)
            else:
                assert d >= 2
                near = [int(dist[j]) for j in nbrs[i] if j != i]
                assert min(near) == d - 1


def _fmix32(h):
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def _unxorshift(h, s):
    x = h
    for _ in range(32 // s + 1):
        x = h ^ (x >> s)
    return x & 0xFFFFFFFF


def test_fmix32_is_a_bijection():
    """The third piercing key must never tie: fmix32 is invertible (each step
    is), checked by undoing it on a sample."""
    inv1 = pow(0x85EBCA6B, -1, 1 << 32)
    inv2 = pow(0xC2B2AE35, -1, 1 << 32)
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 1 << 32, 2000, dtype=np.uint64).tolist() + [0, 1, 0xFFFFFFFF]:
        h = _fmix32(x)
        y = _unxorshift(h, 16)
        y = (y * inv2) & 0xFFFFFFFF
        y = _unxorshift(y, 13)
        y = (y * inv1) & 0xFFFFFFFF
        y = _unxorshift(y, 16)
        assert y == x


def test_flowcutter_invariants():
    """Algorithm 2: the result is balanced, its cut equals the final flow, the
    flow is at least the best balanced cut (brute force), and augmenting the
    previous flow gives exactly what recomputing from scratch gives."""
    rng = np.random.default_rng(17)
    done = pierced = 0
    for _ in range(400):
        n = int(rng.integers(6, 16))
        H, side, region = random_instance(rng, n, int(rng.integers(4, 24)), max_size=4,
                                          region_frac=0.8, w_max=5, c_max=4)
        net = oracle.build_network(H, side, region)
        if net.n_nodes - 2 > 14:
            continue
        W = int(net.node_w.sum())
        L = oracle.max_block_weight(W, 2, 3)
        dist = oracle.dist_from_cut(H, side, region)
        orig, d, gid = oracle.node_arrays(net, side, region, dist)
        seed = int(rng.integers(0, 1 << 31))
        r = oracle.flowcutter(net, L, orig, d, gid, seed=seed)
        r2 = oracle.flowcutter(net, L, orig, d, gid, seed=seed, recompute=True)
        assert r.status == r2.status
        assert np.array_equal(r.pierce_node, r2.pierce_node)
        assert np.array_equal(r.pierce_side, r2.pierce_side)
        if r.status != oracle.OK:
            assert r.status == oracle.NO_BALANCED_CUT
            continue
        assert np.array_equal(r.final_side, r2.final_side)
        fs = r.final_side
        assert fs[0] == 0 and fs[1] == 1
        w0 = int(net.node_w[fs == 0].sum())
        assert w0 <= L and W - w0 <= L
        assert oracle.cut_weight(net, fs == 0) == r.flow
        bf = oracle.bruteforce(net, L)
        assert bf["min_balanced"] >= 0 and r.flow >= bf["min_balanced"]
        assert r.flow >= bf["min_cut"]
        # every pierced node is a region vertex, pierced at most once
        assert len(set(r.pierce_node.tolist())) == len(r.pierce_node)
        assert np.all(r.pierce_node >= 2)
        done += 1
        pierced += len(r.pierce_node) > 0
    assert done > 120 and pierced > 30


def test_seqpr_matches_dinic_random():
    """The sequential FIFO push-relabel CPU baseline (SeqPR) reaches the
    same flow value and the same minimal cut sides as Dinic, which the other
    tests pin to brute force and scipy."""
    checked = 0
    for H, side, region, net in _random_nets(2024, 300, n_hi=40, m_hi=80, c_max=3):
        mc = oracle.max_flow_min_cut(net)
        r = oracle.seqpr(net)
        assert r.flow == mc.flow
        assert np.array_equal(r.source_side, mc.source_side)
        assert np.array_equal(r.sink_side, mc.sink_side)
        checked += 1
    assert checked == 300


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_seqpr_matches_dinic_ring4096(seed):
    inst = synth.instance("ring_n4096_geom", seed)
    net = oracle.build_network(inst["H"], inst["part"], inst["region"])
    mc = oracle.max_flow_min_cut(net)
    r = oracle.seqpr(net)
    assert r.flow == mc.flow
    assert np.array_equal(r.source_side, mc.source_side)
    assert np.array_equal(r.sink_side, mc.sink_side)
    assert r.global_relabels >= 1


def test_seqpr_scaled_zipf_ring():
    """A heavy-tailed ring (the 2M workload's generator at n = 20,000)."""
    inst = synth.instance("ring_n2M_zipf", 3, n=20000, m=30000, radius=2000)
    net = oracle.build_network(inst["H"], inst["part"], inst["region"])
    mc = oracle.max_flow_min_cut(net)
    r = oracle.seqpr(net)
    assert r.flow == mc.flow
    assert np.array_equal(r.source_side, mc.source_side)
    assert np.array_equal(r.sink_side, mc.sink_side)
