"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and index results must match bit for bit: network structure, flow
value, the minimal source side S_r and minimal sink side T_r over every
Lawler node, cut nets, side weights, the FlowCutter piercing sequence, final
bipartition and cut weight.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.flowcheck import check_preflow
from tests.helpers import hypergraph_from_lists, load_golden, random_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hfp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_01556_gb300 import hfp as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def ctx(hfp):
    c = hfp.ctx_create(0)
    yield c
    c.close()


def _gpu_net(hfp, ctx, H, side, region, dist=None):
    return hfp.build_flow_network(ctx, H.net_off, H.pins, H.net_w, H.node_w, region, side, H.n,
                                  dist_from_cut=dist)


def _expected_incidence(onet):
    off = np.zeros(onet.n_nodes + 1, np.int64)
    np.add.at(off, onet.pins.astype(np.int64) + 1, 1)
    off = np.cumsum(off)
    order = np.argsort(onet.pins, kind="stable")          # slots grouped by node, ascending
    return off.astype(np.uint32), order.astype(np.int32)


def _check_structure(hfp, gnet, onet, H, side, region):
    ex = hfp.net_export(gnet)
    assert gnet.info.n_nodes == onet.n_nodes
    assert gnet.info.m_nets == onet.m_nets
    assert gnet.info.p_pins == onet.p
    assert np.array_equal(ex["net_off"], onet.net_off)
    assert np.array_equal(ex["pins"], onet.pins)
    assert np.array_equal(ex["net_w"], onet.net_w)
    assert np.array_equal(ex["net_gid"], onet.net_gid)
    assert np.array_equal(ex["node_w"].astype(np.int64), onet.node_w)
    off, slots = _expected_incidence(onet)
    assert np.array_equal(ex["node_off"], off)
    assert np.array_equal(ex["inc_slot"], slots)
    d = oracle.dist_from_cut(H, side, region)
    assert np.array_equal(ex["dist"][2:], d)


def _check_feasible(hfp, gnet, flow):
    """The device's per-arc preflow: capacities (with the (u, e_in) cap),
    conservation and value (per-arc flows are not unique, so they are
    checked, not compared)."""
    ex = hfp.net_export(gnet)
    check_preflow(gnet.info.n_nodes, ex["net_off"], ex["pins"], ex["net_w"],
                  hfp.net_export_flow(gnet), flow)


def _check_flow(hfp, gnet, onet):
    mc = oracle.max_flow_min_cut(onet)
    flow = hfp.max_flow(gnet)
    assert flow == mc.flow
    _check_feasible(hfp, gnet, flow)
    law, reg, cuts, ws = hfp.min_cut_source_side(gnet)
    assert np.array_equal(law, mc.source_side)
    assert np.array_equal(reg, mc.source_side[2:onet.n_nodes])
    nh, m = onet.n_nodes, onet.m_nets
    S = mc.source_side
    exp_cuts = onet.net_gid[(S[nh:nh + m] == 1) & (S[nh + m:nh + 2 * m] == 0)]
    assert np.array_equal(cuts, exp_cuts)
    assert ws == int(onet.node_w[S[:nh] == 1].sum())
    tlaw, treg, wt = hfp.min_cut_sink_side(gnet)
    assert np.array_equal(tlaw, mc.sink_side)
    assert np.array_equal(treg, mc.sink_side[2:onet.n_nodes])
    assert wt == int(onet.node_w[mc.sink_side[:nh] == 1].sum())
    # the cut nets carry exactly the flow (max-flow = min-cut)
    assert int(onet.net_w[(S[nh:nh + m] == 1) & (S[nh + m:nh + 2 * m] == 0)].sum()) == flow
    return mc


def test_hand_fixture(hfp, ctx):
    g = load_golden("lawler_hand_example.json")
    h = g["hypergraph"]
    H = hypergraph_from_lists(h["n"], h["nets"], h["net_w"], h["node_w"])
    side = np.array(g["side"], np.int32)
    region = np.array(g["region"], np.int32)
    gnet = _gpu_net(hfp, ctx, H, side, region)
    onet = oracle.build_network(H, side, region)
    _check_structure(hfp, gnet, onet, H, side, region)
    assert hfp.max_flow(gnet) == g["expected_flow"]
    _check_flow(hfp, gnet, onet)
    fc = g["flowcutter"]
    r = hfp.flowcutter(gnet, hfp.fc_params(fc["max_block_weight"], seed=0))
    assert r.status == 0
    assert r.pierce_side.tolist() == fc["expected_pierce_side"]
    assert r.pierce_node.tolist() == fc["expected_pierce_node"]
    assert r.final_side.tolist() == fc["expected_final_side"][2:]
    assert r.flow == fc["expected_cut"]


@pytest.mark.parametrize("seed", list(range(1, 101)))
def test_ring4096_flow_and_cuts(hfp, ctx, seed):
    inst = synth.instance("ring_n4096_geom", seed)
    H, part, region = inst["H"], inst["part"], inst["region"]
    gnet = _gpu_net(hfp, ctx, H, part, region)
    onet = oracle.build_network(H, part, region)
    if seed <= 5:
        _check_structure(hfp, gnet, onet, H, part, region)
    _check_flow(hfp, gnet, onet)


def _random_cases(seed, count, n_lo=3, n_hi=60, m_hi=120, c_max=1, k_sides=2):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        m = int(rng.integers(1, m_hi + 1))
        H, side, region = random_instance(rng, n, m, max_size=int(rng.integers(2, 9)),
                                          region_frac=float(rng.uniform(0.05, 1.0)),
                                          w_max=int(rng.integers(1, 12)), c_max=c_max,
                                          k_sides=k_sides)
        yield H, side, region


def test_random_small_structure_and_flow(hfp, ctx):
    for H, side, region in _random_cases(101, 150):
        gnet = _gpu_net(hfp, ctx, H, side, region)
        onet = oracle.build_network(H, side, region)
        _check_structure(hfp, gnet, onet, H, side, region)
        _check_flow(hfp, gnet, onet)
        gnet.close()


def test_random_pair_sides_ignore_other_blocks(hfp, ctx):
    """Vertices of neither block (side -1) are dropped from nets (k-way pairs)."""
    for H, side, region in _random_cases(202, 60, k_sides=4):
        if len(region) == 0:
            continue
        gnet = _gpu_net(hfp, ctx, H, side, region)
        onet = oracle.build_network(H, side, region)
        _check_structure(hfp, gnet, onet, H, side, region)
        _check_flow(hfp, gnet, onet)
        gnet.close()


def test_edge_cases(hfp, ctx):
    # empty region: only s and t, no nets
    H = hypergraph_from_lists(4, [[0, 1], [2, 3], [1, 2]], [3, 4, 5])
    side = np.array([0, 0, 1, 1], np.int32)
    gnet = _gpu_net(hfp, ctx, H, side, np.zeros(0, np.int32))
    assert gnet.info.n_nodes == 2 and gnet.info.m_nets == 0
    assert hfp.max_flow(gnet) == 0
    law, reg, cuts, ws = hfp.min_cut_source_side(gnet)
    assert law.tolist() == [1, 0] and ws == 2
    # single region vertex between s and t
    gnet = _gpu_net(hfp, ctx, H, side, np.array([1], np.int32))
    onet = oracle.build_network(H, side, np.array([1], np.int32))
    _check_flow(hfp, gnet, onet)
    # every vertex in the region: s and t carry no weight and no pins
    region = np.arange(4, dtype=np.int32)
    gnet = _gpu_net(hfp, ctx, H, side, region)
    onet = oracle.build_network(H, side, region)
    _check_structure(hfp, gnet, onet, H, side, region)
    _check_flow(hfp, gnet, onet)
    # a heavy net (more than a warp of pins) on both sides of the cut
    n = 200
    nets = [list(range(0, 150)), list(range(100, 200)), [0, 199], [10, 190]]
    H = hypergraph_from_lists(n, nets, [7, 3, 2, 9])
    side = (np.arange(n) >= 100).astype(np.int32)
    region = np.arange(50, 150, dtype=np.int32)
    gnet = _gpu_net(hfp, ctx, H, side, region)
    onet = oracle.build_network(H, side, region)
    _check_structure(hfp, gnet, onet, H, side, region)
    _check_flow(hfp, gnet, onet)


def test_invalid_inputs(hfp, ctx):
    H = hypergraph_from_lists(4, [[0, 1], [2, 3], [1, 2]], [3, 4, 5])
    side = np.array([0, 0, 1, 1], np.int32)
    with pytest.raises(hfp.HfpError) as e:
        _gpu_net(hfp, ctx, H, side, np.array([1, 1], np.int32))      # repeated vertex
    assert e.value.status == hfp.ERR_INVALID
    with pytest.raises(hfp.HfpError):
        _gpu_net(hfp, ctx, H, np.array([0, -1, 1, 1], np.int32), np.array([1], np.int32))
    with pytest.raises(hfp.HfpError):
        _gpu_net(hfp, ctx, H, side, np.array([7], np.int32))         # out of range
    bad = hypergraph_from_lists(4, [[0, 9]], [3])
    with pytest.raises(hfp.HfpError):
        _gpu_net(hfp, ctx, bad, side, np.array([0], np.int32))       # pin out of range
    bad = hypergraph_from_lists(4, [[0, 1]], [0])
    with pytest.raises(hfp.HfpError):
        _gpu_net(hfp, ctx, bad, side, np.array([0], np.int32))       # weight 0
    gnet = _gpu_net(hfp, ctx, H, side, np.array([1, 2], np.int32))
    with pytest.raises(hfp.HfpError) as e:
        hfp.min_cut_source_side(gnet)                                # before max_flow
    assert e.value.status == hfp.ERR_STATE


def test_device_inputs_match_host_inputs(hfp, ctx):
    torch = pytest.importorskip("torch")
    inst = synth.instance("ring_n4096_geom", 7)
    H, part, region = inst["H"], inst["part"], inst["region"]
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    gnet = hfp.build_flow_network(ctx, dev(H.net_off.view(np.int32), np.int32),
                                  dev(H.pins, np.int32), dev(H.net_w, np.int32),
                                  dev(H.node_w, np.int32), dev(region, np.int32),
                                  dev(part, np.int32), H.n)
    torch.cuda.synchronize()
    onet = oracle.build_network(H, part, region)
    _check_structure(hfp, gnet, onet, H, part, region)
    _check_flow(hfp, gnet, onet)


def _fc_compare(hfp, ctx, H, side, region, eps_pct=3, seed=0, dist_given=False, **ext):
    onet = oracle.build_network(H, side, region)
    W = int(onet.node_w.sum())
    L = oracle.max_block_weight(W, 2, eps_pct)
    dist = oracle.dist_from_cut(H, side, region)
    orig, d, gid = oracle.node_arrays(onet, side, region, dist)
    o = oracle.flowcutter(onet, L, orig, d, gid, seed=seed, **ext)
    gnet = _gpu_net(hfp, ctx, H, side, region, dist=dist if dist_given else None)
    r = hfp.flowcutter(gnet, hfp.fc_params(L, seed=seed, **ext))
    assert r.status == o.status
    assert (r.bulk_steps, r.mb_steps) == (o.bulk_steps, o.mb_steps)
    if r.status in (oracle.OK, oracle.NO_BALANCED_CUT):
        _check_feasible(hfp, gnet, o.flow)
    assert np.array_equal(r.pierce_side, o.pierce_side)
    assert np.array_equal(r.pierce_node, o.pierce_node)
    if o.status == oracle.OK:
        assert r.flow == o.flow
        assert r.iterations == o.iterations
        assert r.result_side == o.result_side
        assert r.source_weight == o.source_weight
        assert np.array_equal(r.final_side, o.final_side[2:])
    gnet.close()
    return o


def test_flowcutter_random(hfp, ctx):
    pierced = 0
    for i, (H, side, region) in enumerate(_random_cases(303, 150, n_lo=6, n_hi=50, m_hi=90,
                                                        c_max=4)):
        o = _fc_compare(hfp, ctx, H, side, region, seed=i, dist_given=(i % 2 == 1))
        pierced += len(o.pierce_node) > 0
    assert pierced > 20


@pytest.mark.parametrize("beta,warmup,min_bulk", [(55, 1, 40), (55, 3, 15), (70, 1, 3)])
def test_flowcutter_bulk_piercing_random(hfp, ctx, beta, warmup, min_bulk):
    """Bulk piercing (Section 7, "Bulk Piercing") against the oracle's
    reading: piercing sequence, final bipartition, flow, bulk step count."""
    bulk = 0
    for i, (H, side, region) in enumerate(_random_cases(505 + beta + warmup, 120, n_lo=10,
                                                        n_hi=60, m_hi=120, c_max=2)):
        o = _fc_compare(hfp, ctx, H, side, region, eps_pct=int((3, 10)[i % 2]), seed=i,
                        bulk_beta_pct=beta, bulk_warmup=warmup)
        bulk += o.bulk_steps
    assert bulk >= min_bulk     # (the oracle's count on this sample, so bulk steps occur)


def test_flowcutter_most_balanced_random(hfp, ctx):
    """Most balanced cut (Section 7) against the oracle: the path-free
    piercings after the first balanced cut and the chosen bipartition."""
    steps = moved = 0
    for i, (H, side, region) in enumerate(_random_cases(606, 120, n_lo=8, n_hi=50, m_hi=90,
                                                        c_max=3)):
        o = _fc_compare(hfp, ctx, H, side, region, eps_pct=int((3, 10, 25)[i % 3]), seed=i,
                        mb_reps=2)
        steps += o.mb_steps
        moved += o.result_side == 2
    assert steps > 100 and moved >= 3


def test_most_balanced_hand_case(hfp, ctx):
    c = load_golden("most_balanced.json")
    H = hypergraph_from_lists(6, c["nets"], c["net_w"], c["node_w"])
    side = np.array(c["side"], np.int32)
    region = np.array(c["region"], np.int32)
    gnet = _gpu_net(hfp, ctx, H, side, region, dist=np.array(c["dist"], np.int32))
    e = c["expected"]
    r = hfp.flowcutter(gnet, hfp.fc_params(c["max_block_weight"], seed=c["seed"],
                                           mb_reps=e["mb_reps"]))
    assert r.status == 0
    assert r.final_side.tolist() == e["final_side"][2:]
    assert (r.flow, r.source_weight, r.result_side, r.mb_steps) == \
        (e["flow"], e["source_weight"], e["result_side"], e["mb_steps"])
    assert r.pierce_side.tolist() == [2, 3] and r.pierce_node.tolist() == [4, 3]
    _check_feasible(hfp, gnet, r.flow)


@pytest.mark.parametrize("seed", [1, 2])
def test_flowcutter_extensions_ring_scaled(hfp, ctx, seed):
    """Both extensions on the 500k FlowCutter workload's generator at
    n = 20,000."""
    inst = synth.instance("ring_n500k_zipf_fc", seed, n=20000, m=30000, radius=2000)
    o = _fc_compare(hfp, ctx, inst["H"], inst["part"], inst["region"], seed=seed,
                    bulk_beta_pct=55, bulk_warmup=3, mb_reps=2)
    assert o.status == oracle.OK


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_flowcutter_ring_weighted_scaled(hfp, ctx, seed):
    """The 500k-vertex FlowCutter workload's generator (vertex weights 1..4,
    eps 0.03) at n = 20,000."""
    inst = synth.instance("ring_n500k_zipf_fc", seed, n=20000, m=30000, radius=2000)
    o = _fc_compare(hfp, ctx, inst["H"], inst["part"], inst["region"], seed=seed)
    assert o.status == oracle.OK


def test_pierce_and_augment_explicit(hfp, ctx):
    """S <- S_r + {p} and T <- T_r + {p} with caller-chosen nodes, against the
    oracle augmenting its own flow after the same terminal changes."""
    rng = np.random.default_rng(5)
    checked = 0
    for H, side, region in _random_cases(404, 80, n_lo=8, n_hi=40, m_hi=70):
        onet = oracle.build_network(H, side, region)
        if onet.n_nodes <= 3:
            continue
        gnet = _gpu_net(hfp, ctx, H, side, region)
        G = oracle.Lawler(onet)
        S = G.mask([0])
        T = G.mask([1])
        G.augment(S, T)
        hfp.max_flow(gnet)
        for step in range(12):
            Sr = G.reach_from(S)
            Tr = G.reach_to(T)
            free = [h for h in range(2, onet.n_nodes) if not Sr[h] and not Tr[h]]
            if not free:
                break
            p = int(rng.choice(free))
            side_ = int(rng.integers(0, 2))
            if side_ == 0:
                S = np.maximum(Sr, G.mask([p]))
            else:
                T = np.maximum(Tr, G.mask([p]))
            G.augment(S, T)
            _, flow = hfp.pierce_and_augment(gnet, side_, [p])
            assert flow == G.flow_value(S)
            _check_feasible(hfp, gnet, flow)
            law, _, _, _ = hfp.min_cut_source_side(gnet)
            assert np.array_equal(law, G.reach_from(S))
            tlaw, _, _ = hfp.min_cut_sink_side(gnet)
            assert np.array_equal(tlaw, G.reach_to(T))
            checked += 1
        gnet.close()
    assert checked > 150


PIERCING = load_golden("piercing_order.json")["cases"]


@pytest.mark.parametrize("c", PIERCING, ids=[c["name"] for c in PIERCING])
def test_piercing_order_hand_cases(hfp, ctx, c):
    """The hand-worked piercing cases (each key of Section 7 "Piercing"
    decides one of them) through hfp_flowcutter, distances given."""
    H = hypergraph_from_lists(6, c["nets"], c["net_w"], c["node_w"])
    side = np.array(c["side"], np.int32)
    region = np.array(c["region"], np.int32)
    gnet = _gpu_net(hfp, ctx, H, side, region, dist=np.array(c["dist"], np.int32))
    r = hfp.flowcutter(gnet, hfp.fc_params(c["max_block_weight"], seed=c["seed"]))
    e = c["expected"]
    assert r.status == 0
    assert r.pierce_side.tolist() == e["pierce_side"]
    assert r.pierce_node.tolist() == e["pierce_node"]
    assert r.final_side.tolist() == e["final_side"][2:]
    assert (r.flow, r.source_weight, r.result_side, r.iterations) == \
        (e["flow"], e["source_weight"], e["result_side"], e["iterations"])
    _check_feasible(hfp, gnet, r.flow)
    gnet.close()


def test_deterministic_runs(hfp, ctx):
    inst = synth.instance("ring_n4096_geom", 42)
    H, part, region = inst["H"], inst["part"], inst["region"]
    runs = []
    for _ in range(3):
        gnet = _gpu_net(hfp, ctx, H, part, region)
        f = hfp.max_flow(gnet)
        law, _, _, _ = hfp.min_cut_source_side(gnet)
        st = hfp.net_stats(gnet)
        runs.append((f, law.tobytes(), st["rounds"], st["pushes"], st["global_relabels"]))
        gnet.close()
    assert runs[0] == runs[1] == runs[2]


def test_round_budget_trips_and_context_stays_usable(hfp):
    """A bounded device loop that runs out returns HFP_ERR_ITER_LIMIT (no
    trap, no hang), and the same context then computes a normal flow."""
    c = hfp.ctx_create(0)
    inst = synth.instance("ring_n4096_geom", 3)
    H, part, region = inst["H"], inst["part"], inst["region"]
    onet = oracle.build_network(H, part, region)
    default = hfp.ctx_get_tuning(c)
    hfp.ctx_set_tuning(c, max_rounds=1)
    gnet = _gpu_net(hfp, c, H, part, region)
    with pytest.raises(hfp.HfpError) as e:
        hfp.max_flow(gnet)
    assert e.value.status == hfp.ERR_ITER_LIMIT
    gnet.close()
    hfp.ctx_set_tuning(c, **default)
    gnet = _gpu_net(hfp, c, H, part, region)
    _check_flow(hfp, gnet, onet)
    gnet.close()
    c.close()


@pytest.mark.parametrize("barrier", [0, 1, 2])
def test_barrier_wait_runs_out_and_context_stays_usable(hfp, barrier):
    """Each kind of device barrier (0: the engine's grid barrier, 1: a
    batched group's barrier in global memory, 2: a cluster barrier in
    distributed shared memory) waits on a count that no CTA completes: the
    wait ends by the context's timeout with HFP_ERR_ITER_LIMIT, no trap and no
    hang, and the same context then gives the oracle's flow and cuts."""
    c = hfp.ctx_create(0)
    default = hfp.ctx_get_tuning(c)
    assert default["wait_timeout_ms"] == 10000
    hfp.ctx_set_tuning(c, wait_timeout_ms=200)
    assert hfp.ctx_get_tuning(c)["wait_timeout_ms"] == 200
    st, ms = hfp.ctx_wait_selftest(c, barrier)
    assert st == hfp.ERR_ITER_LIMIT
    assert 200.0 <= ms < 5000.0
    for bad in (0, 600001):
        with pytest.raises(hfp.HfpError) as e:
            hfp.ctx_set_tuning(c, wait_timeout_ms=bad)
        assert e.value.status == hfp.ERR_INVALID
    assert hfp.ctx_get_tuning(c)["wait_timeout_ms"] == 200   # a refused set changes nothing
    inst = synth.instance("ring_n4096_geom", 4)
    H, part, region = inst["H"], inst["part"], inst["region"]
    onet = oracle.build_network(H, part, region)
    gnet = _gpu_net(hfp, c, H, part, region)
    _check_flow(hfp, gnet, onet)
    gnet.close()
    c.close()


@pytest.fixture(scope="module")
def ctx_dedup(hfp):
    c = hfp.ctx_create(0)
    hfp.ctx_set_tuning(c, identical_nets=1)
    yield c
    c.close()


def _check_dedup(hfp, ctx_dedup, H, side, region, fc_seed=None):
    """The device network with identical nets merged equals the oracle's
    merged network (structure bit for bit), and so do its flow and cuts; the
    hypernode cut sides equal those of the unmerged network."""
    gnet = _gpu_net(hfp, ctx_dedup, H, side, region)
    full = oracle.build_network(H, side, region)
    onet = oracle.dedup_network(full)
    ex = hfp.net_export(gnet)
    assert (gnet.info.m_nets, gnet.info.p_pins) == (onet.m_nets, onet.p)
    assert np.array_equal(ex["net_off"], onet.net_off)
    assert np.array_equal(ex["pins"], onet.pins)
    assert np.array_equal(ex["net_w"], onet.net_w)
    assert np.array_equal(ex["net_gid"], onet.net_gid)
    off, slots = _expected_incidence(onet)
    assert np.array_equal(ex["node_off"], off)
    assert np.array_equal(ex["inc_slot"], slots)
    mc = _check_flow(hfp, gnet, onet)
    mf = oracle.max_flow_min_cut(full)
    nh = full.n_nodes
    assert mc.flow == mf.flow
    assert np.array_equal(mc.source_side[:nh], mf.source_side[:nh])
    assert np.array_equal(mc.sink_side[:nh], mf.sink_side[:nh])
    gnet.close()
    return full.m_nets - onet.m_nets


def test_identical_nets_hand_case(hfp, ctx_dedup):
    g = load_golden("identical_nets.json")
    side = np.array(g["side"], np.int32)
    region = np.array(g["region"], np.int32)
    for nets, w in ((g["nets"], g["net_w"]), (g["collision"]["nets"], g["collision"]["net_w"])):
        H = hypergraph_from_lists(g["n"], nets, w)
        _check_dedup(hfp, ctx_dedup, H, side, region)


def test_identical_nets_random_and_rings(hfp, ctx_dedup):
    merged = 0
    for H, side, region in _random_cases(707, 120, n_lo=4, n_hi=40, m_hi=120):
        merged += _check_dedup(hfp, ctx_dedup, H, side, region)
    for seed in (1, 2, 3):
        inst = synth.instance("ring_n4096_geom", seed)
        merged += _check_dedup(hfp, ctx_dedup, inst["H"], inst["part"], inst["region"])
    inst = synth.instance("ring_n2M_zipf", 2, n=20000, m=30000, radius=2000)
    merged += _check_dedup(hfp, ctx_dedup, inst["H"], inst["part"], inst["region"])
    assert merged > 50


def test_identical_nets_flowcutter_unchanged(hfp, ctx, ctx_dedup):
    inst = synth.instance("ring_n500k_zipf_fc", 2, n=20000, m=30000, radius=2000)
    H, side, region = inst["H"], inst["part"], inst["region"]
    L = oracle.max_block_weight(int(oracle.build_network(H, side, region).node_w.sum()), 2, 3)
    res = []
    for c in (ctx, ctx_dedup):
        gnet = _gpu_net(hfp, c, H, side, region)
        r = hfp.flowcutter(gnet, hfp.fc_params(L, seed=4))
        res.append((r.status, r.flow, r.iterations, r.pierce_node.tolist(), r.final_side.tobytes()))
        gnet.close()
    assert res[0] == res[1]


@pytest.fixture(scope="module")
def ctx_parpr(hfp):
    c = hfp.ctx_create(0)
    hfp.ctx_set_tuning(c, parpr_block=1)
    yield c
    c.close()


def test_parpr_block_flows_and_cuts(hfp, ctx_parpr):
    """ParPR-Block (Section 8.2, first fix of the push-relabel conflict) as
    the rounds' relabel rule: the flow value, both minimal cuts and the
    per-arc preflow's feasibility are checked against the oracle like the
    default rule's."""
    for H, side, region in _random_cases(909, 120, n_lo=4, n_hi=60, m_hi=120):
        gnet = _gpu_net(hfp, ctx_parpr, H, side, region)
        _check_flow(hfp, gnet, oracle.build_network(H, side, region))
        gnet.close()
    for seed in range(1, 21):
        inst = synth.instance("ring_n4096_geom", seed)
        gnet = _gpu_net(hfp, ctx_parpr, inst["H"], inst["part"], inst["region"])
        _check_flow(hfp, gnet, oracle.build_network(inst["H"], inst["part"], inst["region"]))
        gnet.close()


def test_parpr_block_flowcutter_unchanged(hfp, ctx, ctx_parpr):
    """FlowCutter with ParPR-Block rounds takes the same piercing sequence and
    ends in the same bipartition (max flow values and minimal cuts are
    unique), on a scaled ring and on random networks."""
    cases = [(synth.instance("ring_n500k_zipf_fc", 3, n=20000, m=30000, radius=2000), 5)]
    for inst, seed in cases:
        H, side, region = inst["H"], inst["part"], inst["region"]
        L = oracle.max_block_weight(int(oracle.build_network(H, side, region).node_w.sum()), 2, 3)
        res = []
        for c in (ctx, ctx_parpr):
            gnet = _gpu_net(hfp, c, H, side, region)
            r = hfp.flowcutter(gnet, hfp.fc_params(L, seed=seed))
            res.append((r.status, r.flow, r.iterations, r.pierce_node.tolist(),
                        r.final_side.tobytes()))
            gnet.close()
        assert res[0] == res[1]
        assert res[0][2] > 3
    for i, (H, side, region) in enumerate(_random_cases(911, 40, n_lo=6, n_hi=50, m_hi=90,
                                                        c_max=4)):
        _fc_compare(hfp, ctx_parpr, H, side, region, seed=i)
