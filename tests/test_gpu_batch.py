"""Batched FlowCutter (all problems in one cooperative launch, a device work
queue, groups of CTAs per problem): outcome identical to one hfp_flowcutter
call per network (piercing sequence, final bipartition, flow), for several
group sizes; the batched k-way round identical to the plain round and to
the oracle; the autotuner."""
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
    return torch, hfp, hfp.ctx_create(0)


def _problems(seeds, n=None, radius=None):
    out = []
    for wl, seed in seeds:
        kw = {}
        if n is not None and wl != "ring_n4096_geom":
            kw = dict(n=n, m=n * 3 // 2, radius=radius)
        inst = synth.instance(wl, seed, **kw)
        out.append(inst)
    return out


def _build(hfp, ctx, inst):
    H, part, region = inst["H"], inst["part"], inst["region"]
    return hfp.build_flow_network(ctx, H.net_off, H.pins, H.net_w, H.node_w, region, part, H.n)


def _fc_params(hfp, inst, seed, bound=-1):
    H = inst["H"]
    L = oracle.max_block_weight(int(H.node_w.sum()), 2, 3)
    return hfp.fc_params(L, flow_bound=bound, seed=seed)


CASES = ([("ring_n4096_geom", s) for s in range(1, 9)] +
         [("ring_n500k_zipf_fc", s) for s in range(1, 5)])


@pytest.mark.parametrize("group", [0, 1, 2, 8])
def test_batch_equals_single_calls(env, group):
    torch, hfp, ctx = env
    insts = _problems(CASES, n=40_000, radius=4_000)
    single = []
    for t, inst in enumerate(insts):
        net = _build(hfp, ctx, inst)
        single.append(hfp.flowcutter(net, _fc_params(hfp, inst, t)))
        net.close()
    nets = [_build(hfp, ctx, inst) for inst in insts]
    res = hfp.flowcutter_batch(ctx, nets, [_fc_params(hfp, inst, t) for t, inst in enumerate(insts)],
                               group_ctas=group)
    for a, b in zip(res, single):
        assert (a.status, a.flow, a.iterations, a.result_side, a.source_weight) == (
            b.status, b.flow, b.iterations, b.result_side, b.source_weight)
        assert np.array_equal(a.pierce_side, b.pierce_side)
        assert np.array_equal(a.pierce_node, b.pierce_node)
        assert np.array_equal(a.final_side, b.final_side)
    assert sum(r.iterations for r in res) > len(res)    # piercing happened


def test_batch_outcomes_and_errors(env):
    torch, hfp, ctx = env
    insts = _problems([("ring_n4096_geom", 11), ("ring_n4096_geom", 12)])
    nets = [_build(hfp, ctx, inst) for inst in insts]
    # a flow bound of 0 aborts the first problem; the second runs normally
    prm = [_fc_params(hfp, insts[0], 0, bound=0), _fc_params(hfp, insts[1], 0)]
    res = hfp.flowcutter_batch(ctx, nets, prm)
    assert res[0].status == hfp.ABORTED_WORSE
    assert res[1].status == hfp.OK
    # networks with a flow already computed are refused
    with pytest.raises(hfp.HfpError) as e:
        hfp.flowcutter_batch(ctx, nets[:1], prm[:1])
    assert e.value.status == hfp.ERR_STATE
    assert hfp.flowcutter_batch(ctx, [], []) == []
    # the oracle agrees on the second problem
    inst = insts[1]
    H, part, region = inst["H"], inst["part"], inst["region"]
    onet = oracle.build_network(H, part, region)
    L = oracle.max_block_weight(int(onet.node_w.sum()), 2, 3)
    dist = oracle.dist_from_cut(H, part, region)
    orig, d, gid = oracle.node_arrays(onet, part, region, dist)
    o = oracle.flowcutter(onet, L, orig, d, gid, seed=0)
    assert res[1].flow == o.flow and np.array_equal(res[1].pierce_node, o.pierce_node)


def _kway(env, seed, n, k):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n8M_zipf_k64", seed, n=n, m=n * 3 // 2)
    H = inst["H"]
    part = inst["part"] if k == 64 else synth.kway_partition(n, k, 50_000, seed)
    hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
    return H, part, hg


@pytest.mark.parametrize("seed,n,k,group", [(3, 16000, 64, 0), (4, 40000, 16, 2),
                                            (5, 60000, 8, 4)])
def test_batched_round_equals_plain_round(env, seed, n, k, group):
    torch, hfp, ctx = env
    H, part, hg = _kway(env, seed, n, k)
    p1 = torch.from_numpy(part.copy()).cuda()
    p2 = torch.from_numpy(part.copy()).cuda()
    s1, r1 = hfp.refine_round(hg, p1, k, hfp.refine_params(seed=5))
    s2, r2, ms = hfp.refine_round_batched(hg, p2, k, hfp.refine_params(seed=5), group_ctas=group)
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    for f in ("connectivity_before", "connectivity_after", "gain", "moves_applied", "pairs",
              "pairs_improved", "pairs_applied"):
        assert getattr(s1, f) == getattr(s2, f), f
    for a, b in zip(r1, r2):
        for f in ("bi", "bj", "status", "region_size", "pins", "original_cut", "flow",
                  "delta_exp", "n_moves", "iterations", "applied", "valid_moves", "gain"):
            assert getattr(a, f) == getattr(b, f), f
    assert ms > 0
    if seed == 3:
        newp, total, _, _ = oracle.refine_round(H, part, k, seed=5)
        assert np.array_equal(p2.cpu().numpy(), newp) and s2.gain == total


@pytest.mark.parametrize("group,big_ctas,big_groups,cluster", [(4, 16, 3, 1), (2, 32, 2, 1),
                                                                (4, 0, 0, 0), (8, 0, 0, 1),
                                                                (16, 0, 0, 2), (4, 0, 0, 2)])
def test_batched_round_group_layouts(env, group, big_ctas, big_groups, cluster):
    """Mixed group sizes (big groups for the largest problems), and uniform
    groups as clusters or in one cooperative launch, give the plain round's
    outcome and report per-pair device times.  batch_cluster = 2 always
    launches clusters (as many groups as can be resident), 0 never does."""
    torch, hfp, ctx = env
    H, part, hg = _kway(env, 6, 30000, 16)
    base = hfp.ctx_get_tuning(ctx)
    p1 = torch.from_numpy(part.copy()).cuda()
    p2 = torch.from_numpy(part.copy()).cuda()
    s1, r1 = hfp.refine_round(hg, p1, 16, hfp.refine_params(seed=2))
    try:
        hfp.ctx_set_tuning(ctx, batch_big_ctas=big_ctas, batch_big_groups=big_groups,
                           batch_cluster=cluster)
        s2, r2, ms = hfp.refine_round_batched(hg, p2, 16, hfp.refine_params(seed=2),
                                              group_ctas=group)
        layout = hfp.ctx_last_batch_layout(ctx)
    finally:
        hfp.ctx_set_tuning(ctx, **base)
    assert layout["group_ctas"] == group
    if cluster == 2:
        assert layout["cluster"] == 1 and layout["groups"] >= 1
    if cluster == 0 or big_groups:
        assert layout["cluster"] == 0
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    assert s1.connectivity_after == s2.connectivity_after and s1.pairs == s2.pairs
    for a, b in zip(r1, r2):
        for f in ("bi", "bj", "status", "flow", "delta_exp", "n_moves", "iterations"):
            assert getattr(a, f) == getattr(b, f), f
    assert all(r.device_us > 0 for r in r2) and all(r.device_us == 0 for r in r1)
    sizes = sorted({r.group_ctas for r in r2})
    if big_groups:
        # the largest problems started on the big groups
        by_pins = sorted(r2, key=lambda r: -r.pins)
        assert all(r.group_ctas == big_ctas for r in by_pins[:min(big_groups, len(r2))])
        assert sizes == sorted({group, big_ctas}) or sizes == [big_ctas]
    else:
        assert sizes == [group]


def test_autotune_and_tuned_round(env):
    torch, hfp, ctx = env
    H, part, hg = _kway(env, 7, 30000, 32)
    pd = torch.from_numpy(part.copy()).cuda()
    best, ms = hfp.autotune_round(hg, pd, 32, [1, 2, 4])
    assert best in (1, 2, 4) and np.all(ms > 0)
    assert ms[[1, 2, 4].index(best)] == ms.min()
    assert np.array_equal(pd.cpu().numpy(), part)          # the autotuner applies nothing
    p1 = torch.from_numpy(part.copy()).cuda()
    s1, _ = hfp.refine_round(hg, p1, 32)
    s2, _, _ = hfp.refine_round_batched(hg, pd, 32)         # uses the tuned group size
    assert s1.gain == s2.gain and np.array_equal(p1.cpu().numpy(), pd.cpu().numpy())
    with pytest.raises(hfp.HfpError):
        hfp.autotune_round(hg, pd, 32, [0])
