"""hfp_max_flow_noalloc: the entry point for callers that cannot allocate
device memory where they need a flow (a plug-in held to a host
application's fixed device-memory budget or allocator, a loop in which
allocation is forbidden).  Its working state is a fixed static device array,
so these tests check that, called twice in a row on different networks
through the C ABI, it gives exactly the flow value, source-side weight and
minimal source side S_r of the allocating entry points (hfp_max_flow +
hfp_min_cut_source_side); that repeated calls leave the device's free memory
where it was; that it rejects networks that do not fit its array; and that
an inconsistent view is refused with HFP_ERR_INVALID before any flow runs.

This file is collected last on purpose; it passes alone in a fresh process
and after the other tests.
"""
import numpy as np
import pytest

import synth
from tests.helpers import random_instance

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
    ctx.close()


def _reference(hfp, ctx, H, side, region):
    net = hfp.build_flow_network(ctx, H.net_off, H.pins, H.net_w, H.node_w, region, side, H.n)
    flow = hfp.max_flow(net)
    law, _, _, ws = hfp.min_cut_source_side(net)
    view = hfp.net_export_device(net)
    return net, flow, law, ws, view


def test_noalloc_matches_allocating_path_twice_in_a_row(env):
    torch, hfp, ctx = env
    cases = []
    for seed in (3, 4):
        inst = synth.instance("ring_n4096_geom", seed)
        cases.append((inst["H"], inst["part"], inst["region"]))
    rng = np.random.default_rng(77)
    cases.append(random_instance(rng, 40, 70, max_size=6, region_frac=0.7, w_max=9))
    stream = torch.cuda.current_stream().cuda_stream
    for H, side, region in cases:
        net, flow, law, ws, view = _reference(hfp, ctx, H, side, region)
        i = net.info
        for _ in range(2):                       # two calls in a row on the same array
            out = torch.full((i.lawler_nodes,), 7, dtype=torch.uint8, device="cuda")
            f2, w2 = hfp.max_flow_noalloc(0, stream, view, i.n_nodes, i.m_nets, i.p_pins, out)
            torch.cuda.synchronize()
            assert f2 == flow
            assert w2 == ws
            assert np.array_equal(out.cpu().numpy(), law)
        net.close()


def test_noalloc_rejects_networks_beyond_its_array(env):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n4096_geom", 5)
    net, flow, law, ws, view = _reference(hfp, ctx, inst["H"], inst["part"], inst["region"])
    i = net.info
    with pytest.raises(hfp.HfpError) as e:
        hfp.max_flow_noalloc(0, torch.cuda.current_stream().cuda_stream, view, i.n_nodes,
                             4_000_000, i.p_pins)
    assert e.value.status == hfp.ERR_INVALID
    net.close()


def test_noalloc_does_not_change_free_device_memory(env):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n4096_geom", 6)
    net, flow, law, ws, view = _reference(hfp, ctx, inst["H"], inst["part"], inst["region"])
    i = net.info
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.zeros(i.lawler_nodes, dtype=torch.uint8, device="cuda")
    hfp.max_flow_noalloc(0, stream, view, i.n_nodes, i.m_nets, i.p_pins, out)   # loads kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        f2, w2 = hfp.max_flow_noalloc(0, stream, view, i.n_nodes, i.m_nets, i.p_pins, out)
        assert (f2, w2) == (flow, ws)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # an allocation in the call would lower the free memory; pools of earlier
    # work may only hand memory back
    assert free1 >= free0
    net.close()


def test_noalloc_rejects_inconsistent_views(env):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n4096_geom", 8)
    net, flow, law, ws, view = _reference(hfp, ctx, inst["H"], inst["part"], inst["region"])
    i = net.info
    stream = torch.cuda.current_stream().cuda_stream
    # a pin id equal to n_nodes (out of range)
    bad = dict(view)
    bad["pins"] = view["pins"].clone()
    bad["pins"][5] = i.n_nodes
    with pytest.raises(hfp.HfpError) as e:
        hfp.max_flow_noalloc(0, stream, bad, i.n_nodes, i.m_nets, i.p_pins)
    assert e.value.status == hfp.ERR_INVALID
    # two incidence entries of different hypernodes swapped: every id is in
    # range, but the lists name pin slots of other nodes
    off = view["node_off"].cpu().numpy()
    deg = np.diff(off.astype(np.int64))
    u, w = [int(h) for h in np.nonzero(deg[2:] >= 2)[0][:2] + 2]
    bad = dict(view)
    bad["inc_slot"] = view["inc_slot"].clone()
    a, b = int(off[u]), int(off[w])
    bad["inc_slot"][a], bad["inc_slot"][b] = view["inc_slot"][b].item(), view["inc_slot"][a].item()
    with pytest.raises(hfp.HfpError) as e:
        hfp.max_flow_noalloc(0, stream, bad, i.n_nodes, i.m_nets, i.p_pins)
    assert e.value.status == hfp.ERR_INVALID
    # the same slot named twice (another slot of the node left out)
    bad = dict(view)
    bad["inc_slot"] = view["inc_slot"].clone()
    bad["inc_slot"][a + 1] = view["inc_slot"][a].item()
    with pytest.raises(hfp.HfpError) as e:
        hfp.max_flow_noalloc(0, stream, bad, i.n_nodes, i.m_nets, i.p_pins)
    assert e.value.status == hfp.ERR_INVALID
    # the untouched view still gives the allocating path's answer
    f2, w2 = hfp.max_flow_noalloc(0, stream, view, i.n_nodes, i.m_nets, i.p_pins)
    assert (f2, w2) == (flow, ws)
    net.close()
