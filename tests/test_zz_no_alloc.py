"""hfp_max_flow_noalloc: the entry point for callers that cannot allocate
device memory (inside a stream capture, under a host application's fixed
memory budget or allocator, in an allocation-free loop).  Its working state
is a fixed static device array, so these tests check that, called twice in a
row on different networks through the C ABI, it gives exactly the flow value,
source-side weight and minimal source side S_r of the allocating entry points
(hfp_max_flow + hfp_min_cut_source_side), and that it rejects networks that
do not fit its array.

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
