"""Full-size parity with values the CPU oracle wrote (tests/golden/
make_golden.py calls only oracle/): the 2,000,000-vertex max flow (flow,
S_r and T_r over every Lawler node, as sha256 of the packed bits) and the
500,000-vertex FlowCutter run (piercing sequence, final bipartition, cut),
in the same call sequence bench.py times.  Also optimality certificates
that hold at any size."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth
from tests.flowcheck import check_preflow

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _digest(mask):
    return hashlib.sha256(np.packbits(np.asarray(mask, dtype=np.uint8), bitorder="little")
                          .tobytes()).hexdigest()


def _load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.fail(f"missing oracle golden file {name}")
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def hfp_ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_01556_gb300 import hfp
    hfp.load()
    return torch, hfp, hfp.ctx_create(0, torch.cuda.current_stream().cuda_stream)


def test_ring_2M_max_flow_and_cuts(hfp_ctx):
    torch, hfp, ctx = hfp_ctx
    g = _load("ring_n2M_zipf_seed1_maxflow.json")
    inst = synth.instance("ring_n2M_zipf", 1)
    H, part, region = inst["H"], inst["part"], inst["region"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    net = hfp.build_flow_network(ctx, dev(H.net_off), dev(H.pins), dev(H.net_w), dev(H.node_w),
                                 dev(region), dev(part), H.n)
    assert (net.info.n_nodes, net.info.m_nets, net.info.p_pins) == (g["n_nodes"], g["m_nets"],
                                                                    g["p_pins"])
    assert hfp.max_flow(net) == g["flow"]
    law, reg, cuts, ws = hfp.min_cut_source_side(net)
    assert int(law.sum()) == g["source_side_count"]
    assert _digest(law) == g["source_side_sha256"]
    tlaw, _, _ = hfp.min_cut_sink_side(net)
    assert int(tlaw.sum()) == g["sink_side_count"]
    assert _digest(tlaw) == g["sink_side_sha256"]
    # certificate: the cut nets of S_r weigh exactly the flow (max-flow = min-cut)
    ex = hfp.net_export(net)
    gid_w = dict(zip(ex["net_gid"].tolist(), ex["net_w"].tolist()))
    assert sum(gid_w[e] for e in cuts.tolist()) == g["flow"]
    # the device's per-arc preflow is feasible and carries the value
    check_preflow(net.info.n_nodes, ex["net_off"], ex["pins"], ex["net_w"],
                  hfp.net_export_flow(net), g["flow"])


def test_ring_500k_flowcutter(hfp_ctx):
    torch, hfp, ctx = hfp_ctx
    g = _load("ring_n500k_zipf_fc_seed1_flowcutter.json")
    inst = synth.instance("ring_n500k_zipf_fc", 1)
    H, part, region = inst["H"], inst["part"], inst["region"]
    net = hfp.build_flow_network(ctx, H.net_off, H.pins, H.net_w, H.node_w, region, part, H.n)
    r = hfp.flowcutter(net, hfp.fc_params(g["max_block_weight"], seed=g["fc_seed"]))
    assert r.status == g["status"]
    assert r.flow == g["flow"]
    assert r.iterations == g["iterations"]
    assert r.result_side == g["result_side"]
    assert r.source_weight == g["source_weight"]
    assert r.pierce_side.tolist() == g["pierce_side"]
    assert r.pierce_node.tolist() == g["pierce_node"]
    assert int(r.final_side.sum()) == g["final_side_count"]
    assert _digest(r.final_side) == g["final_side_sha256"]
