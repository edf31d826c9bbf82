"""Nesting of the minimal source side across FlowCutter steps (Algorithm 2,
Section 7; the min-cut lattice of Section 2).  Growing S to S_r + {v} can
only keep or enlarge the minimal source side S_r, and growing T to
T_r + {v} can only keep or shrink it.  Checked on the oracle's own piercing
sequences, replayed with its Lawler graph (augment to a maximum flow, then
residual reachability), on random networks and on scaled rings whose runs
pierce on either side.  These are the facts an incremental source-side
search after a piercing relies on."""
import numpy as np

import oracle
import synth
from tests.helpers import random_instance


def _run(H, side, region, seed):
    net = oracle.build_network(H, side, region)
    dist = oracle.dist_from_cut(H, side, region)
    orig, d, gid = oracle.node_arrays(net, side, region, dist)
    L = oracle.max_block_weight(int(net.node_w.sum()), 2, 3)
    return net, oracle.flowcutter(net, L, orig, d, gid, seed=seed)


def _replay(net, fc):
    """Counts of checked steps after a source-side and a sink-side piercing."""
    G = oracle.Lawler(net)
    ids = np.arange(net.lawler_nodes)
    S, T = G.mask([0]), G.mask([1])
    prev = None
    checked = [0, 0]
    for v, sd in zip(fc.pierce_node.tolist(), fc.pierce_side.tolist()):
        G.augment(S, T)
        sr = G.reach_from(S).astype(bool)
        tr = G.reach_to(T).astype(bool)
        if prev is not None:
            old, pside = prev
            if pside == 0:
                assert not (old & ~sr).any(), "source-side piercing lost S_r nodes"
            else:
                assert not (sr & ~old).any(), "sink-side piercing added S_r nodes"
            checked[pside] += 1
        prev = (sr, sd)
        if sd == 0:
            S = (sr | (ids == v)).astype(np.uint8)
        else:
            T = (tr | (ids == v)).astype(np.uint8)
    return checked


def test_source_side_nesting_on_random_networks():
    rng = np.random.default_rng(2024)
    tot = [0, 0]
    for i in range(60):
        H, side, region = random_instance(rng, int(rng.integers(12, 60)), int(rng.integers(15, 110)),
                                          max_size=5, region_frac=0.8, w_max=6)
        net, fc = _run(H, side, region, seed=i)
        c = _replay(net, fc)
        tot[0] += c[0]
        tot[1] += c[1]
    assert tot[0] > 0 and tot[1] > 0


def test_source_side_nesting_on_scaled_rings():
    tot = [0, 0]
    for seed in (3, 9):
        inst = synth.instance("ring_n500k_zipf_fc", seed, n=6000, m=9000, radius=600)
        net, fc = _run(inst["H"], inst["part"], inst["region"], seed)
        c = _replay(net, fc)
        tot[0] += c[0]
        tot[1] += c[1]
    assert sum(tot) > 20
