"""The oracle's piercing order pinned by hand-worked cases (CPU only).

tests/golden/piercing_order.json holds small networks where each rule of
Section 7 "Piercing" decides the pierced node on its own: a path-free
candidate before one that opens an augmenting path, then the larger signed
distance from the original cut (for either growing side), then the smaller
fmix32(id ^ seed).  Every expected value was worked out by hand from the
paper's rules; the hash values used are published MurmurHash3 test vectors.
A flipped distance comparison, a dropped sign, a dropped or inverted
path-free key, or a hash compared the other way each change at least one
case's pierced node.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import hypergraph_from_lists, load_golden

CASES = load_golden("piercing_order.json")["cases"]


def run_case(c):
    H = hypergraph_from_lists(6, c["nets"], c["net_w"], c["node_w"])
    side = np.array(c["side"], np.int32)
    region = np.array(c["region"], np.int32)
    net = oracle.build_network(H, side, region)
    orig, d, gid = oracle.node_arrays(net, side, region, np.array(c["dist"], np.int32))
    return oracle.flowcutter(net, c["max_block_weight"], orig, d, gid, seed=c["seed"])


@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_piercing_order_hand_cases(c):
    r = run_case(c)
    e = c["expected"]
    assert r.status == oracle.OK
    assert r.pierce_side.tolist() == e["pierce_side"]
    assert r.pierce_node.tolist() == e["pierce_node"]
    assert r.final_side.tolist() == e["final_side"]
    assert r.flow == e["flow"]
    assert r.source_weight == e["source_weight"]
    assert r.result_side == e["result_side"]
    assert r.iterations == e["iterations"]


def test_cases_cover_each_rule():
    # the set of cases separates every key: both growing sides, a signed
    # distance that contradicts the unsigned one, a path-opening candidate
    # with the best distance, and both orders of the hash
    names = {c["name"] for c in CASES}
    assert {"grow_s_larger_distance_wins", "grow_s_signed_distance",
            "grow_t_larger_distance_wins", "grow_t_signed_distance",
            "path_free_beats_closer_to_cut", "tie_broken_by_hash_seed2",
            "tie_broken_by_hash_seed3"} <= names
    sides = {c["expected"]["pierce_side"][0] for c in CASES}
    assert sides == {0, 1}
