"""Shared test helpers: small random instances and hand fixtures.

Only seeded input construction lives here; no flow arithmetic.
"""
import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def hypergraph_from_lists(n, nets, net_w, node_w=None):
    off = np.zeros(len(nets) + 1, dtype=np.uint32)
    for i, e in enumerate(nets):
        off[i + 1] = off[i] + len(e)
    pins = np.array([v for e in nets for v in e], dtype=np.int32)
    nw = np.ones(n, np.int32) if node_w is None else np.asarray(node_w, np.int32)
    return synth.Hypergraph(n, len(nets), off, pins, np.asarray(net_w, np.int32), nw)


def random_instance(rng, n, m, max_size=4, region_frac=0.6, w_max=5, c_max=1, k_sides=2):
    """Random small hypergraph, random sides (0/1) and a random region."""
    nets = []
    for _ in range(m):
        sz = int(rng.integers(2, max_size + 1))
        sz = min(sz, n)
        nets.append(sorted(rng.choice(n, size=sz, replace=False).tolist()))
    net_w = rng.integers(1, w_max + 1, size=m)
    node_w = rng.integers(1, c_max + 1, size=n)
    H = hypergraph_from_lists(n, nets, net_w, node_w)
    side = rng.integers(0, k_sides, size=n).astype(np.int32)
    if k_sides > 2:
        side[side >= 2] = -1
    cand = np.nonzero(side >= 0)[0]
    r = max(1, int(len(cand) * region_frac))
    region = np.sort(rng.choice(cand, size=min(r, len(cand)), replace=False)).astype(np.int32)
    return H, side, region
