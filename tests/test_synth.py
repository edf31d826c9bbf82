"""The seeded generators: deterministic, and shaped as the workloads state."""
import numpy as np

import synth


def test_deterministic_and_seed_dependent():
    a = synth.ring_hypergraph(5000, 7000, synth.ZIPF, 500, 256, (1, 10), (1, 4), seed=7)
    b = synth.ring_hypergraph(5000, 7000, synth.ZIPF, 500, 256, (1, 10), (1, 4), seed=7)
    c = synth.ring_hypergraph(5000, 7000, synth.ZIPF, 500, 256, (1, 10), (1, 4), seed=8)
    for f in ("net_off", "pins", "net_w", "node_w"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.pins[:1000], c.pins[:1000])


def test_ring_windows_and_weights():
    n, window = 4096, 64
    H = synth.ring_hypergraph(n, 6144, synth.GEOMETRIC, 16, window, (1, 4), (1, 1), seed=3)
    sizes = np.diff(H.net_off.astype(np.int64))
    assert sizes.min() >= 2 and sizes.max() <= 16
    # 2 + Geometric(1/2): mean 3
    assert abs(sizes.mean() - 3.0) < 0.1
    assert H.net_w.min() >= 1 and H.net_w.max() <= 4
    assert np.all(H.node_w == 1)
    for e in range(0, H.m, 7):
        ps = H.pins[H.net_off[e]:H.net_off[e + 1]]
        assert len(set(ps.tolist())) == len(ps)          # without replacement
        assert np.all(np.diff(ps) > 0)                   # ascending
        # all pins fit in one window of the ring (circular span < window)
        gaps = np.diff(np.concatenate([ps, [ps[0] + n]]))
        assert n - gaps.max() < max(window, 2 * len(ps))


def test_zipf_sizes():
    H = synth.ring_hypergraph(100000, 150000, synth.ZIPF, 5000, 4096, (1, 10), (1, 1), seed=1)
    sizes = np.diff(H.net_off.astype(np.int64)) - 2
    # P(Z = 1) = 1 / zeta_truncated(2.5) ~ 0.7454
    assert abs((sizes == 1).mean() - 0.7454) < 0.01
    assert sizes.max() <= 4998


def test_region_and_partitions():
    n = 1000
    r = synth.region_near_cuts(n, 10)
    assert r.tolist() == list(range(0, 10)) + list(range(490, 510)) + list(range(990, 1000))
    p = synth.halves(n)
    assert p[:500].sum() == 0 and p[500:].sum() == 500
    k = synth.kway_partition(64000, 64, 50000, seed=2)
    base = (np.arange(64000) * 64) // 64000
    moved = k != base
    assert abs(moved.mean() - 0.05) < 0.005
    d = (k[moved] - base[moved]) % 64
    assert set(d.tolist()) <= {1, 63}
