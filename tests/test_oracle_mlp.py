"""Pins of the scheduler oracle (CPU only): bfloat16 rounding, the pair
statistics and features, forward / backward of the MLP, Adam."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from tests.helpers import hypergraph_from_lists


def test_bf16_hand_values():
    f = np.float32
    one = f(1.0)
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7 + 2.0 ** -20,
                     -(1 + 2.0 ** -8 + 2.0 ** -20), 3.0e38, 0.0, -0.0], f)
    exp = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -(1 + 2.0 ** -7), None, 0.0, -0.0],
                   dtype=object)
    got = mlp.bf16(vals)
    for g, e, v in zip(got, exp, vals):
        if e is not None:
            assert g == f(e), (v, g, e)
    assert got[0] == one
    assert np.isnan(mlp.bf16(np.array([np.nan], f)))[0]


def test_bf16_matches_torch_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = rng.standard_normal(200_000).astype(np.float32) * np.float32(10.0) ** rng.integers(
        -30, 30, 200_000).astype(np.float32)
    # exact ties: lower 16 bits 0x8000 with both parities of the kept part
    u = rng.integers(0, 2 ** 31, 20_000, dtype=np.uint64).astype(np.uint32)
    ties = ((u & np.uint32(0x7F7F0000)) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([a, ties])
    x = x[np.isfinite(x)]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16(x).view(np.uint32), ref.view(np.uint32))


def _small_kway():
    nets = [[0, 1], [1, 3], [2, 4, 6], [5, 7], [7, 8], [0, 8], [3, 4, 5]]
    H = hypergraph_from_lists(9, nets, [1, 2, 3, 4, 5, 6, 7])
    return H, np.array([0, 0, 0, 1, 1, 1, 2, 2, 2], np.int32)


def test_pair_stats_hand_example():
    H, part = _small_kway()
    s = mlp.pair_stats(H, part, 3)
    # (0,1): nets {1,3} (w2, size 2, blocks {0,1}) and {2,4,6} (w3, size 3, blocks {0,1,2})
    assert s[0, 1].tolist() == [2, 5, 5, 3, 1, 2, 2, 0]
    # (0,2): {2,4,6} and {0,8} (w6, size 2, exactly {0,2})
    assert s[0, 2].tolist() == [2, 9, 5, 3, 1, 6, 2, 0]
    # (1,2): {2,4,6} and {5,7} (w4, size 2, exactly {1,2})
    assert s[1, 2].tolist() == [2, 7, 5, 3, 1, 4, 2, 0]
    assert np.all(s[np.tril_indices(3)] == 0)


def test_pair_stats_brute_force_and_quotient():
    rng = np.random.default_rng(5)
    for _ in range(10):
        n, k = int(rng.integers(10, 60)), int(rng.integers(2, 7))
        nets = [sorted(rng.choice(n, int(rng.integers(2, 8)), replace=False).tolist())
                for _ in range(int(rng.integers(5, 80)))]
        w = rng.integers(1, 10, len(nets))
        H = hypergraph_from_lists(n, nets, w)
        part = rng.integers(0, k, n).astype(np.int32)
        s = mlp.pair_stats(H, part, k)
        qn, qw = oracle.quotient(H, part, k)
        assert np.array_equal(s[:, :, 0], qn) and np.array_equal(s[:, :, 1], qw)
        exp = np.zeros((k, k, 8), np.int64)
        for e, pins in enumerate(nets):
            blocks = sorted(set(part[pins].tolist()))
            for a in blocks:
                for b in blocks:
                    if a < b:
                        r = exp[a, b]
                        r[0] += 1
                        r[1] += w[e]
                        r[2] += len(pins)
                        r[3] = max(r[3], len(pins))
                        if len(blocks) == 2:
                            r[4] += 1
                            r[5] += w[e]
                            r[6] += len(pins)
        assert np.array_equal(s, exp)


def test_pair_features_hand_example():
    H, part = _small_kway()
    prev = -np.ones((3, 3), np.int64)
    prev[0, 2] = 4
    pairs, X = mlp.pair_features(H, part, 3, 4, prev)
    assert pairs.tolist() == [[0, 1], [0, 2], [1, 2]]
    f = np.float32
    r = X[0]
    assert r[0] == np.log1p(f(2)) and r[1] == np.log1p(f(5)) and r[2] == np.log1p(f(5))
    assert r[3] == np.log1p(f(3)) and r[4] == np.log1p(f(1)) and r[5] == np.log1p(f(2))
    assert r[6] == f(2) / f(5) and r[7] == np.log1p(f(2))
    assert r[8] == f(0.75) and r[9] == f(0.75) and r[10] == f(0.75)
    assert r[11] == np.log1p(f(2.5))
    assert r[12] == 0 and r[13] == 0 and X[1, 12] == np.log1p(f(4)) and X[1, 13] == 1
    assert r[14] == f(np.log2(3)) / f(6)
    # relative weight: 5 * 3 / (5 + 9 + 7)
    assert r[15] == f(5) * f(3) / f(21)


def _rand_params(rng, scale=0.3):
    return (rng.standard_normal(mlp.N_PARAMS) * scale).astype(np.float32)


def test_forward_hand_example():
    p = mlp.unflatten(np.zeros(mlp.N_PARAMS, np.float32))
    p["W1"][0, 0] = 1
    p["W2"][0, 0] = 1
    p["w3"][0] = 2
    p["b3"][0] = -1
    flat = mlp.flatten(p)
    X = np.zeros((2, 16), np.float32)
    X[0, 0] = 3
    X[1, 0] = -3                       # ReLU cuts the second row: z = b3
    s, c = mlp.forward(flat, X)
    assert c["z"].tolist() == [5.0, -1.0]
    assert np.allclose(s, 1 / (1 + np.exp(-np.array([5.0, -1.0]))))
    y = np.array([1.0, 0.0], np.float32)
    loss, g = mlp.backward(flat, X, y)
    gd = mlp.unflatten(g)
    dz = (s - y) / 2
    assert np.isclose(gd["b3"][0], dz.sum())
    assert np.isclose(gd["w3"][0], 3 * dz[0])
    assert np.isclose(gd["W2"][0, 0], 2 * dz[0] * 3)
    assert np.isclose(gd["W1"][0, 0], 2 * dz[0] * 3)
    assert np.isclose(gd["b1"][0], 2 * dz[0]) and np.isclose(gd["b2"][0], 2 * dz[0])
    assert np.count_nonzero(g) == 6
    assert np.isclose(loss, np.mean([np.log1p(np.exp(-5.0)), np.log1p(np.exp(-1.0))]))


def test_gradient_matches_finite_differences():
    """Central differences in float64 without rounding: every one of the
    5313 partial derivatives of the mean BCE loss."""
    rng = np.random.default_rng(11)
    flat = rng.standard_normal(mlp.N_PARAMS) * 0.3
    X = rng.standard_normal((24, 16))
    y = (rng.random(24) < 0.5).astype(np.float64)
    _, g = mlp.backward(flat, X, y, quant=False, dtype=np.float64)
    h = 1e-6
    fd = np.zeros_like(g)
    for t in range(mlp.N_PARAMS):
        e = np.zeros(mlp.N_PARAMS)
        e[t] = h
        lp = mlp.bce_loss(mlp.forward(flat + e, X, False, np.float64)[1]["z"], y)
        lm = mlp.bce_loss(mlp.forward(flat - e, X, False, np.float64)[1]["z"], y)
        fd[t] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    assert np.count_nonzero(g) > mlp.N_PARAMS // 2


def test_rounding_is_the_only_difference():
    """With weights and inputs that bf16 holds exactly and integer-valued
    hidden activations, the rounded and unrounded networks agree exactly."""
    rng = np.random.default_rng(2)
    flat = rng.integers(-1, 2, mlp.N_PARAMS).astype(np.float32)
    X = rng.integers(-3, 4, (16, 16)).astype(np.float32)
    y = (rng.random(16) < 0.5).astype(np.float32)
    s1, _ = mlp.forward(flat, X, True)
    s0, _ = mlp.forward(flat, X, False)
    assert np.array_equal(s1, s0)
    _, g1 = mlp.backward(flat, X, y, True)
    _, g0 = mlp.backward(flat, X, y, False)
    assert np.array_equal(g1, g0)
    # and rounding does change a generic network
    flat = _rand_params(rng)
    X = rng.standard_normal((16, 16)).astype(np.float32)
    assert not np.array_equal(mlp.forward(flat, X, True)[0], mlp.forward(flat, X, False)[0])


def test_adam_hand_step():
    p = np.array([1.0, -2.0, 0.5], np.float32)
    g = np.array([0.5, -4.0, 0.0], np.float32)
    m = np.zeros(3, np.float32)
    v = np.zeros(3, np.float32)
    p1, m1, v1 = mlp.adam_step(p, g, m, v, 1, lr=0.1)
    # first step: m_hat = g and v_hat = g^2, so the step is lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.1 * g / (np.abs(g) + 1e-8), atol=1e-6)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    p2, m2, v2 = mlp.adam_step(p1, g, m1, v1, 2, lr=0.1)
    mh = (0.9 * 0.1 * g + 0.1 * g) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g * g) / (1 - 0.999 ** 2)
    assert np.allclose(p2, p1 - 0.1 * mh / (np.sqrt(vh) + 1e-8), atol=1e-6)


def test_training_fits_a_separable_rule():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((512, 16)).astype(np.float32)
    w = rng.standard_normal(16).astype(np.float32)
    y = (X @ w > 0).astype(np.float32)
    flat = _rand_params(rng, 0.2)
    m = np.zeros_like(flat)
    v = np.zeros_like(flat)
    first = None
    for t in range(1, 301):
        loss, g = mlp.backward(flat, X, y)
        first = loss if first is None else first
        flat, m, v = mlp.adam_step(flat, g, m, v, t, lr=3e-3)
    s, _ = mlp.forward(flat, X)
    assert loss < 0.3 * first
    assert np.mean((s > 0.5) == (y > 0.5)) > 0.95
