"""Parity of the learned pair scheduler's kernels with the CPU oracle
(oracle/mlp.py): pair features, the bf16 tensor-core forward pass, the fp32
gradient, Adam training replayed from a CUDA graph, and the k x k score
table.  Scores and gradients within 1e-3."""
import numpy as np
import pytest

import synth
from oracle import max_block_weight
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_01556_gb300 import hfp
    hfp.load()
    return torch, hfp, hfp.ctx_create(0)


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(mlp.N_PARAMS) * scale).astype(np.float32)


def _kway(env, seed, n, m, k):
    torch, hfp, ctx = env
    inst = synth.instance("ring_n8M_zipf_k64", seed, n=n, m=m)
    H = inst["H"]
    part = inst["part"] if k == 64 else synth.kway_partition(n, k, 50_000, seed)
    hg = hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n)
    return H, part, hg, torch.from_numpy(part.copy()).cuda()


@pytest.mark.parametrize("seed,n,m,k", [(1, 20000, 30000, 64), (2, 50000, 75000, 8),
                                        (3, 4000, 6000, 2)])
def test_pair_features_match_oracle(env, seed, n, m, k):
    torch, hfp, ctx = env
    H, part, hg, pd = _kway(env, seed, n, m, k)
    rng = np.random.default_rng(seed)
    prev = np.where(rng.random((k, k)) < 0.5, rng.integers(0, 50, (k, k)), -1).astype(np.int64)
    L = max_block_weight(int(H.node_w.sum()), k, 3)
    for pg in (None, prev):
        op, ox = mlp.pair_features(H, part, k, L, pg)
        gp, gx = hfp.pair_features(hg, pd, k, 3, pg)
        assert np.array_equal(gp.cpu().numpy(), op)
        np.testing.assert_allclose(gx.cpu().numpy(), ox, rtol=2e-6, atol=1e-7)


@pytest.mark.parametrize("rows", [1, 15, 64, 777, 2016, 50_001])
def test_forward_matches_oracle(env, rows):
    torch, hfp, ctx = env
    rng = np.random.default_rng(rows)
    X = (rng.standard_normal((rows, 16)) * 2).astype(np.float32)
    flat = _params(rows)
    s = hfp.mlp_forward(ctx, torch.from_numpy(flat).cuda(), torch.from_numpy(X).cuda())
    o, _ = mlp.forward(flat, X)
    assert np.max(np.abs(s.cpu().numpy() - o)) < 1e-3


def test_forward_empty(env):
    torch, hfp, ctx = env
    s = hfp.mlp_forward(ctx, torch.zeros(mlp.N_PARAMS).cuda(), torch.zeros((0, 16)).cuda())
    assert s.numel() == 0


@pytest.mark.parametrize("rows", [1, 63, 64, 1000, 4097])
def test_gradient_matches_oracle(env, rows):
    torch, hfp, ctx = env
    rng = np.random.default_rng(100 + rows)
    X = rng.standard_normal((rows, 16)).astype(np.float32)
    y = (rng.random(rows) < 0.4).astype(np.float32)
    flat = _params(200 + rows)
    loss, g = hfp.mlp_grad(ctx, torch.from_numpy(flat).cuda(), torch.from_numpy(X).cuda(),
                           torch.from_numpy(y).cuda())
    ol, og = mlp.backward(flat, X, y)
    g = g.cpu().numpy()
    assert abs(loss - ol) < 1e-3
    scale = max(1.0, float(np.max(np.abs(og))))
    assert np.max(np.abs(g - og)) < 1e-3 * scale
    # the gradient is not trivially small
    assert np.max(np.abs(og)) > 1e-3


def test_training_matches_oracle(env):
    torch, hfp, ctx = env
    rng = np.random.default_rng(7)
    rows = 3000
    X = rng.standard_normal((rows, 16)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 3] - X[:, 7] > 0).astype(np.float32)
    flat = _params(8, 0.2)
    st = hfp.MlpState(torch.from_numpy(flat.copy()).cuda())
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    losses = hfp.mlp_train(ctx, st, xd, yd, 10, lr=2e-3).cpu().numpy()
    losses = np.concatenate([losses, hfp.mlp_train(ctx, st, xd, yd, 15, lr=2e-3).cpu().numpy()])
    assert int(st.step.item()) == 25
    p, m, v = flat.copy(), np.zeros_like(flat), np.zeros_like(flat)
    ol = []
    for t in range(1, 26):
        loss, g = mlp.backward(p, X, y)
        ol.append(loss)
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=2e-3)
    np.testing.assert_allclose(losses, ol, atol=1e-3)
    assert np.max(np.abs(st.params.cpu().numpy() - p)) < 1e-3
    assert ol[-1] < ol[0]


def test_pair_scores_table(env):
    torch, hfp, ctx = env
    H, part, hg, pd = _kway(env, 4, 20000, 30000, 64)
    flat = _params(9)
    pdev = torch.from_numpy(flat).cuda()
    table = hfp.pair_scores(hg, pd, 64, pdev)
    L = max_block_weight(int(H.node_w.sum()), 64, 3)
    op, ox = mlp.pair_features(H, part, 64, L)
    os_, _ = mlp.forward(flat, ox)
    exp = -np.ones((64, 64), np.float32)
    exp[op[:, 0], op[:, 1]] = os_
    assert np.max(np.abs(table - exp)) < 1e-3
    assert np.all(table[exp < 0] == -1)
