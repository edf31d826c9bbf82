"""What the learned scheduler gains: trained on the GPU (hfp_mlp_train) from
the outcomes of unpruned rounds on seeded k-way instances, then used to
prune pairs on held-out seeds.  The pruned schedule refines clearly fewer
block pairs and ends within 0.5 % of the unpruned schedule's (lambda - 1)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N = 60_000


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_01556_gb300 import hfp, scheduler
    hfp.load()
    return torch, hfp, scheduler, hfp.ctx_create(0)


def _inst(hfp, ctx, seed, k):
    inst = synth.instance("ring_n8M_zipf_k64", seed, n=N, m=N * 3 // 2)
    H = inst["H"]
    part = synth.kway_partition(N, k, 50_000, seed)
    return hfp.HGraph(ctx, H.net_off, H.pins, H.net_w, H.node_w, H.n), part


def test_learned_schedule_prunes_pairs_at_equal_quality(env):
    torch, hfp, scheduler, ctx = env
    S = scheduler.Samples()
    for seed in range(1, 5):
        for k in (16, 32):
            hg, part = _inst(hfp, ctx, seed, k)
            scheduler.collect(hg, torch.from_numpy(part).cuda(), k, rounds=6, samples=S)
    X, y, _ = S.arrays()
    assert 0.05 < y.mean() < 0.98          # both outcomes occur
    params, losses = scheduler.train(ctx, X, y, steps=2000, lr=3e-3)
    assert losses[-1] < 0.7 * losses[0]
    full_c = pruned_c = full_p = pruned_p = 0
    for seed in (1001, 1002):
        for k in (16, 32):
            hg, part = _inst(hfp, ctx, seed, k)
            f = scheduler.refine(hg, torch.from_numpy(part.copy()).cuda(), k, 10)
            p = scheduler.refine(hg, torch.from_numpy(part.copy()).cuda(), k, 10,
                                 mlp_params=params, threshold=0.5)
            full_c += f["connectivity"][-1]
            pruned_c += p["connectivity"][-1]
            full_p += f["pairs"]
            pruned_p += p["pairs"]
    assert pruned_c <= 1.005 * full_c
    assert pruned_p <= 0.95 * full_p
