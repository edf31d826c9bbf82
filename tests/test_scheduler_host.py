"""Host logic of the learned scheduler (paper_2201_01556_gb300.scheduler) on
CPU, with the library calls replaced by a scripted stand-in: the unpruned
fallback after a pruned round without gain, stopping at a round without
gain, the previous-round gain table, and the labels collect() records."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_01556_gb300 import hfp, scheduler  # noqa: E402


class Script:
    """refine_round_batched answers from a list of (gain, pairs, skipped)
    per call; records whether each call was pruned."""

    def __init__(self, rounds, k=4):
        self.rounds = list(rounds)
        self.calls = []
        self.k = k

    def refine_round_batched(self, hg, part, k, params, pair_scores=None, min_score=0.0):
        gain, pairs, skipped = self.rounds.pop(0)
        pruned = pair_scores is not None
        self.calls.append(pruned)
        st = types.SimpleNamespace(gain=gain, pairs=pairs, pairs_skipped=skipped if pruned else 0,
                                   connectivity_after=1000 - 10 * len(self.calls))
        res = [types.SimpleNamespace(bi=0, bj=1, gain=gain, applied=1 if gain > 0 else 0,
                                     status=hfp.OK, delta_exp=gain, pins=100 + gain)]
        return st, res, 1.0

    def pair_scores(self, hg, part, k, params, eps_pct, prev):
        self.prev_seen = prev
        return np.zeros((k, k), np.float32)


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    def install(rounds):
        s = Script(rounds)
        monkeypatch.setattr(scheduler.hfp, "refine_round_batched", s.refine_round_batched)
        monkeypatch.setattr(scheduler.hfp, "pair_scores", s.pair_scores)
        return s
    return install


def test_unpruned_rounds_stop_at_the_first_round_without_gain(fake):
    s = fake([(5, 3, 0), (2, 3, 0), (0, 3, 0), (9, 3, 0)])
    out = scheduler.refine(None, None, 4, rounds=10, params=hfp.refine_params())
    assert s.calls == [False, False, False]
    assert out["pairs"] == 9 and out["skipped"] == 0 and out["fallbacks"] == 0
    assert len(out["connectivity"]) == 3


def test_pruned_round_without_gain_is_repeated_unpruned(fake):
    # pruned: gain 4; pruned: no gain with skipped pairs -> unpruned rerun
    # finds 3; pruned: no gain -> unpruned rerun finds none -> stop
    s = fake([(4, 2, 1), (0, 2, 1), (3, 3, 0), (0, 2, 1), (0, 3, 0), (7, 3, 0)])
    out = scheduler.refine(None, None, 4, rounds=10, params=hfp.refine_params(),
                           mlp_params=np.zeros(hfp.MLP_PARAMS, np.float32))
    assert s.calls == [True, True, False, True, False]
    assert out["fallbacks"] == 2
    assert out["pairs"] == 2 + 2 + 3 + 2 + 3 and out["skipped"] == 3
    assert len(out["connectivity"]) == 3
    # the scores of a round see the previous round's applied gains
    assert s.prev_seen[0, 1] == 3


def test_pruned_round_with_nothing_skipped_is_not_repeated(fake):
    s = fake([(0, 3, 0)])
    out = scheduler.refine(None, None, 4, rounds=5, params=hfp.refine_params(),
                           mlp_params=np.zeros(hfp.MLP_PARAMS, np.float32))
    assert s.calls == [True] and out["fallbacks"] == 0


def test_prev_table_marks_unrefined_pairs():
    res = [types.SimpleNamespace(bi=0, bj=2, gain=5, applied=1),
           types.SimpleNamespace(bi=1, bj=3, gain=-2, applied=0)]
    prev = scheduler._prev_from(res, 4)
    assert prev[0, 2] == 5 and prev[1, 3] == 0
    assert (prev[np.triu_indices(4, 1)] == -1).sum() == 4


def test_collect_labels_improving_pairs(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    pairs = np.array([[0, 1], [0, 2], [1, 2]], np.int32)
    feats = np.arange(3 * 16, dtype=np.float32).reshape(3, 16)
    monkeypatch.setattr(scheduler.hfp, "pair_features",
                        lambda hg, part, k, eps, prev: (torch.from_numpy(pairs),
                                                        torch.from_numpy(feats)))
    res = [types.SimpleNamespace(bi=0, bj=1, status=hfp.OK, delta_exp=4, pins=10, gain=4,
                                 applied=1),
           types.SimpleNamespace(bi=0, bj=2, status=hfp.OK, delta_exp=0, pins=20, gain=0,
                                 applied=0),
           types.SimpleNamespace(bi=1, bj=2, status=hfp.NO_BALANCED_CUT, delta_exp=9, pins=30,
                                 gain=0, applied=0)]
    st = types.SimpleNamespace(gain=4)
    monkeypatch.setattr(scheduler.hfp, "refine_round_batched",
                        lambda *a, **k: (st, res, 1.0))
    s = scheduler.collect(None, None, 3, rounds=2, params=hfp.refine_params())
    x, y, pins = s.arrays()
    assert x.shape == (6, 16) and np.array_equal(x[:3], feats)
    assert y.tolist() == [1, 0, 0, 1, 0, 0]
    assert pins.tolist() == [10, 20, 30, 10, 20, 30]


def test_active_blocks_and_scores():
    """Active block scheduling (Section 5): a block is active after an
    applied move set with positive gain on one of its pairs; the next round's
    scores select exactly the pairs with an active block."""
    R = types.SimpleNamespace
    res = [R(bi=0, bj=1, gain=5, applied=1), R(bi=2, bj=3, gain=0, applied=1),
           R(bi=1, bj=4, gain=7, applied=0), R(bi=3, bj=5, gain=2, applied=1)]
    act = scheduler.active_blocks(res, 6)
    assert act.tolist() == [True, True, False, True, False, True]
    sc = scheduler.active_scores(act)
    for i in range(6):
        for j in range(6):
            assert (sc[i, j] > 0.5) == (act[i] or act[j])


def test_refine_active_stops_without_active_blocks(monkeypatch):
    """The first round refines every pair; later rounds are pruned to active
    blocks; refinement stops once a round activates no block, or improves
    (lambda - 1) by less than the relative threshold."""
    calls = []

    def fake_round(hg, part, k, params, pair_scores=None, min_score=0.0):
        calls.append(None if pair_scores is None else pair_scores.copy())
        n = len(calls)
        gain = {1: 50, 2: 20, 3: 0}[n]
        st = types.SimpleNamespace(gain=gain, pairs=3, pairs_skipped=0 if n == 1 else 2,
                                   connectivity_before=1000, connectivity_after=1000 - gain)
        res = [types.SimpleNamespace(bi=n - 1, bj=n, gain=gain, applied=1 if gain else 0)]
        return st, res, 1.0

    monkeypatch.setattr(hfp, "refine_round_batched", fake_round)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    r = scheduler.refine_active(None, None, 4, rounds=10, min_rel_gain=0.0)
    assert calls[0] is None
    assert calls[1][0, 1] == 1.0 and calls[1][2, 3] == 0.0
    assert calls[2][1, 2] == 1.0 and calls[2][0, 3] == 0.0
    assert r["connectivity"] == [950, 980, 1000] and len(calls) == 3
    calls.clear()
    r = scheduler.refine_active(None, None, 4, rounds=10, min_rel_gain=0.03)
    assert len(calls) == 2   # the second round gains 2 % < 3 %
