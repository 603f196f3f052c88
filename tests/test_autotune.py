"""Host logic of the batched form's launch-shape autotuner (CPU; the batched
solver is replaced by a stand-in that reports a fixed time per shape).

Checked: the timed sub-batch takes every k-th solve of the size-sorted batch
(so the largest and the smallest size classes are both timed), every
candidate shape is timed, the fastest one is returned and cached per
(GPU, m), and a second call is served from the cache without timing.
"""
import json

import numpy as np
import pytest

import aa_synth
import paper_2110_09667_gb300 as aa
from paper_2110_09667_gb300 import autotune


class FakeBatch:
    made = []

    def __init__(self, sides, lams, *, m=10, max_iters=100000, **kw):
        self.sides = np.asarray(sides)
        self.lams = np.asarray(lams)
        self.m, self.max_iters = m, max_iters
        self.calls = []
        FakeBatch.made.append(self)

    def solve(self, block, ctas_per_sm):
        self.calls.append((block, ctas_per_sm))
        # fixed cost per shape; (256, 2) is the fastest
        return {(128, 2): 9.0, (128, 4): 7.0, (256, 1): 6.0, (256, 2): 4.0,
                (512, 1): 5.0}[(block, ctas_per_sm)]

    def close(self):
        pass


@pytest.fixture
def tuner(monkeypatch, tmp_path):
    FakeBatch.made.clear()
    monkeypatch.setattr(aa, "Batch", FakeBatch)
    monkeypatch.setattr(autotune, "_key", lambda m: f"TEST-GPU|batch|m{m}|fp32")
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("AA_AUTOTUNE_CACHE", str(cache))
    return cache


def test_stratified_subbatch_and_best_shape(tuner):
    sides, lams = aa_synth.bratu_batch(0, 4096)
    best, times = autotune.tune_batch(sides, lams, m=10, sample=256, max_iters=300)
    assert best == (256, 2)
    assert set(times) == set(autotune.CANDIDATES)
    (B,) = FakeBatch.made
    assert B.m == 10 and B.max_iters == 300
    assert len(B.sides) == 256
    # every candidate is run twice (capture + timed)
    assert sorted(B.calls) == sorted(autotune.CANDIDATES * 2)
    # every 16th solve of the size-sorted batch: both ends of the size range
    s = np.sort(np.asarray(sides))
    assert B.sides.max() == s.max()
    assert B.sides.min() <= np.quantile(s, 1 / 256 + 1 / 16)
    # the picked sizes follow the batch's size distribution (quantiles within a class)
    for q in (0.1, 0.5, 0.9):
        assert abs(np.quantile(B.sides, q) - np.quantile(s, q)) <= 0.1 * np.quantile(s, q) + 2


def test_cache_round_trip(tuner):
    sides, lams = aa_synth.bratu_batch(1, 1000)
    best, _ = autotune.tune_batch(sides, lams, m=10, sample=100)
    data = json.loads(tuner.read_text())
    entry = data["TEST-GPU|batch|m10|fp32"]
    assert tuple(entry["shape"]) == best
    assert entry["ms"]["256x2"] == 4.0
    FakeBatch.made.clear()
    again, times = autotune.tune_batch(sides, lams, m=10, sample=100)
    assert again == best and times == {} and FakeBatch.made == []
    # another history depth is tuned separately
    other, _ = autotune.tune_batch(sides, lams, m=5, sample=100)
    assert other == (256, 2) and len(FakeBatch.made) == 1
    assert set(json.loads(tuner.read_text())) == {"TEST-GPU|batch|m10|fp32",
                                                   "TEST-GPU|batch|m5|fp32"}


def test_small_batch_is_timed_whole(tuner):
    sides = np.array([40, 33, 250, 90, 120])
    lams = np.linspace(1, 6, 5)
    autotune.tune_batch(sides, lams, m=10, sample=256)
    (B,) = FakeBatch.made
    assert sorted(B.sides) == sorted(sides)
