"""Host logic of the batched form's launch-shape autotuner (CPU; the batched
solver is replaced by a stand-in whose time per row iteration depends on the
launch shape and on the sides of the solves it is given).

Checked: solves are grouped into side buckets [2^b, 2^(b+1)); each bucket
present is timed on a sample spread over its sizes, with every candidate
shape; the shape for a batch minimises the rows-weighted sum of the buckets'
times; measurements are cached per (GPU, m, bucket), so a later batch is
served from the cache and only buckets never seen are timed.
"""
import json

import numpy as np
import pytest

import aa_synth
import paper_2110_09667_gb300 as aa
from paper_2110_09667_gb300 import autotune

# time per row iteration (arbitrary units): small grids favour many small
# CTAs, large grids one wide CTA
COST = {
    (128, 2): {5: 1.0, 6: 2.0, 7: 4.0, 8: 6.0},
    (128, 4): {5: 0.8, 6: 2.2, 7: 4.5, 8: 7.0},
    (256, 1): {5: 1.5, 6: 1.6, 7: 2.0, 8: 3.0},
    (256, 2): {5: 1.2, 6: 1.5, 7: 2.5, 8: 3.5},
    (512, 1): {5: 3.0, 6: 2.5, 7: 1.5, 8: 1.0},
}


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
        b = autotune.bucket_of(int(self.sides[0]))
        assert all(autotune.bucket_of(int(s)) == b for s in self.sides)  # one bucket per timing
        rows = float((self.sides.astype(np.float64) ** 2).sum())
        return COST[(block, ctas_per_sm)][b] * rows * self.max_iters

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


def test_buckets():
    assert [autotune.bucket_of(s) for s in (32, 63, 64, 127, 128, 255, 256)] == [5, 5, 6, 6, 7, 7, 8]


def test_per_bucket_timing_and_weighted_choice(tuner):
    sides, lams = aa_synth.bratu_batch(0, 4096)
    best, pred = autotune.tune_batch(sides, lams, m=10, sample=152, max_iters=300)
    buckets = sorted(set(autotune.bucket_of(s) for s in sides))
    assert len(FakeBatch.made) == len(buckets)
    for B in FakeBatch.made:
        assert B.m == 10 and B.max_iters == 300 and len(B.sides) <= 152
        # every candidate twice (capture + timed)
        assert sorted(B.calls) == sorted(autotune.CANDIDATES * 2)
        # the sample spans its bucket: its smallest and largest sides
        b = autotune.bucket_of(int(B.sides[0]))
        inb = np.asarray([s for s in sides if autotune.bucket_of(s) == b])
        assert B.sides.min() == inb.min() and B.sides.max() == inb.max()
    # the choice minimises sum over buckets of cost x rows
    rows = {b: float(sum(float(s) ** 2 for s in sides if autotune.bucket_of(s) == b))
            for b in buckets}
    want = {c: sum(COST[c][b] * rows[b] for b in buckets) for c in autotune.CANDIDATES}
    assert best == min(want, key=want.get)
    for c in autotune.CANDIDATES:
        assert pred[c] == pytest.approx(want[c])
    # the batch's rows sit mostly in the large buckets, so the wide CTA wins
    assert best == (512, 1)


def test_small_grids_choose_small_ctas(tuner):
    sides = np.array([32, 40, 47, 55, 63, 33, 36])
    best, _ = autotune.tune_batch(sides, np.linspace(1, 6, len(sides)), m=10)
    assert best == (128, 4)
    (B,) = FakeBatch.made
    assert sorted(B.sides) == sorted(sides)  # a small bucket is timed whole


def test_cache_per_bucket(tuner):
    small = np.array([40, 50, 60, 35])
    autotune.tune_batch(small, np.full(4, 3.0), m=10)
    assert len(FakeBatch.made) == 1
    data = json.loads(tuner.read_text())
    entry = data["TEST-GPU|batch|m10|fp32"]
    assert set(entry["buckets"]) == {"5"}
    assert entry["buckets"]["5"]["128x4"] == pytest.approx(0.8)
    # a mixed batch: bucket 5 from the cache, only bucket 7 timed
    FakeBatch.made.clear()
    mixed = np.array([40, 50, 200, 150])
    best, _ = autotune.tune_batch(mixed, np.full(4, 3.0), m=10)
    assert len(FakeBatch.made) == 1
    assert all(autotune.bucket_of(int(s)) == 7 for s in FakeBatch.made[0].sides)
    assert set(json.loads(tuner.read_text())["TEST-GPU|batch|m10|fp32"]["buckets"]) == {"5", "7"}
    # served entirely from the cache the second time
    FakeBatch.made.clear()
    again, _ = autotune.tune_batch(mixed, np.full(4, 3.0), m=10)
    assert again == best and FakeBatch.made == []
    # another history depth is tuned separately
    autotune.tune_batch(small, np.full(4, 3.0), m=5)
    assert len(FakeBatch.made) == 1
    assert set(json.loads(tuner.read_text())) == {"TEST-GPU|batch|m10|fp32", "TEST-GPU|batch|m5|fp32"}
