"""Launch-shape autotuner for the batched persistent form.

The batched form runs every solve of a batch in one persistent launch, so a
batch has one launch shape (threads per CTA, CTAs per SM).  Which shape is
fastest depends on the sizes of the solves: small grids favour several small
CTAs per SM, large ones one wide CTA.  The tuner therefore measures per side
bucket (bucket b holds the sides in [2^b, 2^(b+1))): for every bucket present
in a batch and every candidate shape it times a sample of that bucket's
solves, capped at a fixed iteration count, and records the time per row
iteration.  The shape for a batch is the one with the least predicted time,
the sum over its buckets of (time per row iteration) x (rows in the bucket).
Measurements are cached per (GPU, m, storage, bucket) in a JSON file
($AA_AUTOTUNE_CACHE, default: _autotune.json next to this module), so a
later batch with another size mix is served from the cache and only its new
buckets are timed.
"""
from __future__ import annotations

import json
import os

CANDIDATES = [(128, 2), (128, 4), (256, 1), (256, 2), (512, 1)]


def _cache_path() -> str:
    return os.environ.get("AA_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json"))


def _key(m: int) -> str:
    import torch
    return f"{torch.cuda.get_device_name()}|batch|m{m}|fp32"


def bucket_of(side: int) -> int:
    """Side bucket: b with 2^b <= side < 2^(b+1)."""
    return max(0, int(side).bit_length() - 1)


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(data: dict) -> None:
    try:
        with open(_cache_path(), "w") as f:
            json.dump(data, f, indent=1)
    except OSError:
        pass


def _shape_key(shape) -> str:
    return f"{shape[0]}x{shape[1]}"


def time_bucket(sides, lams, m: int, candidates, max_iters: int):
    """Time every candidate on these solves (every solve capped at max_iters);
    returns {shape: ms per row iteration}."""
    import numpy as np

    import paper_2110_09667_gb300 as aa
    B = aa.Batch(sides, lams, m=m, max_iters=max_iters)
    row_iters = float((np.asarray(sides, dtype=np.float64) ** 2).sum()) * max_iters
    out = {}
    for blk, cps in candidates:
        B.solve(blk, cps)  # capture + warm
        out[(blk, cps)] = B.solve(blk, cps) / row_iters
    B.close()
    return out


def tune_batch(sides, lams, m: int = 10, sample: int = 152, candidates=CANDIDATES,
               max_iters: int = 300, use_cache: bool = True):
    """Returns ((block, ctas_per_sm), {shape: predicted ms}) for the batch.
    Buckets missing from the cache (or all, with use_cache=False) are timed
    on up to `sample` of their solves, spread over the bucket's sizes; the
    prediction weights each bucket's time per row iteration by its rows."""
    import numpy as np
    sides = np.asarray(sides)
    lams = np.asarray(lams)
    key = _key(m)
    data = _load() if use_cache else {}
    entry = data.get(key, {})
    per_bucket = entry.get("buckets", {})
    buckets = sorted(set(bucket_of(s) for s in sides))
    for b in buckets:
        if use_cache and str(b) in per_bucket and all(_shape_key(c) in per_bucket[str(b)]
                                                     for c in candidates):
            continue
        idx = np.nonzero([bucket_of(s) == b for s in sides])[0]
        idx = idx[np.argsort(sides[idx], kind="stable")]
        pick = idx[np.linspace(0, len(idx) - 1, min(sample, len(idx))).round().astype(int)]
        pick = np.unique(pick)
        t = time_bucket(sides[pick], lams[pick], m, candidates, max_iters)
        per_bucket[str(b)] = {_shape_key(c): v for c, v in t.items()}
    rows = {b: float((sides[[bucket_of(s) == b for s in sides]].astype(np.float64) ** 2).sum())
            for b in buckets}
    predicted = {c: sum(per_bucket[str(b)][_shape_key(c)] * rows[b] for b in buckets)
                 for c in candidates}
    best = min(predicted, key=predicted.get)
    entry["buckets"] = per_bucket
    entry["last_shape"] = list(best)
    data[key] = entry
    _store(data)
    return best, predicted
