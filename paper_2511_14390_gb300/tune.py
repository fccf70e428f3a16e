"""Measured tuner of the decoupled chunked path's launch shape, with a JSON cache.

The chunk-state scan of state buckets 8..64 has two free parameters the paper leaves
open (its batches are uniform and its scan is a library call): the span length (tiles of
8192 samples per scan span; a longer channel is cut into spans scanned by different CTAs
and joined by the look-back) and the number of scan chains (CTAs) per SM.  Shorter spans
cost rescans, longer spans lengthen the longest chain; more chains keep the FP32 pipes
busier but slow each one.  The best pair depends on the batch shape, so it is measured:

    tune(step, buckets)    time `step` for every candidate pair of each bucket in turn
                           (coordinate descent over the buckets), install the best pair
                           with dfilt_tuning_set, and return the table.

The choice is deterministic given the measurements (ties go to the shorter span, then to
fewer chains).  Results are cached in a JSON file keyed by the device, the state bucket
and the batch's shape classes (log2 buckets of channel count, mean channel length and
samples), and the operand precision; `lookup` installs a cached table.
"""
from __future__ import annotations

import json
import math
import os

from . import dfilt

SPANS = (1, 2, 4, 8, 16, 32, 64)
CHAINS = {8: (8, 16, 32), 16: (8, 16, 32), 32: (4, 8, 16), 64: (2, 4, 8)}
CACHE_ENV = "DFILT_TUNE_CACHE"


def cache_path() -> str:
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                     "_tune_cache.json")


def shape_key(device: str, mb: int, B: int, total: int, precision: str = "tf32x3") -> str:
    """Cache key: device, state bucket, log2 classes of channels, mean length, samples."""
    lg = lambda v: int(math.floor(math.log2(max(1, v))))
    return f"{device}|MB{mb}|B{lg(B)}|T{lg(total // max(1, B))}|S{lg(total)}|{precision}"


def choose(times: dict) -> tuple:
    """The fastest (span, chains) of a {(span, chains): ms} table; ties broken toward the
    shorter span, then toward fewer chains (the order of the candidates does not matter)."""
    if not times:
        raise ValueError("no measurements")
    return min(times, key=lambda k: (times[k], k[0], k[1]))


def tune(step, buckets, timer, *, spans=SPANS, chains=None):
    """Coordinate descent over the state buckets present: for each bucket in turn, every
    (span, chains) candidate is installed and `timer(step)` (ms, lower is better) taken;
    the best is kept installed before the next bucket.  Returns {mb: (span, chains, ms)}
    and the full measurements."""
    chains = chains or CHAINS
    table, seen = {}, {}
    for mb in buckets:
        times = {}
        for s in spans:
            for c in chains.get(mb, (0,)):
                dfilt.dfilt_tuning_set(mb, s, c)
                times[(s, c)] = float(timer(step))
        best = choose(times)
        dfilt.dfilt_tuning_set(mb, *best)
        table[mb] = (best[0], best[1], times[best])
        seen[mb] = times
    return table, seen


def save(entries: dict, path: str | None = None):
    """Merge {key: {"span_tiles": s, "chains_per_sm": c, "ms": t}} into the cache file."""
    path = path or cache_path()
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data.update(entries)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(keys: dict, path: str | None = None) -> dict:
    """Install the cached pair of each {mb: key} found in the cache; returns the hits."""
    path = path or cache_path()
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    hits = {}
    for mb, key in keys.items():
        e = data.get(key)
        if e:
            dfilt.dfilt_tuning_set(mb, int(e["span_tiles"]), int(e["chains_per_sm"]))
            hits[mb] = e
    return hits


def reset(buckets=(8, 16, 32, 64)):
    """Back to the built-in rule for the given buckets."""
    for mb in buckets:
        dfilt.dfilt_tuning_set(mb, 0, 0)
