"""Autotuner for the launch parameters libadcomb exposes.

* batched hist -> scan -> sum: work-item size (``chunk``), shared-memory
  table size (``smem_bins``) and elements per thread and step (``items``) of
  the persistent histogram launch;
* reduce_by_index (single call): the forward strategy -- per-thread tables,
  per-warp copies, one block-wide table, global atomics, or partitioning by bin
  range into shared-memory-sized buckets
  (``adc_debug_force_hist_strategy``; the library validates that the table fits);
* scan (single call): items per thread and tile shape -- 64 contiguous bytes
  per thread and tile, or 16 bytes (a warp's load then covers 512 contiguous
  bytes), each with the range-partitioned engine at several tiles per range;
  the per-tile look-back engine; and one tile per block staged in shared
  memory by bulk copies (``adc_debug_set_scan_engine``,
  ``adc_debug_set_scan_range_tiles``).

Each candidate is timed with CUDA events on the real inputs (warm-up, then the
mean of a few runs); the winner is cached in a JSON file keyed by the shape
bucket, so later calls with a similar shape reuse it without measuring.
Cache file: ``$ADC_AUTOTUNE_CACHE`` or ``~/.cache/adcomb_autotune.json``.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import adcomb

_lock = threading.Lock()
_cache = None

BATCHED_CHUNKS = (1 << 14, 1 << 16, 1 << 18)
BATCHED_SMEM_BINS = (4096, 8192, 16384)
BATCHED_ITEMS = (1, 4, 8)
HIST_STRATEGIES = (3, 0, 1, 2, 4, 5, 6, 7)  # per-thread, per-warp, per-block, global, partitioned, split,
                                          # cluster, two passes
# scan candidates (engine, tiles per range): 64-byte items with the automatic
# choice and with ranges of 16 / 32 tiles; the per-tile engine; 16-byte items
# with the default and 32-tile ranges; one TMA-staged tile per block
SCAN_CANDIDATES = ((0, 0), (2, 16), (2, 32), (1, 0), (5, 0), (5, 32), (4, 0))


def cache_path():
    return os.environ.get("ADC_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                             "adcomb_autotune.json"))


def _load():
    global _cache
    if _cache is None:
        try:
            with open(cache_path()) as f:
                _cache = json.load(f)
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _store():
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(_cache, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # a read-only home: the in-memory cache still serves this process


def _bucket(x):
    return int(round(math.log2(max(int(x), 1))))


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def batched_key(desc):
    dev = torch.cuda.get_device_name()
    return (f"batched|{dev}|count={_bucket(len(desc))}|n={_bucket(desc['n'].sum())}|"
            f"mmean={_bucket(desc['m'].mean())}")


def tune_batched(problem, force=False):
    """Chooses (chunk, smem_bins, items) for a BatchedHistScan and applies them
    (items -- elements per thread and step -- is a library-wide setting)."""
    key = batched_key(problem.desc_h)
    with _lock:
        hit = _load().get(key)
    if hit is not None and not force and "items" in hit:
        problem.smem_bins = hit["smem_bins"]
        adcomb.debug_set_batched_items(hit["items"])
        if hit["chunk"] != problem.chunk:
            problem.set_plan(hit["chunk"])
        return hit
    best = None
    results = []
    for chunk in BATCHED_CHUNKS:
        problem.set_plan(chunk)
        for sb in BATCHED_SMEM_BINS:
            problem.smem_bins = sb
            for items in BATCHED_ITEMS:
                adcomb.debug_set_batched_items(items)
                ms = _time(lambda: (problem.forward(), problem.backward()))
                results.append({"chunk": chunk, "smem_bins": sb, "items": items, "ms": ms})
                if best is None or ms < best["ms"]:
                    best = results[-1]
    problem.set_plan(best["chunk"])
    problem.smem_bins = best["smem_bins"]
    adcomb.debug_set_batched_items(best["items"])
    entry = dict(best, candidates=results)
    with _lock:
        _load()[key] = entry
        _store()
    return entry


def hist_key(op, dtype, n, m):
    return f"hist|{torch.cuda.get_device_name()}|{op}|{dtype}|n={_bucket(n)}|m={_bucket(m)}"


def tune_hist(op, m, keys, vals, force=False):
    """Chooses the forward strategy for reduce_by_index(op) at this shape; returns it
    and leaves it selected in the library (-1 restores the built-in choice)."""
    key = hist_key(op, vals.dtype, keys.shape[0], m)
    with _lock:
        hit = _load().get(key)
    if hit is not None and not force:
        adcomb.debug_force_hist_strategy(hit["strategy"])
        return hit
    hist, saved = adcomb.hist_fwd(op, m, keys, vals)
    results = []
    for s in HIST_STRATEGIES:
        adcomb.debug_force_hist_strategy(s)
        ms = _time(lambda: adcomb.hist_fwd(op, m, keys, vals, None, hist, saved))
        results.append({"strategy": s, "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    adcomb.debug_force_hist_strategy(best["strategy"])
    entry = dict(best, candidates=results)
    with _lock:
        _load()[key] = entry
        _store()
    return entry


def scan_key(op, dtype, n):
    return f"scan|{torch.cuda.get_device_name()}|{op}|{dtype}|n={_bucket(n)}"


def tune_scan(op, x, force=False):
    """Chooses the scan engine and tiles per range for scan(op) at x's shape,
    timing the forward and the vjp together; returns the choice and leaves it
    selected in the library (``apply_scan(None)`` restores the built-in one).
    Results never depend on the choice beyond rounding order."""
    key = scan_key(op, x.dtype, x.shape[0])
    with _lock:
        hit = _load().get(key)
    if hit is not None and not force:
        apply_scan(hit)
        return hit
    y = adcomb.scan_fwd(op, x)
    yb = torch.randn_like(x)
    xb = torch.empty_like(x)
    results = []
    for eng, rt in SCAN_CANDIDATES:
        apply_scan({"engine": eng, "range_tiles": rt})
        ms = _time(lambda: (adcomb.scan_fwd(op, x, y), adcomb.scan_vjp(op, x, y, yb, xbar=xb)))
        results.append({"engine": eng, "range_tiles": rt, "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    apply_scan(best)
    entry = dict(best, candidates=results)
    with _lock:
        _load()[key] = entry
        _store()
    return entry


def apply_scan(choice):
    """Selects a tuned scan configuration (None: the library's own choice)."""
    adcomb.debug_set_scan_engine(0 if choice is None else int(choice["engine"]))
    adcomb.debug_set_scan_range_tiles(0 if choice is None else int(choice["range_tiles"]))
