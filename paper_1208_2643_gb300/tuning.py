"""Tile-shape autotuner of the batched smoother.

For every aligned level of a batch it times the red-black sweep with each candidate
thread-tile shape (mpfc_batch_time_smooth) and keeps the fastest, caching the choice
in a JSON file keyed by the GPU name, the scheme and the level's instance sizes, so
later batches of the same shape skip the timing.
"""
from __future__ import annotations

import json
import os

CANDIDATES = [(32, 8), (64, 4), (16, 16), (128, 2), (32, 4), (64, 2), (32, 16)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tiles.json")


def _level_key(batch, level):
    sizes = []
    L = batch.levels
    for i in range(batch.count):
        p = batch.params[i]
        from . import mpfc  # noqa: F401
        # instance i joins the aligned hierarchy at L - levels(i); its level there:
        li = level - (L - _levels_of(p))
        if li >= 0:
            sizes.append(f"{p.m >> li}x{p.n >> li}")
    return ",".join(sorted(sizes))


def _levels_of(p):
    L, m, n = 1, p.m, p.n
    while m % 2 == 0 and n % 2 == 0 and m // 2 >= p.coarsest and n // 2 >= p.coarsest and (m // 2) % 2 == 0 \
            and (n // 2) % 2 == 0 and L < 16:
        m //= 2
        n //= 2
        L += 1
    return L


def autotune(batch, scheme=1, cache_path=DEFAULT_CACHE, reps=5, use_cache=True):
    """Chooses the smoother tile of every level of `batch`; returns {level: (tx, ty, ms)}."""
    import torch
    gpu = torch.cuda.get_device_name()
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    chosen = {}
    for level in range(batch.levels - 1):
        key = f"{gpu}|s{scheme}|{_level_key(batch, level)}"
        if not _level_key(batch, level):
            continue
        if key in cache:
            tx, ty, ms = cache[key]
            batch.set_tile(level, tx, ty)
            chosen[level] = (tx, ty, ms)
            continue
        best = None
        for tx, ty in CANDIDATES:
            batch.set_tile(level, tx, ty)
            ms = batch.time_smooth(scheme, level, reps)
            if best is None or ms < best[2]:
                best = (tx, ty, ms)
        batch.set_tile(level, best[0], best[1])
        chosen[level] = best
        cache[key] = list(best)
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    with open(cache_path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return chosen
