"""Host logic of the batched smoother's tile autotuner (paper_1208_2643_gb300/tuning.py),
on the CPU with a stand-in batch: the level count of an instance, the level keys, the
choice of the fastest candidate and the cache."""
import json

import pytest

from paper_1208_2643_gb300 import tuning


class _P:
    def __init__(self, m, n, coarsest=4):
        self.m, self.n, self.coarsest = m, n, coarsest


class _FakeBatch:
    """Instances of the given sizes; a sweep's time is a fixed function of the tile and
    the level, so the best tile of each level is known."""

    def __init__(self, sizes, best):
        self.params = [_P(m, n) for m, n in sizes]
        self.count = len(sizes)
        self.levels = max(tuning._levels_of(p) for p in self.params)
        self.best = best            # level -> (tx, ty)
        self.tile = {}
        self.timed = 0

    def set_tile(self, level, tx, ty):
        self.tile[level] = (tx, ty)

    def time_smooth(self, scheme, level, reps=5):
        self.timed += 1
        tx, ty = self.tile[level]
        return 1.0 if (tx, ty) == self.best.get(level) else 2.0 + 0.01 * tx + 0.001 * ty


@pytest.mark.parametrize("m,n", [(4, 4), (6, 6), (8, 12), (64, 64), (96, 160), (512, 384), (1024, 1024)])
def test_levels_follow_the_coarsening_rule(oracle_mod, m, n):
    """Halve while both sides stay even and at least 4 cells: the same count as the
    oracle's hierarchy."""
    assert tuning._levels_of(_P(m, n)) == oracle_mod.num_levels(m, n, 4)


def test_level_keys_align_instances_at_the_coarse_end():
    b = _FakeBatch([(64, 64), (128, 128)], {})
    # 128^2 has one level more; at aligned level 0 only it takes part
    assert tuning._level_key(b, 0) == "128x128"
    assert tuning._level_key(b, 1) == "64x64,64x64"


def test_autotune_picks_the_fastest_tile_and_caches_it(tmp_path, monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "FAKE GPU")
    sizes = [(64, 64), (128, 128)]
    levels = max(tuning._levels_of(_P(m, n)) for m, n in sizes)
    best = {lv: tuning.CANDIDATES[(3 * lv + 1) % len(tuning.CANDIDATES)] for lv in range(levels - 1)}
    b = _FakeBatch(sizes, best)
    cache = tmp_path / "tiles.json"
    chosen = tuning.autotune(b, scheme=2, cache_path=str(cache), reps=1)
    for level, (tx, ty, ms) in chosen.items():
        assert (tx, ty) == best[level] and ms == 1.0
        assert b.tile[level] == best[level]
    assert b.timed == len(chosen) * len(tuning.CANDIDATES)
    keys = json.load(open(cache))
    assert all(k.startswith("FAKE GPU|s2|") for k in keys)
    # a second batch of the same shape takes the cached tiles without timing
    b2 = _FakeBatch(sizes, best)
    chosen2 = tuning.autotune(b2, scheme=2, cache_path=str(cache), reps=1)
    assert b2.timed == 0 and chosen2 == {k: tuple(v) for k, v in chosen.items()}
