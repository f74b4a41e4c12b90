"""Host logic of the autotuner (no GPU): size and density classes, the
one-parameter-at-a-time search and the JSON cache."""
from __future__ import annotations

from paper_1607_00908_gb300 import autotune


class FakeBatch:
    """Stands in for vd.Batch: push costs depend on the tuning."""

    def __init__(self, sizes, bubbles, cost):
        self.sizes = sizes
        self._bubbles = bubbles
        self.cost = cost
        self.t = dict(autotune.DEFAULT, graph_blocks=1)
        self.sets = 0

    def push(self, fields):
        pass

    def counts(self, i):
        return self._bubbles[i], 0, 0

    def set_tuning(self, voronoi_patch, bucket_pct, ring0, graph_blocks=None):
        gb = self.t["graph_blocks"] if graph_blocks is None else graph_blocks
        self.t = dict(voronoi_patch=voronoi_patch, bucket_pct=bucket_pct, ring0=ring0, graph_blocks=gb)
        self.sets += 1

    def tuning(self):
        return dict(self.t)


def _fake_time(b, fields, stream, reps):
    return b.cost(b.t)


def test_keys_class_size_and_density():
    assert autotune.key_of([(1024, 1024)], [1024]) == "L20_s10"
    assert autotune.key_of([(256, 256), (2048, 2048)], [100, 2000]) == autotune.key_of([(2048, 2048), (256, 256)],
                                                                                      [2000, 100])
    assert autotune.key_of([(4096, 4096)], [30000]) != autotune.key_of([(4096, 4096)], [3000])


def test_search_finds_the_separable_minimum_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setenv("VD_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    monkeypatch.setattr(autotune, "_time_push", _fake_time)

    def cost(t):   # best: grid-wide graph stage, 16x16 patches, buckets at 70 %, first reach 0
        return (abs(t["voronoi_patch"] - 3) + abs(t["bucket_pct"] - 70) / 10 + t["ring0"] / 9 + 1.0 +
                t["graph_blocks"])

    b = FakeBatch([(512, 512)], [300], cost)
    r = autotune.tune(b, None, None)
    assert (r["voronoi_patch"], r["bucket_pct"], r["ring0"], r["graph_blocks"]) == (3, 70, 0, 0)
    assert not r["cached"] and r["tuned_ms"] < r["default_ms"]
    assert b.t == dict(voronoi_patch=3, bucket_pct=70, ring0=0, graph_blocks=0)
    # the second batch of the same classes takes the cached choice without timing
    b2 = FakeBatch([(512, 512)], [310], lambda t: 1 / 0)
    r2 = autotune.tune(b2, None, None)
    assert r2["cached"] and b2.t == dict(voronoi_patch=3, bucket_pct=70, ring0=0, graph_blocks=0)


def test_default_kept_when_nothing_is_faster(tmp_path, monkeypatch):
    monkeypatch.setenv("VD_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(autotune, "_time_push", _fake_time)
    b = FakeBatch([(128, 128)], [30], lambda t: 1.0 if t == autotune.DEFAULT else 2.0)
    r = autotune.tune(b, None, None, use_cache=False)
    assert {k: r[k] for k in autotune.DEFAULT} == autotune.DEFAULT
    assert not (tmp_path / "c.json").exists()
