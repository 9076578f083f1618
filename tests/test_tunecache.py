"""The tuned-shape table (tunecache.py), on the host: canonical keys, persistence, and the
hit/miss logic against a stand-in batch that records the calls a real one would receive."""
import json
import os

import numpy as np

from paper_2507_04115_gb300 import tunecache


def test_keys_are_canonical():
    a = tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 100), (2048, 0.2, 1.2, 1.0, 3)], 0, 0, 0, "GB300")
    b = tunecache.batch_key([(2048, 0.2, 1.2, 1.0, 3), (4096, 0.15, 1.19, 1.0, 100)], 0, 0, 0, "GB300")
    assert a == b
    assert a != tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 101), (2048, 0.2, 1.2, 1.0, 3)], 0, 0, 0, "GB300")
    assert a != tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 100), (2048, 0.2, 1.2, 1.0, 3)], 1, 0, 0, "GB300")
    assert a != tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 100), (2048, 0.2, 1.2, 1.0, 3)], 0, 1, 0, "GB300")
    assert a != tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 100), (2048, 0.2, 1.2, 1.0, 3)], 0, 0, 8, "GB300")
    assert a != tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 100), (2048, 0.2, 1.2, 1.0, 3)], 0, 0, 0, "B200")


class _FakeBatch:
    """What tunecache touches on a tdse.Batch: its parameters, autotune and set_launch."""

    def __init__(self):
        self.N = np.array([4096, 4096, 2048])
        self.dx = np.array([0.15, 0.15, 0.2])
        self.softening = np.array([1.19, 1.19, 1.2])
        self.charge = np.ones(3)
        self.precision, self.scheme, self.lanes_per_instance = 0, 0, 0
        self.calls = []

    def autotune(self, E, d, a, **kw):
        self.calls.append(("autotune", kw))
        return [dict(warps_per_cta=8, ctas_per_sm=1, slice_steps=16, ctas=152, ms=3.0),
                dict(warps_per_cta=12, ctas_per_sm=1, slice_steps=16, ctas=152, ms=2.5),
                dict(warps_per_cta=6, ctas_per_sm=2, slice_steps=32, ctas=304, ms=2.7)]

    def set_launch(self, **shape):
        self.calls.append(("set_launch", shape))


def test_miss_then_hit_and_persistence(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    b = _FakeBatch()
    key = tunecache.key_of(b, "GB300")
    assert key == tunecache.batch_key([(4096, 0.15, 1.19, 1.0, 2), (2048, 0.2, 1.2, 1.0, 1)], 0, 0, 0, "GB300")
    cache = tunecache.TuneCache(path)
    shape, trials = tunecache.tune(b, None, None, None, cache, key, repeats=2)
    assert shape == dict(warps_per_cta=12, ctas_per_sm=1, slice_steps=16) and len(trials) == 3
    assert b.calls == [("autotune", {"repeats": 2})]
    # a new process reads the table back and applies the shape without timing
    b2 = _FakeBatch()
    shape2, trials2 = tunecache.tune(b2, None, None, None, tunecache.TuneCache(path), key)
    assert shape2 == shape and trials2 == []
    assert b2.calls == [("set_launch", shape)]
    with open(path) as fh:
        data = json.load(fh)
    assert data["version"] == 1 and data["shapes"][key] == shape
    assert [f for f in os.listdir(tmp_path / "sub") if f.endswith(".tmp")] == []


def test_other_versions_and_keys_are_ignored(tmp_path):
    path = str(tmp_path / "tune.json")
    with open(path, "w") as fh:
        json.dump({"version": 0, "shapes": {"k": {"warps_per_cta": 4, "ctas_per_sm": 1, "slice_steps": 8}}}, fh)
    cache = tunecache.TuneCache(path)
    assert cache.get("k") is None
    cache.put("k2", dict(warps_per_cta=4, ctas_per_sm=2, slice_steps=8, ms=1.0))
    assert tunecache.TuneCache(path).get("k2") == dict(warps_per_cta=4, ctas_per_sm=2, slice_steps=8)
    assert tunecache.TuneCache(path).get("k") is None
