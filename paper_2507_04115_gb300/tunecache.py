"""Persistent table of tuned launch shapes.

The autotuner (tdse_autotune) times launch shapes on a batch and keeps the fastest.  Its choice
depends only on the batch's grid classes and their instance counts, the precision, the scheme, the
lanes per instance and the GPU, so a shape found once can be reused by later runs of the same
kind of batch without timing again.  This module keeps such shapes in a JSON file:

    {"version": 1, "shapes": {<key>: {"warps_per_cta": W, "ctas_per_sm": C, "slice_steps": S}}}

Keys are canonical JSON strings of the quantities above.  Writes go to a temporary file in the
same directory that then replaces the table, so a reader never sees a partial file.  Host logic
only: applying a shape is one tdse_set_launch call, exactly what the autotuner does with its
fastest trial.
"""
from __future__ import annotations

import json
import os
import tempfile

SHAPE_FIELDS = ("warps_per_cta", "ctas_per_sm", "slice_steps")


def batch_key(classes, precision, scheme, lanes_per_instance, gpu_name) -> str:
    """Canonical key.  ``classes``: iterable of (N, dx, softening, charge, instance count); the order
    of the classes does not matter."""
    cls = sorted((int(N), float(dx), float(a), float(Z), int(c)) for N, dx, a, Z, c in classes)
    payload = {"classes": cls, "precision": int(precision), "scheme": int(scheme),
               "lanes": int(lanes_per_instance), "gpu": str(gpu_name)}
    return json.dumps(payload, sort_keys=True, separators=(",", ":"))


def key_of(batch, gpu_name) -> str:
    """Key of a ``tdse.Batch`` (its classes counted from the per-instance parameters)."""
    counts = {}
    for t in zip(batch.N.tolist(), batch.dx.tolist(), batch.softening.tolist(), batch.charge.tolist()):
        counts[t] = counts.get(t, 0) + 1
    return batch_key([k + (c,) for k, c in counts.items()], batch.precision, batch.scheme,
                     batch.lanes_per_instance, gpu_name)


class TuneCache:
    VERSION = 1

    def __init__(self, path: str):
        self.path = path
        self.table = {}
        if os.path.exists(path):
            with open(path) as fh:
                data = json.load(fh)
            if isinstance(data, dict) and data.get("version") == self.VERSION:
                self.table = {k: dict(v) for k, v in data.get("shapes", {}).items()}

    def get(self, key):
        shape = self.table.get(key)
        return None if shape is None else {f: int(shape[f]) for f in SHAPE_FIELDS}

    def put(self, key, shape):
        self.table[key] = {f: int(shape[f]) for f in SHAPE_FIELDS}
        self.save()

    def save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tunecache.", suffix=".tmp")
        try:
            with os.fdopen(fd, "w") as fh:
                json.dump({"version": self.VERSION, "shapes": self.table}, fh, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def tune(batch, E, d, a, cache: TuneCache, key: str, **autotune_kw):
    """Apply the cached shape for ``key`` to ``batch``, or run ``batch.autotune`` and store its
    fastest trial.  Returns (shape, trials); trials is empty on a cache hit."""
    hit = cache.get(key)
    if hit is not None:
        batch.set_launch(**hit)
        return hit, []
    trials = batch.autotune(E, d, a, **autotune_kw)
    best = min(trials, key=lambda t: t["ms"])
    shape = {f: int(best[f]) for f in SHAPE_FIELDS}
    cache.put(key, shape)
    return shape, trials
