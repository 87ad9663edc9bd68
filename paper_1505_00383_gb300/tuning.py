"""A JSON cache of the tracker's tuned launch shape.

``ht_tune_track`` times every candidate launch shape (team warps x Newton
rounds per launch) on a sample of paths and keeps the fastest in the system
object.  This module remembers that choice across processes, keyed by what
it depends on: the number of variables, the number of terms, the largest
degree, the precision, whether the learned step runs, whether DD/QD
evaluation runs on the integer pipe, and the GPU (the kernels of the learned
and integer modes use other shared memory and registers, so their best shape
differs).  The cache is a plain JSON object {key: {"team_warps": t,
"iters_per_launch": k, "ms": ms}} at a path the caller chooses.
"""
from __future__ import annotations

import json
import os
import tempfile

from . import ht


def cache_key(system, limbs: int, device_name: str, learned: bool = False, int_eval: bool | None = None) -> str:
    """int_eval None means the library's default: integer-pipe evaluation for
    DD and QD systems of at most 32 variables."""
    if int_eval is None:
        int_eval = limbs > 1 and system.n_vars <= 32
    deg = int(system.exps.astype(int).sum(axis=1).max())
    return "n=%d;terms=%d;deg=%d;limbs=%d;learned=%d;int=%d;gpu=%s" % (
        system.n_vars, int(sum(system.n_terms)), deg, limbs, int(bool(learned)), int(bool(int_eval)), device_name)


def _load(path):
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        data = json.load(f)
    return data if isinstance(data, dict) else {}


def _store(path, data):
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)  # atomic: concurrent readers see the old or the new file


def tuned_track_shape(sys_handle, system, limbs, gamma, n_sample, params, cache_path, device_name,
                      tune=None, learned=False, int_eval=None):
    """Return a copy of params with team_warps and iters_per_launch set from
    the cache, tuning (and recording) first when the key is missing."""
    tune = tune or ht.ht_tune_track
    key = cache_key(system, limbs, device_name, learned, int_eval)
    data = _load(cache_path)
    hit = data.get(key)
    if hit is None:
        team, iters, ms = tune(sys_handle, system.degrees(), gamma, n_sample, params)
        hit = {"team_warps": int(team), "iters_per_launch": int(iters), "ms": float(ms)}
        data[key] = hit
        if cache_path:
            _store(cache_path, data)
    out = ht.ht_params()
    for name, _ in ht.ht_params._fields_:
        setattr(out, name, getattr(params, name))
    out.team_warps = hit["team_warps"]
    out.iters_per_launch = hit["iters_per_launch"]
    return out
