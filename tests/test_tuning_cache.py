"""Host logic of the tracker tuning cache (no GPU: a fake tuner)."""
import json

import numpy as np

import synth
from paper_1505_00383_gb300 import ht, tuning


def _params():
    p = ht.ht_params()
    p.h0, p.h_min, p.h_max, p.newton_max = 0.05, 1e-9, 0.1, 3
    return p


def test_cache_tunes_once_per_key_and_reuses(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    s = synth.config_system("plain_n6_d")
    calls = []

    def fake(handle, deg, gamma, n, params):
        calls.append((handle, tuple(deg), n))
        return 4, 2, 12.5

    p = _params()
    a = tuning.tuned_track_shape("H", s, 1, (1.0, 0.0), 256, p, path, "GB300", tune=fake)
    assert (a.team_warps, a.iters_per_launch) == (4, 2) and len(calls) == 1
    assert a.h_min == p.h_min and a.newton_max == 3 and p.team_warps == 0  # a copy; the input is unchanged
    b = tuning.tuned_track_shape("H", s, 1, (1.0, 0.0), 256, p, path, "GB300", tune=fake)
    assert (b.team_warps, b.iters_per_launch) == (4, 2) and len(calls) == 1  # from the cache
    data = json.load(open(path))
    key = tuning.cache_key(s, 1, "GB300")
    assert data[key] == {"team_warps": 4, "iters_per_launch": 2, "ms": 12.5}
    # another precision or GPU is another key
    tuning.tuned_track_shape("H", s, 2, (1.0, 0.0), 256, p, path, "GB300", tune=fake)
    tuning.tuned_track_shape("H", s, 1, (1.0, 0.0), 256, p, path, "other", tune=fake)
    assert len(calls) == 3 and len(json.load(open(path))) == 3


def test_key_depends_on_shape_not_on_coefficients():
    a = synth.config_system("batched_n12_dd")
    b = synth.config_system("batched_n12_dd", 2001)
    assert tuning.cache_key(a, 2, "g") == tuning.cache_key(b, 2, "g")
    c = synth.config_system("plain_n6_d")
    assert tuning.cache_key(a, 2, "g") != tuning.cache_key(c, 2, "g")
    assert tuning.cache_key(a, 2, "g").startswith("n=12;terms=%d;deg=2;" % int(np.sum(a.n_terms)))


def test_key_separates_learned_integer_and_degree():
    """The learned and integer-evaluation kernels use other shared memory and
    registers, and the degree changes the work per monomial: each is a key."""
    a = synth.config_system("batched_n12_dd")
    base = tuning.cache_key(a, 2, "g")
    assert base == tuning.cache_key(a, 2, "g", learned=False, int_eval=True)  # DD at n = 12: integer by default
    assert tuning.cache_key(a, 2, "g", learned=True) != base
    assert tuning.cache_key(a, 2, "g", int_eval=False) != base
    assert tuning.cache_key(a, 1, "g").endswith("learned=0;int=0;gpu=g")  # double: FP64 pipe
    q = synth.config_system("stress_n10_qd")
    assert ";deg=3;" in tuning.cache_key(q, 4, "g")


def test_cache_keeps_learned_and_plain_shapes_apart(tmp_path):
    path = str(tmp_path / "tune.json")
    s = synth.config_system("plain_n6_d")
    calls = []

    def fake(handle, deg, gamma, n, params):
        calls.append(n)
        return (8, 4, 1.0) if len(calls) == 1 else (2, 8, 2.0)

    p = _params()
    a = tuning.tuned_track_shape("H", s, 1, (1.0, 0.0), 64, p, path, "G", tune=fake)
    b = tuning.tuned_track_shape("H", s, 1, (1.0, 0.0), 64, p, path, "G", tune=fake, learned=True)
    assert (a.team_warps, b.team_warps) == (8, 2) and len(calls) == 2
