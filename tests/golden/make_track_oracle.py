"""Write the oracle's tracking results on a seeded subset of the paths of the
two batched tracking workloads (tests/golden/track_oracle_*.npz).

The oracle tracks each selected path on its own (plain step rule, the
workload's parameters); the GPU tests compare their full-size batched runs
with these path by path.  Only oracle/ and synth/ are called: no value here
comes from the CUDA library.

  python tests/golden/make_track_oracle.py [--threads N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

# workload: (precision in limbs, step floor, number of sampled paths, seed of the sample)
CASES = {
    "batched_n12_dd": (2, 1e-6, 1024, 12),
    "stress_n10_qd": (4, 1e-9, 1024, 10),
}


def sample_ids(name: str) -> np.ndarray:
    """The first and last path plus seeded distinct indices, taken in the
    order drawn until there are CASES[name][2] of them; returned sorted."""
    cfg = synth.CONFIGS[name]
    m = cfg["degree"] ** cfg["n"]
    k, seed = CASES[name][2], CASES[name][3]
    rng = synth.SplitMix64(seed)
    ids = [0, m - 1]
    seen = set(ids)
    while len(ids) < k:
        for i in rng.integers(0, m, k):
            if int(i) not in seen and len(ids) < k:
                seen.add(int(i))
                ids.append(int(i))
    return np.array(sorted(ids), dtype=np.int64)


def path(name: str) -> str:
    return os.path.join(HERE, "track_oracle_%s.npz" % name)


def track(name: str, ids, threads: int = 0):
    L, h_min = CASES[name][0], CASES[name][1]
    cfg = synth.CONFIGS[name]
    s = synth.config_system(name)
    g = synth.random_gamma(cfg["seed"])
    return oracle.track(s, s.degrees(), g, ids, L, oracle.default_params(L, h_min=h_min), n_threads=threads)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    oracle.build()
    for name in CASES:
        ids = sample_ids(name)
        t0 = time.perf_counter()
        o = track(name, ids, a.threads)
        np.savez_compressed(path(name), ids=ids, status=o["status"], steps=o["steps"], rejects=o["rejects"],
                            newton=o["newton"], t_end=o["t_end"], x_lead=o["x_end"][:, :, 0, :])
        print(name, len(ids), "paths", "%.1f s" % (time.perf_counter() - t0), flush=True)


if __name__ == "__main__":
    main()
