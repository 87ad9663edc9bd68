"""Track the paths of one of the synthetic workloads and print the statistics.

    python -m paper_1505_00383_gb300.run_workload WORKLOAD [--paths M] [--limbs L] [--h-min H]

WORKLOAD is a tracking workload of synth.CONFIGS (plain_n6_d, batched_n12_dd,
learned_n16_d, stress_n10_qd); the first M paths of its total-degree homotopy
are tracked with the plain step rule through ht_track_paths_ex in L limbs
(default: the workload's precision) with the chosen predictor.  Used as the command of the tracker
profiles; every step runs in libht.so.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402

from . import ht  # noqa: E402


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("workload", choices=[k for k, c in synth.CONFIGS.items() if c["kind"] == "track"])
    p.add_argument("--paths", type=int, default=0, help="first M paths (0: all, the Bezout number)")
    p.add_argument("--limbs", type=int, default=0, help="1, 2 or 4 (0: the workload's)")
    p.add_argument("--h-min", type=float, default=1e-9)
    p.add_argument("--predictor", type=int, default=0, help="0 extrapolation, 1 Euler, 2 cubic Hermite")
    a = p.parse_args(argv)
    import numpy as np
    import torch
    cfg = synth.CONFIGS[a.workload]
    L = a.limbs or cfg["limbs"]
    s = synth.config_system(a.workload)
    gam = synth.random_gamma(cfg["seed"])
    m = a.paths or int(np.prod(s.degrees().astype(np.int64)))
    hs = ht.system_from(s, L)
    x = torch.empty((s.n_vars, 2, L, m), dtype=torch.float64, device="cuda")
    st = torch.empty((m,), dtype=torch.int8, device="cuda")
    t = torch.empty((m,), dtype=torch.float64, device="cuda")
    stats = ht.ht_stats()
    prm = ht.ht_default_params(L, h_min=a.h_min, predictor=a.predictor)
    ht.ht_track_paths_ex(hs, s.degrees(), gam, m, 0, None, prm, x, st, t, None, stats, None)
    torch.cuda.synchronize()
    print(json.dumps(dict(workload=a.workload, limbs=L, paths=m, **stats.as_dict())))


if __name__ == "__main__":
    main()
