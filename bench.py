"""Benchmark of the hot path: evaluation and differentiation of a polynomial
system at many points (the 65,536-point sweep of a 32-variable system with
2,048 monomials of 2-8 variables), in complex double, double double and quad
double -- one step is one pass over the batch in all three precisions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is whole-job eval-diff points per second, a
point counting once when it has been evaluated (values and full Jacobian) in
all three precisions.  For N > 1 (torchrun) every rank evaluates its own batch
(weak scaling, no collective on the data path).  ``--impl reference`` times
the CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "eval-diff pts/s (values + 32x32 Jacobian per point, complex D+DD+QD)"
UNIT = "pts/s"
WORKLOAD = "evaldiff_n32"
PRECISIONS = (1, 2, 4)
NAMES = {1: "D", 2: "DD", 4: "QD"}

# FP64 instructions per complex operation of the device arithmetic
# (paper_1505_00383_gb300/csrc/ht_mp.cuh): multiply, add, and accumulate of a
# product scaled by a small integer exponent.
OPS = {1: dict(cmul=4, cadd=2, caxpy=2),
       2: dict(cmul=38, cadd=22, caxpy=34),
       4: dict(cmul=448, cadd=140, caxpy=270)}


def eval_ops_per_point(system, L):
    """FP64 instructions the reverse-mode evaluation of one point needs:
    per monomial with k variables of exponents a_r: sum(a_r - 1) multiplications
    for the common factor, 3k - 3 (k >= 2; 1 for k = 1) for value and
    derivatives, one add for the value and one (scaled) add per derivative."""
    o = OPS[L]
    tot = 0
    for a in system.exps.astype(int):
        a = a[a > 0]
        k = a.size
        if k == 0:
            tot += o["cadd"]
            continue
        ncm = int((a - 1).sum()) + (1 if k == 1 else 3 * k - 3)
        tot += ncm * o["cmul"] + o["cadd"] + sum(o["cadd"] if e == 1 else o["caxpy"] for e in a)
    return tot


# Limb products (32x32 -> 64-bit multiply-adds) per complex multiplication of
# the integer variant (paper_1505_00383_gb300/csrc/ht_mpi.cuh): 3 real
# products (Gauss's form), each over the limb pairs whose column is kept
# (x + y >= W - 2).
INT_W = {1: 3, 2: 5, 4: 8}
VARIANT_NAMES = {0: "unrolled fp64", 1: "compact fp64", 2: "integer limbs", 3: "three kernels fp64"}


def int_products_per_point(system, L):
    W = INT_W[L]
    pairs = sum(1 for x in range(W) for y in range(W) if x + y >= W - 2)
    tot = 0
    for a in system.exps.astype(int):
        a = a[a > 0]
        k = a.size
        if k:
            tot += int((a - 1).sum()) + (1 if k == 1 else 3 * k - 3)
    return tot * 3 * pairs


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--n-pts", type=int, default=65536)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--track", default="plain_n6_d,batched_n12_dd",
                   help="tracking workloads to time as well (comma list, '' for none)")
    p.add_argument("--learned", type=int, default=65536,
                   help="paths of the held-out n = 16 double system for learned vs plain (0: skip)")
    p.add_argument("--stress", type=int, default=59049,
                   help="paths of the held-out n = 10 quad double system for learned vs plain (0: skip)")
    p.add_argument("--no-ablation", action="store_true",
                   help="skip the three-kernel (coeff, mon, sum) evaluation against the fused kernel")
    p.add_argument("--no-predictors", action="store_true",
                   help="skip the comparison of the extrapolation, Euler and Hermite predictors")
    p.add_argument("--no-quality-up", action="store_true",
                   help="skip the mixed-precision (double tracking, double double refinement) comparison")
    p.add_argument("--no-paper-sweep", action="store_true",
                   help="skip the evaluation sweep of the stand-ins shaped like the paper's applications")
    return p.parse_args()


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(x, world, dev):
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself on a single rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _traffic(L):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "evaldiff_n32_65536pts.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"sources_sha256:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != _kernel_sha():
        return None
    m = re.search(r"traffic_bytes_per_launch_%s:\s*([0-9.eE+]+)" % NAMES[L], txt)
    return float(m.group(1)) if m else None


def _track_sha():
    h = hashlib.sha256()
    for f in ("ht_track.cu", "ht_track.h", "ht_eval.cuh", "ht_int_row.cuh", "ht_mp.cuh", "ht_mpi.cuh", "ht_mpi_eval.cuh",
              "ht_mpi_ops.cuh", "ht_mlp.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1505_00383_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _track_pipes():
    """Pipe utilisation of the QD tracker kernel from the committed ncu
    summary, if the tracker sources are unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "track_qd_n10_59049paths.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"track_sources_sha256:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != _track_sha():
        return None
    out = {"source": "profiles/track_qd_n10_59049paths.md (ncu, one launch at 16,384 paths)"}
    for key in ("fp64_pipe_pct", "alu_pipe_pct", "fma_pipe_pct", "issue_active_pct", "warps_active_pct"):
        m = re.search(r"%s:\s*([0-9.]+)" % key, txt)
        if m:
            out[key] = float(m.group(1))
    return out


def _kernel_sha():
    h = hashlib.sha256()
    for f in ("ht_evaldiff.cu", "ht_eval.cuh", "ht_int_row.cuh", "ht_mp.cuh", "ht_mpi.cuh", "ht_mpi_eval.cuh",
              "ht_mpi_ops.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1505_00383_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# bounded oracle samples of the tracking workloads (first paths of the system
# the GPU tracks, at least two per host core; about 5-15 s each on 16 cores)
ORACLE_TRACK_SAMPLE = {"plain_n6_d": 64, "batched_n12_dd": 64, "learned_n16_d": 2048, "stress_n10_qd": 32}


def oracle_track_rate(name, seed, limbs, h_min, sample):
    """The oracle tracker (plain rule, all host cores) on the first `sample`
    paths of the workload's system: paths/s and the cores used."""
    import oracle
    oracle.build()
    s = synth.config_system(name, seed)
    g = synth.random_gamma(seed)
    P = oracle.default_params(limbs, h_min=h_min)
    t0 = time.perf_counter()
    oracle.track(s, s.degrees(), g, np.arange(sample), limbs, P, n_threads=0)
    sec = time.perf_counter() - t0
    return {"value": sample / sec, "unit": "paths/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": "first %d paths, plain rule" % sample}


def cpu_oracle_rate(system, budget_pts, threads=0, seed=77):
    """Oracle throughput in the metric's unit on a bounded sample: for each
    precision, budget_pts[L] points evaluated by the oracle's reverse mode."""
    import oracle
    oracle.build()
    per_pt = 0.0
    for L in PRECISIONS:
        n = budget_pts[L]
        x = synth.unit_points(seed + L, system.n_vars, n, L)
        t0 = time.perf_counter()
        oracle.eval_(system, x, n_threads=threads)
        per_pt += (time.perf_counter() - t0) / n
    return 1.0 / per_pt


TRACK_LIMBS = {"plain_n6_d": 1, "batched_n12_dd": 2, "learned_n16_d": 1, "stress_n10_qd": 4}


def track_workload(ht, torch, name, rank, world, reps=2):
    """paths/s of ht_track_paths on one tracking workload (all its paths on
    every rank: weak scaling), with the final status counts."""
    cfg = synth.CONFIGS[name]
    L = TRACK_LIMBS[name]
    system = synth.config_system(name)
    deg = system.degrees()
    m = int(np.prod(deg.astype(np.int64)))
    gam = synth.random_gamma(cfg["seed"])
    over = {"h_min": 0.01} if name == "plain_n6_d" else {"h_min": 1e-6}
    prm = ht.ht_default_params(L, **over)
    hs = ht.system_from(system, L)
    n = system.n_vars
    x = torch.empty((n, 2, L, m), dtype=torch.float64, device="cuda")
    st = torch.empty((m,), dtype=torch.int8, device="cuda")
    t = torch.empty((m,), dtype=torch.float64, device="cuda")
    stats = ht.ht_stats()
    ht.ht_track_paths(hs, deg, gam, m, 0, None, prm, x, st, t, None, stats)  # warm-up (graphs, workspace)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ht.ht_track_paths(hs, deg, gam, m, 0, None, prm, x, st, t, None, stats)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    d = stats.as_dict()
    return {"paths": m, "precision": NAMES[L], "n": n, "s": sec, "paths_per_s": world * m / sec,
            "converged": d["converged"], "failed": d["failed"], "diverged": d["diverged"],
            "steps_per_path": d["steps"] / m, "newton_per_path": d["newton"] / m, "launches": d["launches"],
            "syncs": d["syncs"]}


def _agreement(A, B, tol=1e-10):
    """Fraction of the endpoints of each set that have a partner in the other
    within tol * max(1, |x|_inf) (both directions; the smaller fraction)."""
    from scipy.spatial import cKDTree
    if len(A) == 0 or len(B) == 0:
        return 1.0 if len(A) == len(B) else 0.0
    def emb(X):
        return np.concatenate([X.real, X.imag], axis=1)
    fr = []
    for P, Q in ((A, B), (B, A)):
        d, _ = cKDTree(emb(Q)).query(emb(P), k=1, p=np.inf)
        scale = np.maximum(1.0, np.max(np.abs(P), axis=1))
        fr.append(float(np.mean(d <= tol * scale)))
    return min(fr)


def unfused_ablation(ht, torch, stream, flush, system, xs, n, fused_ms, fused_fp64_ms):
    """The paper's three-kernel organisation (coeff, mon, sum over a vertical
    workspace; Section 3, Tables tabcpugpu and tabmemory) against the fused
    kernel on the same points: per precision one timed call after a warm-up,
    each kernel's time and its algorithmic bandwidth (Table tabbench reports
    the mon and sum kernels' GB/s on the K20C)."""
    out = {}
    for L in PRECISIONS:
        hs = ht.system_from(system, L)
        ht.ht_set_eval_config(hs, 1, 0)
        val = torch.empty((system.n_polys, 2, L, n), dtype=torch.float64, device="cuda")
        jac = torch.empty((system.n_polys, system.n_vars, 2, L, n), dtype=torch.float64, device="cuda")
        ht.ht_eval_diff_unfused(hs, n, xs[L], val, jac, None, stream)  # workspace, term lists
        flush.zero_()
        st = ht.ht_unfused_stats()
        ht.ht_eval_diff_unfused(hs, n, xs[L], val, jac, st, stream)
        d = st.as_dict()
        tot = d["ms_coeff"] + d["ms_mon"] + d["ms_sum"]
        out[NAMES[L]] = {
            "ms": {"coeff": d["ms_coeff"], "mon": d["ms_mon"], "sum": d["ms_sum"], "total": tot},
            "GB_per_s": {k: d["bytes_" + k] / (d["ms_" + k] * 1e-3) / 1e9 for k in ("coeff", "mon", "sum")},
            "workspace_GB_moved": (d["bytes_coeff"] + d["bytes_mon"] + d["bytes_sum"]) / 1e9,
            "fused_ms": fused_ms[L], "fused_variant": "the benchmark's tuned kernel",
            "unfused_over_fused": tot / fused_ms[L],
            "fused_fp64_ms": fused_fp64_ms.get(L, fused_ms[L]),
            "unfused_over_fused_same_arithmetic": tot / fused_fp64_ms.get(L, fused_ms[L])}
        del val, jac
    return out


def predictor_comparison(ht, torch, world, name="batched_n12_dd", h_min=1e-6):
    """The three predictors of the tracker on one workload (Section 2's
    predictor stage): extrapolation through up to five accepted points (0),
    Euler (1) and cubic Hermite (2) on the path's tangent from J v = -dh/dt.
    Per predictor: wall time, steps and Newton rounds per path, status
    counts, and the endpoints' agreement with the extrapolation run."""
    L = TRACK_LIMBS[name]
    s = synth.config_system(name)
    gam = synth.random_gamma(synth.CONFIGS[name]["seed"])
    m = int(np.prod(s.degrees().astype(np.int64)))
    hs = ht.system_from(s, L)
    out, ends = {}, {}
    for pred in (0, 1, 2):
        prm = ht.ht_default_params(L, h_min=h_min, predictor=pred)
        x = torch.empty((s.n_vars, 2, L, m), dtype=torch.float64, device="cuda")
        st = torch.empty((m,), dtype=torch.int8, device="cuda")
        t = torch.empty((m,), dtype=torch.float64, device="cuda")
        stats = ht.ht_stats()
        ht.ht_track_paths(hs, s.degrees(), gam, m, 0, None, prm, x, st, t, None, stats)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ht.ht_track_paths(hs, s.degrees(), gam, m, 0, None, prm, x, st, t, None, stats)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        d = stats.as_dict()
        xs = x.cpu().numpy()
        ok = st.cpu().numpy() == 1
        ends[pred] = (xs[:, 0, 0, :] + 1j * xs[:, 1, 0, :]).T[ok]
        out[{0: "extrapolation", 1: "euler", 2: "hermite"}[pred]] = {
            "s": sec, "paths_per_s": world * m / sec, "steps_per_path": d["steps"] / m,
            "newton_per_path": d["newton"] / m, "rejects_per_path": d["rejects"] / m,
            "counts": {k: d[k] for k in ("converged", "failed", "diverged")},
            "endpoint_agreement_with_extrapolation_1e-10": _agreement(ends[0], ends[pred]) if pred else 1.0}
    return {"workload": name, "paths": m, "precision": NAMES[L], "h_min": h_min, "by_predictor": out}


def quality_up(ht, torch, world, name="batched_n12_dd", Lh=2, h_min=1e-6):
    """Accuracy against time (the paper's "quality up"): the workload tracked
    in double alone, in double with refinement in the high precision and the
    failures tracked again there (ht_track_refined), and in the high
    precision alone.  Accuracy of each arm: the largest distance of its
    converged endpoints to the high-precision run's (leading two limbs,
    nearest-neighbour pairing)."""
    from scipy.spatial import cKDTree
    s = synth.config_system(name)
    gam = synth.random_gamma(synth.CONFIGS[name]["seed"])
    m = int(np.prod(s.degrees().astype(np.int64)))
    n = s.n_vars
    lo, hi = ht.system_from(s, 1), ht.system_from(s, Lh)
    pl, ph = ht.ht_default_params(1, h_min=h_min), ht.ht_default_params(Lh, h_min=h_min)
    bufs = lambda L: (torch.empty((n, 2, L, m), dtype=torch.float64, device="cuda"),
                      torch.empty((m,), dtype=torch.int8, device="cuda"),
                      torch.empty((m,), dtype=torch.float64, device="cuda"))
    xd, sd, td = bufs(1)
    xr, sr, tr = bufs(Lh)
    xh, sh, th = bufs(Lh)
    rs = ht.ht_refine_stats()
    arms = {"d_only": lambda: ht.ht_track_paths(lo, s.degrees(), gam, m, 0, None, pl, xd, sd, td),
            "refined": lambda: ht.ht_track_refined(lo, hi, s.degrees(), gam, m, 0, pl, ph, xr, sr, tr, rs),
            "high_only": lambda: ht.ht_track_paths(hi, s.degrees(), gam, m, 0, None, ph, xh, sh, th)}
    sec = {}
    for k, f in arms.items():
        f()  # warm-up: workspaces and graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f()
        torch.cuda.synchronize()
        sec[k] = time.perf_counter() - t0

    def lead2(x):
        x = x.cpu().numpy()
        z = x[:, 0, 0, :] + 1j * x[:, 1, 0, :]
        if x.shape[2] > 1:
            z = z + (x[:, 0, 1, :] + 1j * x[:, 1, 1, :])
        return z.T

    ref = lead2(xh)[sh.cpu().numpy() == 1]
    tree = cKDTree(np.concatenate([ref.real, ref.imag], axis=1))

    def dist(x, st):
        z = lead2(x)[st.cpu().numpy() == 1]
        d, _ = tree.query(np.concatenate([z.real, z.imag], axis=1), k=1, p=np.inf)
        return float(np.max(d / np.maximum(1.0, np.max(np.abs(z), axis=1)))) if z.size else None

    count = lambda st: {c: int((st.cpu().numpy() == v).sum()) for c, v in (("converged", 1), ("failed", -1),
                                                                             ("diverged", -2))}
    return {"paths": m, "n": n, "high": NAMES[Lh],
            "seconds": sec, "paths_per_s": {k: world * m / v for k, v in sec.items()},
            "refined_phases_ms": {k: rs.as_dict()[k] for k in ("ms_lo", "ms_refine", "ms_retrack")},
            "retracked": rs.retracked,
            "counts": {"d_only": count(sd), "refined": count(sr), "high_only": count(sh)},
            "max_dist_to_high_run": {"d_only": dist(xd, sd), "refined": dist(xr, sr)},
            "what": "double tracking; double + refinement in %s + failures re-tracked in %s; %s alone"
                    % (NAMES[Lh], NAMES[Lh], NAMES[Lh])}


# learned+batched against plain batched: the workload, its tracking and check
# precisions, the training systems (same shape, other seeds; traces and
# probes in double) and the held-out system tracked by both arms
# The n = 16 network trains on traces of 200 seeded systems of the workload's
# shape (32 paths each, 20 epochs); on the held-out system that gives 334 Newton
# rounds per path against 343 for 6 systems x 256 paths (same sample count
# within 4x), for about 70 s of trace collection.  The n = 16 launch shape is
# tuned on all 65,536 paths: on samples of 4,096 and 16,384 paths 16-warp
# teams won, and they ran the 65,536-path arms 20 % slower than 8-warp teams.
LEARNED_CASES = {
    "learned_n16_d": dict(limbs=1, check_limbs=2, eval_seed=3500, train_seeds=range(3000, 3200), train_paths=32,
                         epochs=20, warm_paths=None, tune_paths=65536),
    "stress_n10_qd": dict(limbs=4, check_limbs=0, eval_seed=4000, train_seeds=range(4100, 4106), train_paths=256,
                         epochs=30, warm_paths=1024, tune_paths=1024),
}


def learned_vs_plain(ht, torch, world, name, m):
    """The learned step against the plain rule on a held-out system of the
    workload's shape: the network is trained first (outside the timing) on
    step-start records of seeded training systems, then both trackers run all
    m paths (plus, for the double workload, the double double check of every
    endpoint) with identical seeds."""
    from paper_1505_00383_gb300 import learned
    case = LEARNED_CASES[name]
    L, CL = case["limbs"], case["check_limbs"]
    prm_train = ht.ht_default_params(1, h_min=1e-9)
    prm = ht.ht_default_params(L, h_min=1e-9)
    t0 = time.perf_counter()
    feats, labs = [], []
    for seed in case["train_seeds"]:
        s = synth.config_system(name, seed)
        g = synth.random_gamma(seed)
        rec = learned.collect_records(s, 1, g, case["train_paths"], prm_train, stride=2)
        labs.append(learned.step_labels(s, 1, g, prm_train, rec))
        feats.append(learned.features(s, 1, prm_train, rec))
    net, losses = learned.train(torch.cat(feats), torch.cat(labs), epochs=case["epochs"], batch=2048, lr=2e-3)
    train_s = time.perf_counter() - t0
    s = synth.config_system(name, case["eval_seed"])
    g = synth.random_gamma(case["eval_seed"])
    # launch shape from the autotuner (plain rule, a sample of the paths), kept
    # in the tuning cache across runs on this machine; both arms use it
    from paper_1505_00383_gb300 import tuning
    cache = os.environ.get("HT_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ht_tune_track.json"))
    before = tuning._load(cache)
    tuned = tuning.tuned_track_shape(ht.system_from(s, L), s, L, g, case["tune_paths"], prm, cache,
                                     torch.cuda.get_device_name())
    from_cache = tuning.cache_key(s, L, torch.cuda.get_device_name()) in before
    team, iters = tuned.team_warps, tuned.iters_per_launch
    prm.team_warps, prm.iters_per_launch = team, iters
    out = {}
    for arm, nn in (("plain", None), ("learned", net)):
        learned.track(s, L, g, case["warm_paths"] or m, prm, net=nn, check_limbs=CL)  # warm-up: workspace, graphs
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = learned.track(s, L, g, m, prm, net=nn, check_limbs=CL)
        sec = time.perf_counter() - t1
        out[arm] = (r, sec)
    (ra, sa), (rb, sb) = out["plain"], out["learned"]

    def ends(r, checked):  # converged endpoints, leading two limbs
        X = r["x_check"] if checked else r["x_end"]
        z = X[:, 0, 0, :] + 1j * X[:, 1, 0, :]
        if X.shape[2] > 1:
            z = z + (X[:, 0, 1, :] + 1j * X[:, 1, 1, :])
        ok = r["status"] == 1
        if checked:
            ok = ok & (r["status_check"] == 1)
        return z.T[ok]
    chk = CL > L
    agree = _agreement(ends(ra, chk), ends(rb, chk))
    counts = lambda r: {k: r["stats"][k] for k in ("converged", "failed", "diverged")}
    res = {"paths": m, "precision": NAMES[L], "n": s.n_vars, "heldout_seed": case["eval_seed"],
           "plain_s": sa, "learned_s": sb, "plain_paths_per_s": world * m / sa,
           "learned_paths_per_s": world * m / sb, "speedup": sa / sb,
           "newton_per_path": {"plain": ra["stats"]["newton"] / m, "learned": rb["stats"]["newton"] / m},
           "rejects_per_path": {"plain": ra["stats"]["rejects"] / m, "learned": rb["stats"]["rejects"] / m},
           "counts": {"plain": counts(ra), "learned": counts(rb)},
           "counts_equal": counts(ra) == counts(rb), "endpoint_agreement_1e-10": agree,
           "launch_shape": {"team_warps": team, "iters_per_launch": iters,
                            "tuned_on_paths": case["tune_paths"], "from_tuning_cache": from_cache},
           "train": {"systems": len(case["train_seeds"]), "paths_each": case["train_paths"], "precision": "D",
                     "epochs": case["epochs"],
                     "samples": int(sum(f.shape[0] for f in feats)), "first_loss": float(losses[0]),
                     "last_loss": float(losses[-1]), "seconds": train_s}}
    if chk:
        checked = lambda r: {"agree_with_tracker_1e-10": _agreement(ends(r, True), ends(r, False)),
                             "max_last_dx": float(np.max(r["dx_check"][r["status"] == 1]))
                             if np.any(r["status"] == 1) else None}
        res["check"] = {"precision": NAMES[CL], "plain": checked(ra), "learned": checked(rb),
                        "what": "Newton on f from every converged endpoint (timed with the arm)"}
    return res


# The paper's GPU totals in ms (K20C, Tables tabevalcyclic10, tabevalnash8,
# tabevalpieri44; evaluation and differentiation at #evals points), for
# context next to the stand-ins of the same shape: other hardware, other
# (real) systems.
PAPER_GPU_MS = {
    "cyclic10_shape": {"D": {10: 0.028, 1000: 0.282, 3000: 0.826}, "DD": {10: 0.088, 1000: 0.743, 3000: 2.163},
                       "QD": {10: 0.705, 1000: 5.853, 3000: 16.864}},
    "nash8_shape": {"D": {10: 0.106, 1000: 1.973, 3000: 5.922}, "DD": {10: 0.361, 1000: 5.341, 3000: 15.922},
                    "QD": {10: 2.964, 1000: 45.253, 3000: 136.510}},
    "pieri44_shape": {"D": {10: 0.324, 1000: 6.751, 3000: 20.597}, "DD": {10: 0.995, 1000: 18.299, 3000: 54.879},
                      "QD": {10: 8.328, 1000: 158.306}},
}


def paper_shape_sweep(ht, torch, stream, flush, fp64_peak, imad_peak, reps=10):
    """ht_eval_diff on the stand-ins shaped like the paper's applications at
    the point counts of its evaluation tables: per shape, precision and point
    count the autotuner's choice (fused FP64 bodies, integer limbs, or the
    three kernels, which spread few points' work over monomials), then the
    median of `reps` launches (CUDA events, L2 flushed before each)."""
    out = {}
    for name in ("cyclic10_shape", "nash8_shape", "pieri44_shape"):
        system = synth.config_system(name)
        res = {"n": system.n_vars, "monomials": system.n_monomials}
        for L in PRECISIONS:
            hs = ht.system_from(system, L)
            nmax = max(synth.PAPER_SWEEP_POINTS)
            x = torch.from_numpy(synth.unit_points(900 + L, system.n_vars, nmax, L)).cuda()
            val = torch.empty((system.n_polys, 2, L, nmax), dtype=torch.float64, device="cuda")
            jac = torch.empty((system.n_polys, system.n_vars, 2, L, nmax), dtype=torch.float64, device="cuda")
            rows = {}
            for n in synth.PAPER_SWEEP_POINTS:
                xs = x[..., :n].contiguous()
                vs = torch.empty((system.n_polys, 2, L, n), dtype=torch.float64, device="cuda")
                js = torch.empty((system.n_polys, system.n_vars, 2, L, n), dtype=torch.float64, device="cuda")
                v, t, _ = ht.ht_tune_eval(hs, n, xs, vs, js, reps=3)  # the autotuner's choice at this size
                ms = []
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ht.ht_eval_diff(hs, n, xs, vs, js, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                m = statistics.median(ms)
                row = {"ms": m, "pts_per_s": n / (m * 1e-3), "variant": VARIANT_NAMES[v], "threads": t}
                if v == 2:
                    row["imad_frac"] = int_products_per_point(system, L) * n / (m * 1e-3) / imad_peak
                else:
                    row["fp64_frac"] = eval_ops_per_point(system, L) * n / (m * 1e-3) / fp64_peak
                paper = PAPER_GPU_MS[name][NAMES[L]].get(n)
                if paper is not None:
                    row["paper_k20c_ms"] = paper
                rows[n] = row
            res[NAMES[L]] = {"by_points": rows}
        out[name] = res
    return out


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    system = synth.config_system(WORKLOAD)
    cores = os.cpu_count() or 1
    budget = {1: 512, 2: 48, 4: 8}
    for _ in range(a.warmup):
        cpu_oracle_rate(system, {1: 16, 2: 4, 4: 1}, threads=cores)
    rates = [cpu_oracle_rate(system, budget, threads=cores, seed=100 + s) for s in range(a.steps)]
    v = float(statistics.median(rates))
    sample = "per step: %d D + %d DD + %d QD points of the %d-point sweep" % (budget[1], budget[2], budget[4],
                                                                               a.n_pts)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": a.n_pts / v * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (D, DD, QD limbs)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_vars": 32, "n_polys": 32, "monomials": 2048, "n_pts": a.n_pts},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_1505_00383_gb300 import _build
    _build.build()
    from paper_1505_00383_gb300 import ht

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    system = synth.config_system(WORKLOAD)
    n = a.n_pts
    sys_h, xs, vals, jacs = {}, {}, {}, {}
    for L in PRECISIONS:
        sys_h[L] = ht.system_from(system, L)
        xs[L] = torch.from_numpy(synth.unit_points(1000 + 7 * rank + L, system.n_vars, n, L)).to(dev)
        vals[L] = torch.empty((system.n_polys, 2, L, n), dtype=torch.float64, device=dev)
        jacs[L] = torch.empty((system.n_polys, system.n_vars, 2, L, n), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    fp64_peak = ht.ht_bench_fp64_rate(100)
    imad_peak = ht.ht_bench_imad_rate(20)
    tuned, variant = {}, {}
    for L in PRECISIONS:  # autotuner: kernel body and CTA size per precision (part of warm-up)
        v, t, ms = ht.ht_tune_eval(sys_h[L], n, xs[L], vals[L], jacs[L], reps=1)
        variant[L] = v
        tuned[NAMES[L]] = {"variant": VARIANT_NAMES[v], "threads": t}
    # where the integer variant won, one launch of the FP64 bodies for reference
    # (FP64-pipe utilisation of the error-free DD/QD arithmetic)
    fp64_ref = {}
    for L in PRECISIONS:
        if variant[L] == 2:
            ht.ht_set_eval_config(sys_h[L], 1, 256)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            ht.ht_eval_diff(sys_h[L], n, xs[L], vals[L], jacs[L], stream)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64_ref[L] = e0.elapsed_time(e1)
            ht.ht_set_eval_config(sys_h[L], variant[L], tuned[NAMES[L]]["threads"])

    def step(events=None):
        for L in PRECISIONS:
            if events is not None:
                events[L][0].record(stream)
            ht.ht_eval_diff(sys_h[L], n, xs[L], vals[L], jacs[L], stream)
            if events is not None:
                events[L][1].record(stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    ev = [{L: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for L in PRECISIONS}
          for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        for s in range(a.steps):
            flush.zero_()
            step(ev[s])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    launch_ms = {L: [ev[s][L][0].elapsed_time(ev[s][L][1]) for s in range(a.steps)] for L in PRECISIONS}
    ms_step = sum(statistics.mean(launch_ms[L]) for L in PRECISIONS)
    ms_step = max_over_ranks(ms_step, world, dev)
    value = world * n / (ms_step * 1e-3)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not a.no_e2e:
        hx = {L: xs[L].cpu().pin_memory() for L in PRECISIONS}
        hv = {L: torch.empty(vals[L].shape, dtype=torch.float64).pin_memory() for L in PRECISIONS}
        hj = {L: torch.empty(jacs[L].shape, dtype=torch.float64).pin_memory() for L in PRECISIONS}
        for L in PRECISIONS:  # warm-up (workspace allocation)
            ht.ht_eval_diff_host(sys_h[L], n, hx[L], hv[L], hj[L], stream)
        del vals, jacs
        ts, per_l = [], {L: [] for L in PRECISIONS}
        for s in range(max(1, min(a.steps, 3))):
            t0 = time.perf_counter()
            for L in PRECISIONS:
                t1 = time.perf_counter()
                ht.ht_eval_diff_host(sys_h[L], n, hx[L], hv[L], hj[L], stream)
                per_l[L].append(time.perf_counter() - t1)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.mean(ts), world, dev)
        e2e = {"value": world * n / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(hx[L].numel() * 8 for L in PRECISIONS)),
               "d2h_bytes_per_step": int(sum((hv[L].numel() + hj[L].numel()) * 8 for L in PRECISIONS)),
               "ms_per_precision": {NAMES[L]: [1e3 * v for v in per_l[L]] for L in PRECISIONS}}

    # roofline of the dominant kernel (the one with the largest share of the step)
    dom = max(PRECISIONS, key=lambda L: statistics.mean(launch_ms[L]))
    dom_ms = statistics.mean(launch_ms[dom])
    tr = _traffic(dom)
    if variant[dom] == 2:
        work = int_products_per_point(system, dom) * n
        achieved = work / (dom_ms * 1e-3)
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": imad_peak / 1e12,
                    "unit": "T IMAD.WIDE/s", "frac": achieved / imad_peak, "traffic": tr,
                    "kernel": "%s<%d> (%s, integer limbs)" % (
                        "evaldiff_intblk_kernel" if tuned[NAMES[dom]]["threads"] == 256 else "evaldiff_int_kernel",
                        dom, NAMES[dom]),
                    "work": "32x32->64-bit limb products of the complex multiplications",
                    "peak_source": "measured live: ht_bench_imad_rate (IMAD.WIDE chains on all SMs)"}
    else:
        ops_launch = eval_ops_per_point(system, dom) * n
        achieved = ops_launch / (dom_ms * 1e-3)
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": fp64_peak / 1e12,
                    "unit": "T FP64-instr/s", "frac": achieved / fp64_peak,
                    "traffic": tr, "kernel": "evaldiff_kernel<%d> (%s)" % (dom, NAMES[dom]),
                    "work": "FP64 instructions of the error-free DD/QD arithmetic",
                    "peak_source": "measured live: ht_bench_fp64_rate (DFMA chains on all SMs)"}
    per_prec = {}
    for L in PRECISIONS:
        m = statistics.mean(launch_ms[L])
        d = {"ms": m, "pts_per_s": n / (m * 1e-3), "variant": tuned[NAMES[L]]["variant"],
             "out_GB_per_s": (system.n_polys * (system.n_vars + 1) * 16 * L * n) / (m * 1e-3) / 1e9}
        if variant[L] == 2:
            d["imad_frac"] = int_products_per_point(system, L) * n / (m * 1e-3) / imad_peak
            if L in fp64_ref:
                d["fp64_bodies"] = {"ms": fp64_ref[L], "pts_per_s": n / (fp64_ref[L] * 1e-3),
                                    "fp64_frac": eval_ops_per_point(system, L) * n / (fp64_ref[L] * 1e-3) / fp64_peak}
        else:
            d["fp64_frac"] = eval_ops_per_point(system, L) * n / (m * 1e-3) / fp64_peak
        per_prec[NAMES[L]] = d
    peaks = {"fp64_instr_per_s": fp64_peak, "imad_wide_per_s": imad_peak}
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        peaks["hbm_GBps_measured"] = json.load(open(mp)).get("hbm_gbs")

    ablation = None
    if not a.no_ablation:
        ablation = unfused_ablation(ht, torch, stream, flush, system, xs, n,
                                    {L: statistics.mean(launch_ms[L]) for L in PRECISIONS}, fp64_ref)
    paper_sweep = None
    if not a.no_paper_sweep:
        paper_sweep = paper_shape_sweep(ht, torch, stream, flush, fp64_peak, imad_peak)

    tracking = {}
    oracle_side = rank == 0 and world == 1 and not a.no_cpu
    for name in [w for w in a.track.split(",") if w]:
        tracking[name] = track_workload(ht, torch, name, rank, world)
        if oracle_side:
            cfg = synth.CONFIGS[name]
            tracking[name]["cpu_baseline"] = oracle_track_rate(name, cfg["seed"], TRACK_LIMBS[name],
                                                               0.01 if name == "plain_n6_d" else 1e-6,
                                                               ORACLE_TRACK_SAMPLE[name])
    if not a.no_quality_up:
        tracking["quality_up_n12_dd"] = quality_up(ht, torch, world)
    if not a.no_predictors:
        tracking["predictors_n12_dd"] = predictor_comparison(ht, torch, world)
    for name, m, key in (("learned_n16_d", a.learned, "learned_n16_d_vs_plain"),
                         ("stress_n10_qd", a.stress, "stress_n10_qd_vs_plain")):
        if m > 0:
            tracking[key] = learned_vs_plain(ht, torch, world, name, m)
            if name == "stress_n10_qd":
                tracking[key]["pipes"] = _track_pipes()
            if oracle_side:
                tracking[key]["cpu_baseline"] = oracle_track_rate(name, LEARNED_CASES[name]["eval_seed"],
                                                                  TRACK_LIMBS[name], 1e-9, ORACLE_TRACK_SAMPLE[name])

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cores = os.cpu_count() or 1
        budget = {1: 1024, 2: 64, 4: 16}
        v = cpu_oracle_rate(system, budget, threads=cores)
        budget1 = {1: 128, 2: 8, 4: 2}
        v1 = cpu_oracle_rate(system, budget1, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d D + %d DD + %d QD points of the sweep, all host cores" % (budget[1], budget[2],
                                                                                         budget[4]),
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample": "%d D + %d DD + %d QD points, one thread (the paper's one-core "
                                           "comparison)" % (budget1[1], budget1[2], budget1[4])}}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (D, DD, QD limbs)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_vars": 32, "n_polys": 32, "monomials": 2048,
                       "monomial_vars": "2-8", "exponents": "1-3", "n_pts_per_gpu": n,
                       "l2": "flushed (512 MB write) before every timed step; outputs 1.1-4.5 GB per launch",
                       "parallelism": "independent batch per GPU"},
            "per_precision": per_prec, "tuned": tuned, "unfused_ablation": ablation, "paper_shapes": paper_sweep, "tracking": tracking, "roofline": roofline, "peaks": peaks, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": a.steps * len(PRECISIONS), "clocks": clk.summary(),
            "wall_s_timed_region": t_wall,
        }))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
