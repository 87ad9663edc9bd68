"""Learned step sizes for ht_track_paths: data collection and training.

Every computation runs in libht.so; this module only sequences the calls and
keeps the device buffers (torch tensors):

1. ``collect_records``: the plain tracker records the state of each path at
   every ``stride``-th step start (``ht_track_paths_ex`` with a trace buffer);
2. ``step_labels``: each record is restarted with its step scaled by each
   multiplier in ``MULTS`` for one step with the tracker's own limit of
   evaluate-correct rounds; the label is the log of the accepted multiplier
   with the most progress per Newton round (``ht_step_labels``) -- the step the
   state allowed at the least cost, not the plain rule's;
3. ``features`` (``ht_step_features``) and ``train`` (``ht_mlp_train``: BF16
   tensor-core forward, FP32 backward, Adam);
4. ``track(..., net=...)`` runs the tracker with the network proposing steps.
"""
from __future__ import annotations

import numpy as np

import synth

from . import ht

# Candidate step multipliers.  The smallest is 1 / f_up: with rho >= log(1/f_up)
# an accepted learned step followed by the plain growth factor never leaves
# the step smaller than it was, so a biased network cannot make paths crawl.
MULTS = (2.0 / 3.0, 1.0, 1.5, 2.0, 3.0, 4.0)
RHO_RANGE = (float(np.log(2.0 / 3.0)), float(np.log(4.0)))
# The network is trained on rho - RHO_MARGIN: it aims a little below the step
# the state allowed, since a rejected step costs the round limit and a retry.
# On the n = 16 double workload (65,536 held-out paths): margin 0 -> 333 Newton
# rounds per path, 0.1 -> 326, 0.2 -> 324, 0.3 -> 323 with 4 % more time,
# 0.45 -> 337.
RHO_MARGIN = 0.15


def _torch():
    import torch
    return torch


def collect_records(system, limbs, gamma, n_paths, params, stride=2, capacity=None, first_path=0):
    """Track n_paths paths with the plain rule, recording step starts.
    Returns a device tensor [n_records][R] of doubles."""
    torch = _torch()
    n = system.n_vars
    R = ht.ht_record_size(n, limbs, params.max_order)
    cap = capacity or n_paths * 200 // stride + 16
    trace = torch.zeros((cap, R), dtype=torch.float64, device="cuda")
    count = torch.zeros((1,), dtype=torch.int64, device="cuda")
    io = ht.ht_track_io(trace=trace.data_ptr(), trace_capacity=cap, trace_count=count.data_ptr(), trace_stride=stride)
    hs = ht.system_from(system, limbs)
    x = torch.empty((n, 2, limbs, n_paths), dtype=torch.float64, device="cuda")
    st = torch.empty((n_paths,), dtype=torch.int8, device="cuda")
    t = torch.empty((n_paths,), dtype=torch.float64, device="cuda")
    ht.ht_track_paths_ex(hs, system.degrees(), gamma, n_paths, first_path, None, params, x, st, t, io=io)
    torch.cuda.synchronize()
    k = min(int(count.item()), cap)
    return trace[:k].contiguous()


def step_labels(system, limbs, gamma, params, records, newton_max=None):
    torch = _torch()
    hs = ht.system_from(system, limbs)
    lab = torch.empty((records.shape[0], 2), dtype=torch.float32, device="cuda")
    nm = params.newton_max if newton_max is None else newton_max
    ht.ht_step_labels(hs, system.degrees(), gamma, params, records.shape[0], records, MULTS, nm, lab)
    return lab


def features(system, limbs, params, records):
    torch = _torch()
    f = torch.empty((records.shape[0], ht.HT_MLP_IN), dtype=torch.float32, device="cuda")
    ht.ht_step_features(system.n_vars, limbs, params.max_order, params.newton_max, records.shape[0], records, f)
    torch.cuda.synchronize()
    return f


def init_params(seed: int, out_scale: float = 0.01) -> np.ndarray:
    """Uniform fan-in initialisation drawn from the SplitMix64 stream; the output
    layer starts small so the first proposals stay close to the plain rule."""
    rng = synth.SplitMix64(seed)
    p = np.zeros(ht.HT_MLP_NPARAM, dtype=np.float64)
    sizes = [(0, 64 * 16, 16), (64 * 16 + 64, 64 * 64, 64), (64 * 16 + 64 + 64 * 64 + 64, 2 * 64, 64)]
    for k, (off, cnt, fan_in) in enumerate(sizes):
        bound = 1.0 / np.sqrt(fan_in) * (out_scale if k == 2 else 1.0)
        p[off:off + cnt] = (rng.uniform(cnt) * 2 - 1) * bound
    return p.astype(np.float32)


def shuffle(n: int, seed: int) -> np.ndarray:
    """A seeded permutation of range(n) (Fisher-Yates from SplitMix64)."""
    rng = synth.SplitMix64(seed)
    perm = np.arange(n)
    u = rng.uniform(n)
    for i in range(n - 1, 0, -1):
        j = int(u[i] * (i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def train(feat, lab, epochs=30, batch=4096, lr=2e-3, seed=1, margin=RHO_MARGIN):
    """Returns (network handle, per-epoch losses).  The step output is
    trained on rho - margin (see RHO_MARGIN)."""
    torch = _torch()
    perm = torch.from_numpy(shuffle(feat.shape[0], seed)).cuda()
    x = feat[perm].contiguous()
    y = lab[perm].clone()
    y[:, 0] -= margin
    y = y.contiguous()
    net = ht.ht_mlp_create()
    ht.ht_mlp_set_params(net, init_params(seed))
    losses = ht.ht_mlp_train(net, x.shape[0], x, y, epochs, batch, lr)
    return net, losses


def track(system, limbs, gamma, n_paths, params, net=None, fallback_steps=1, first_path=0, check_limbs=0,
          check_params=None, alpha_max=0.0):
    """ht_track_paths_ex with (net given) or without the learned step; returns
    host arrays and stats.  With check_limbs > limbs the endpoints are then
    checked in that precision: Newton's method on the target system from
    every endpoint (polish_only), giving x_check, status_check and the last
    update norms dx_check."""
    torch = _torch()
    n = system.n_vars
    hs = ht.system_from(system, limbs)
    x = torch.empty((n, 2, limbs, n_paths), dtype=torch.float64, device="cuda")
    st = torch.empty((n_paths,), dtype=torch.int8, device="cuda")
    t = torch.empty((n_paths,), dtype=torch.float64, device="cuda")
    stats = ht.ht_stats()
    io = None
    if net is not None:
        io = ht.ht_track_io(mlp=net.handle, fallback_steps=fallback_steps, rho_min=RHO_RANGE[0], rho_max=RHO_RANGE[1],
                            alpha_max=alpha_max)
    ht.ht_track_paths_ex(hs, system.degrees(), gamma, n_paths, first_path, None, params, x, st, t, None, stats, io)
    out = dict(stats=stats.as_dict())
    if check_limbs > limbs:
        hc = ht.system_from(system, check_limbs)
        pc = check_params or ht.ht_default_params(check_limbs)
        xc = torch.empty((n, 2, check_limbs, n_paths), dtype=torch.float64, device="cuda")
        sc = torch.empty_like(st)
        tc = torch.empty_like(t)
        dxc = torch.empty((n_paths,), dtype=torch.float64, device="cuda")
        ioc = ht.ht_track_io(x0_limbs=limbs, polish_only=1, last_dx_out=dxc.data_ptr())
        ht.ht_track_paths_ex(hc, system.degrees(), gamma, n_paths, 0, x, pc, xc, sc, tc, None, None, ioc)
        out.update(x_check=xc.cpu().numpy(), status_check=sc.cpu().numpy(), dx_check=dxc.cpu().numpy())
    torch.cuda.synchronize()
    out.update(x_end=x.cpu().numpy(), status=st.cpu().numpy(), t_end=t.cpu().numpy())
    return out
