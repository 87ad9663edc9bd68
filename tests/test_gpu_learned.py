"""The learned step: network kernels against the oracle's fp64 network, the
tracker's record/restart machinery, and what the trained network gains over
the plain step rule on held-out systems."""
import numpy as np
import pytest

import oracle
import synth
from match import match_sets, to_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ht():
    from paper_1505_00383_gb300 import _build, ht as binding
    _build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return binding


def _bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _net(ht, params):
    net = ht.ht_mlp_create()
    ht.ht_mlp_set_params(net, params)
    return net


def _rand_params(seed, scale=0.3):
    rng = synth.SplitMix64(seed)
    return ((rng.uniform(5378) * 2 - 1) * scale).astype(np.float32)


def _bf16_params(p):
    """The network as the GPU holds it: BF16 weights, FP32 biases."""
    pb = p.astype(np.float64).copy()
    wmask = np.ones(5378, bool)
    for off, cnt in ((1024, 64), (1024 + 64 + 4096, 64), (5376, 2)):  # biases stay FP32
        wmask[off:off + cnt] = False
    pb[wmask] = _bf16(p[wmask])
    return pb


@pytest.mark.parametrize("B", [1, 37, 100, 4096 + 17])
def test_network_forward_matches_oracle(ht, B):
    """Tensor-core forward (BF16 operands, FP32 accumulation) against the fp64
    oracle on the same BF16-rounded weights and inputs, output by output,
    within the oracle's rigorous bound for BF16 hidden activations and FP32
    accumulation (oracle.mlp_error_bound)."""
    p = _rand_params(11)
    rng = synth.SplitMix64(B)
    x = (rng.uniform(B * 16).reshape(B, 16) * 2 - 1).astype(np.float32)
    net = _net(ht, p)
    y = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    ht.ht_mlp_forward(net, B, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    pb = _bf16_params(p)
    ref = oracle.mlp_forward(_bf16(x), pb)
    yb, _, _ = oracle.mlp_error_bound(_bf16(x), np.zeros((B, 2)), pb)
    err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= yb), (np.argmax(err - yb), float(np.max(err / yb)))


@pytest.mark.parametrize("B", [1, 63, 64, 65, 333, 2048 + 5])
def test_network_gradient_matches_oracle(ht, B):
    """Loss and every one of the 5,378 gradient entries of the tensor-core
    backward pass against the fp64 oracle, each within its own rigorous bound
    (BF16 activations and gradient operands, FP32 accumulation, ReLU decisions
    that may differ where a pre-activation is within its error of zero).  B
    spans one chunk of 64 samples, its edges and a ragged last chunk."""
    p = _rand_params(12)
    rng = synth.SplitMix64(5 + B)
    x = (rng.uniform(B * 16).reshape(B, 16) * 2 - 1).astype(np.float32)
    tgt = (rng.uniform(B * 2).reshape(B, 2) - 0.5).astype(np.float32)
    net = _net(ht, p)
    g = torch.empty((5378,), dtype=torch.float32, device="cuda")
    loss = torch.empty((1,), dtype=torch.float32, device="cuda")
    ht.ht_mlp_loss_grad(net, B, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(), g, loss)
    torch.cuda.synchronize()
    pb = _bf16_params(p)
    xb, tb = _bf16(x), tgt.astype(np.float64)
    ref_loss, ref_g = oracle.mlp_loss_grad(xb, tb, pb)
    _, gb, lb = oracle.mlp_error_bound(xb, tb, pb)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ref_loss) <= lb
    err = np.abs(gg - ref_g)
    bad = np.flatnonzero(err > gb)
    assert bad.size == 0, (bad[:8], err[bad[:8]], gb[bad[:8]])
    # deterministic: the same call gives the same bits
    g2 = torch.empty_like(g)
    ht.ht_mlp_loss_grad(net, B, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(), g2, None)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


def test_adam_matches_oracle_step_by_step(ht):
    """K = 5 GPU Adam steps (FP32 masters) from identical parameters and
    gradients against the oracle's fp64 Adam with the same constants (the
    FP32 values of 0.9, 0.999 and 1e-8): every parameter and both moments
    after every step, each within a bound derived from FP32 rounding (unit
    u = 2^-24 per operation; the bias corrections 1 - beta^k rounded once to
    FP32), accumulated over the steps; then the BF16 copy the products use."""
    K, lr = 5, 3e-3
    b1, b2, eps = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))
    p = _rand_params(13)
    net = _net(ht, p)
    po = p.astype(np.float64).copy()
    m = np.zeros_like(po)
    v = np.zeros_like(po)
    u = 2.0 ** -24
    ep, em, ev = np.zeros_like(po), np.zeros_like(po), np.zeros_like(po)
    rng = synth.SplitMix64(99)
    for k in range(1, K + 1):
        gk = ((rng.uniform(5378) * 2 - 1) * 10.0 ** (rng.uniform(5378) * 4 - 3)).astype(np.float32)
        gk[::97] = 0.0  # never a gradient there: the parameter must not move
        g64 = gk.astype(np.float64)
        ht.ht_mlp_adam_step(net, torch.from_numpy(gk).cuda(), lr)
        m0, v0 = m.copy(), v.copy()
        oracle.adam_step(po, g64, m, v, lr, b1=b1, b2=b2, eps=eps, step=k)
        # moments b m + (1 - b) g and b v + (1 - b) g g (1 - b is exact in
        # FP32): one rounding per product and per sum, on top of the
        # previous step's error scaled by b
        em = b1 * em + u * (b1 * np.abs(m0) + (1 - b1) * np.abs(g64) + np.abs(m)) * 1.01
        ev = b2 * ev + u * (b2 * v0 + 2 * (1 - b2) * g64 * g64 + v) * 1.01
        c1, c2 = 1 - b1 ** k, 1 - b2 ** k
        mh, vh = m / c1, v / c2
        D = np.sqrt(vh) + eps
        upd = np.abs(mh) / D
        rel = 20 * u  # two divisions, sqrt, the eps sum, the product by lr, and c1, c2 rounded once each
        dsq = np.where(v > 0, (ev / c2 + vh * 4 * u) / (2 * np.sqrt(np.maximum(vh, 1e-300))), 0.0)
        dupd = rel * upd + (em / c1) / D + upd * dsq / D
        ep = ep + lr * dupd + 2 * u * (np.abs(po) + lr * upd)
        pg = ht.ht_mlp_get_params(net).astype(np.float64)
        mg, vg, step = ht.ht_mlp_get_moments(net)
        assert step == k
        assert np.all(np.abs(mg - m) <= em), k
        assert np.all(np.abs(vg - v) <= ev), k
        bad = np.flatnonzero(np.abs(pg - po) > ep)
        assert bad.size == 0, (k, bad[:5], (pg - po)[bad[:5]], ep[bad[:5]])
        assert np.array_equal(pg[::97], p[::97].astype(np.float64))
    # the products use the BF16 rounding of the updated masters: a forward
    # pass through the GPU network equals one through a network set to them
    x = torch.from_numpy((synth.SplitMix64(3).uniform(64 * 16).reshape(64, 16) - 0.5).astype(np.float32)).cuda()
    y1 = torch.empty((64, 2), dtype=torch.float32, device="cuda")
    y2 = torch.empty_like(y1)
    ht.ht_mlp_forward(net, 64, x, y1)
    ht.ht_mlp_forward(_net(ht, ht.ht_mlp_get_params(net)), 64, x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_train_continues_adam_across_calls(ht):
    """Two ht_mlp_train calls of one epoch each equal one call of two epochs:
    the step count behind the bias correction lives in the network."""
    n = 512
    rng = synth.SplitMix64(77)
    x = torch.from_numpy((rng.uniform(n * 16).reshape(n, 16) * 2 - 1).astype(np.float32)).cuda()
    t = torch.from_numpy((rng.uniform(n * 2).reshape(n, 2) - 0.5).astype(np.float32)).cuda()
    p = _rand_params(14)
    a, b = _net(ht, p), _net(ht, p)
    ht.ht_mlp_train(a, n, x, t, 1, 128, 1e-3)
    ht.ht_mlp_train(a, n, x, t, 1, 128, 1e-3)
    ht.ht_mlp_train(b, n, x, t, 2, 128, 1e-3)
    assert np.array_equal(ht.ht_mlp_get_params(a), ht.ht_mlp_get_params(b))
    assert ht.ht_mlp_get_moments(a)[2] == ht.ht_mlp_get_moments(b)[2] == 8


def test_training_fits_a_teacher_network(ht):
    """Adam on the GPU drives the loss of a student well below its start on
    targets produced by a random teacher network."""
    n = 16384
    rng = synth.SplitMix64(21)
    x = (rng.uniform(n * 16).reshape(n, 16) * 2 - 1).astype(np.float32)
    teacher = _rand_params(22, 0.25).astype(np.float64)
    tgt = oracle.mlp_forward(x.astype(np.float64), teacher).astype(np.float32)
    from paper_1505_00383_gb300 import learned
    net = _net(ht, learned.init_params(3))
    losses = ht.ht_mlp_train(net, n, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(), 40, 1024, 3e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.1 * losses[0], losses


def test_zero_network_tracks_exactly_like_the_plain_rule(ht):
    """rho = 0 proposes the plain rule's step, so the learned path machinery
    reproduces the plain tracker bitwise."""
    from paper_1505_00383_gb300 import learned
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    prm = ht.ht_default_params(1, h_min=1e-6)
    plain = learned.track(s, 1, gam, 64, prm)
    net = _net(ht, np.zeros(5378, np.float32))
    lrn = learned.track(s, 1, gam, 64, prm, net=net)
    assert np.array_equal(plain["x_end"], lrn["x_end"]) and np.array_equal(plain["status"], lrn["status"])
    assert plain["stats"]["newton"] == lrn["stats"]["newton"]


def test_restart_from_recorded_states_reproduces_the_run(ht):
    """A path restarted from a recorded step start repeats the same arithmetic
    and ends where the uninterrupted run ended, bitwise."""
    from paper_1505_00383_gb300 import learned
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    prm = ht.ht_default_params(1, h_min=1e-6)
    full = learned.track(s, 1, gam, 64, prm)
    rec = learned.collect_records(s, 1, gam, 64, prm, stride=5)
    assert rec.shape[0] > 64
    # the last record of each path
    pid = rec[:, 0].cpu().numpy().astype(int)
    last = np.array([np.nonzero(pid == p)[0].max() for p in range(64)])
    sub = rec[torch.from_numpy(last).cuda()].contiguous()
    n = s.n_vars
    x = torch.empty((n, 2, 1, 64), dtype=torch.float64, device="cuda")
    st = torch.empty((64,), dtype=torch.int8, device="cuda")
    t = torch.empty((64,), dtype=torch.float64, device="cuda")
    io = ht.ht_track_io(init_records=sub.data_ptr())
    ht.ht_track_paths_ex(ht.system_from(s, 1), s.degrees(), gam, 64, 0, None, prm, x, st, t, io=io)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), full["status"])
    assert np.array_equal(x.cpu().numpy(), full["x_end"])


def test_features_follow_their_definition(ht):
    from paper_1505_00383_gb300 import learned
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    prm = ht.ht_default_params(1, h_min=1e-6)
    rec = learned.collect_records(s, 1, gam, 16, prm, stride=3)
    f = learned.features(s, 1, prm, rec).cpu().numpy()
    r = rec.cpu().numpy()
    cap, n = 5, 6
    for k in range(0, r.shape[0], 7):
        t, h, nh = r[k, 1], r[k, 2], int(r[k, 3])
        tv = r[k, 16:16 + cap]
        hx = r[k, 16 + cap:].reshape(cap, n, 2, 1)
        xs = hx[:, :, 0, 0] + 1j * hx[:, :, 1, 0]
        dxdt, f9, f10 = 0.0, 0.0, 0.0
        if nh >= 2:
            dt = tv[nh - 1] - tv[nh - 2]
            dxdt = np.max(np.abs(xs[nh - 1] - xs[nh - 2])) / dt
            f10 = np.log10(h / dt) / 2
        if nh >= 3 and tv[nh - 1] > tv[nh - 2] > tv[nh - 3]:
            a = (xs[nh - 1] - xs[nh - 2]) / (tv[nh - 1] - tv[nh - 2]) - (xs[nh - 2] - xs[nh - 3]) / (tv[nh - 2] - tv[nh - 3])
            f9 = np.log10(2 * np.max(np.abs(a)) / (tv[nh - 1] - tv[nh - 3]) + 1e-30) / 8
        ref = [t, np.log10(h), np.log10(dxdt + 1e-30) / 4, np.log10(r[k, 4] + 1e-300) / 16,
               np.log10(r[k, 5] + 1e-300) / 16, r[k, 6] / prm.newton_max, r[k, 7], nh / cap,
               np.log10(1 - t + 1e-16) / 16, f9, f10]
        ref = np.clip(ref, -4, 4)
        assert np.allclose(f[k, :11], ref, rtol=1e-5, atol=1e-5), (k, f[k, :11], ref)
        assert np.all(f[k, 11:] == 0)


def test_labels_follow_their_definition(ht):
    """Each record is probed once per multiplier (one step, the tracker's
    round limit); the label is the log of the accepted multiplier with the
    most progress per Newton round, ties to the larger (the smallest if none
    was accepted), and the tangent correction toward that probe's corrected
    point.  Probes re-run here one multiplier at a time; the predictor is
    re-derived from the record in numpy."""
    from paper_1505_00383_gb300 import learned
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    prm = ht.ht_default_params(1, h_min=1e-6)
    rec = learned.collect_records(s, 1, gam, 32, prm, stride=3)
    rec = rec[::5].contiguous()
    lab = learned.step_labels(s, 1, gam, prm, rec).cpu().numpy()
    R = rec.shape[1]
    n_rec = rec.shape[0]
    t0 = rec[:, 1].cpu().numpy()
    acc = np.zeros((n_rec, len(learned.MULTS)), bool)
    rounds = np.zeros((n_rec, len(learned.MULTS)), np.int64)
    ends = np.zeros((n_rec, len(learned.MULTS), s.n_vars), complex)
    hs = ht.system_from(s, 1)
    pp = ht.ht_default_params(1, h_min=1e-300, max_steps=1, polish_max=0)
    for j, mu in enumerate(learned.MULTS):
        r = rec.clone()
        r[:, 2] *= mu
        x = torch.empty((s.n_vars, 2, 1, n_rec), dtype=torch.float64, device="cuda")
        st = torch.empty((n_rec,), dtype=torch.int8, device="cuda")
        t = torch.empty((n_rec,), dtype=torch.float64, device="cuda")
        k = torch.empty((n_rec,), dtype=torch.int32, device="cuda")
        io = ht.ht_track_io(init_records=r.data_ptr(), newton_out=k.data_ptr())
        ht.ht_track_paths_ex(hs, s.degrees(), gam, n_rec, 0, None, pp, x, st, t, None, None, io)
        torch.cuda.synchronize()
        acc[:, j] = t.cpu().numpy() > t0
        rounds[:, j] = k.cpu().numpy()
        xe = x.cpu().numpy()
        ends[:, j] = (xe[:, 0, 0, :] + 1j * xe[:, 1, 0, :]).T
    assert acc.any() and (~acc).any() and np.all(rounds >= 1) and np.all(rounds <= prm.newton_max)
    recs = rec.cpu().numpy()
    cap, n = prm.max_order + 1, s.n_vars
    n_alpha = 0
    for q in range(n_rec):
        best, eff, jb = None, -1.0, -1
        for j, mu in enumerate(learned.MULTS):
            if acc[q, j] and (mu / rounds[q, j] > eff or (mu / rounds[q, j] == eff and mu > best)):
                best, eff, jb = mu, mu / rounds[q, j], j
        want = np.float32(np.log(best if best is not None else min(learned.MULTS)))
        assert lab[q, 0] == want, (q, lab[q], want, acc[q], rounds[q])
        alpha = 0.0
        if jb >= 0:  # tangent correction toward the chosen probe's corrected point
            r = recs[q]
            t, h, nh = r[1], r[2], int(r[3])
            tv = r[16:16 + cap]
            hx = r[16 + cap:].reshape(cap, n, 2)
            step = min(h * best, 1.0 - t)
            t1 = 1.0 if step >= 1.0 - t else t + step
            mm = min(nh, cap)
            base = nh - mm
            w = [np.prod([(t1 - tv[base + i]) / (tv[base + j] - tv[base + i]) for i in range(mm) if i != j])
                 for j in range(mm)]
            pred = sum(w[j] * (hx[base + j, :, 0] + 1j * hx[base + j, :, 1]) for j in range(mm))
            xc = hx[nh - 1, :, 0] + 1j * hx[nh - 1, :, 1]
            d = pred - xc
            nrm = np.sum(np.abs(d) ** 2)
            alpha = float(np.clip(np.sum((np.conj(d) * (ends[q, jb] - pred)).real) / nrm, -1, 1)) if nrm > 0 else 0.0
            n_alpha += alpha != 0.0
        assert abs(lab[q, 1] - alpha) <= 1e-5 + 1e-4 * abs(alpha), (q, lab[q, 1], alpha)
    assert n_alpha > 0


def test_trained_network_gains_over_the_plain_rule(ht):
    """Train on step-start records of training systems (labels: the step
    each state allowed at the least cost per round), then track held-out systems: the learned step
    needs fewer Newton rounds than the plain rule, with the same endpoint set
    and the same counts of converged, failed and diverged paths -- as the
    plain GPU tracker, and on a sample of paths as the oracle's tracker."""
    from paper_1505_00383_gb300 import learned
    cfg = synth.CONFIGS["learned_n16_d"]
    prm = ht.ht_default_params(1, h_min=1e-9)
    feats, labs = [], []
    for seed in range(cfg["train_seeds"][0], cfg["train_seeds"][0] + 6):
        s = synth.config_system("learned_n16_d", seed)
        gam = synth.random_gamma(seed)
        rec = learned.collect_records(s, 1, gam, 256, prm, stride=2)
        labs.append(learned.step_labels(s, 1, gam, prm, rec))
        feats.append(learned.features(s, 1, prm, rec))
    net, losses = learned.train(torch.cat(feats), torch.cat(labs), epochs=30, batch=2048, lr=2e-3)
    assert losses[-1] < losses[0]
    tot_plain = tot_learn = 0
    for seed in range(cfg["heldout_seeds"][0], cfg["heldout_seeds"][0] + 2):
        s = synth.config_system("learned_n16_d", seed)
        gam = synth.random_gamma(seed)
        a = learned.track(s, 1, gam, 512, prm)
        b = learned.track(s, 1, gam, 512, prm, net=net)
        for code in (1, -1, -2):
            assert np.sum(a["status"] == code) == np.sum(b["status"] == code)
        ok, worst = match_sets(to_complex(a["x_end"])[a["status"] == 1], to_complex(b["x_end"])[b["status"] == 1],
                               1e-10)
        assert ok, worst
        # and against the oracle's plain tracker on the first 64 paths
        o = oracle.track(s, s.degrees(), gam, np.arange(64), 1, oracle.default_params(1, h_min=1e-9))
        for code in (1, -1, -2):
            assert np.sum(o["status"] == code) == np.sum(b["status"][:64] == code)
        ok, worst = match_sets(to_complex(o["x_end"])[o["status"] == 1],
                               to_complex(b["x_end"][..., :64])[b["status"][:64] == 1], 1e-10)
        assert ok, worst
        tot_plain += a["stats"]["newton"]
        tot_learn += b["stats"]["newton"]
    assert tot_learn < 0.95 * tot_plain, (tot_learn, tot_plain)


def test_learned_step_with_wide_teams_gives_the_same_bits(ht):
    """The learned step in the 16-warp instantiation (which the tracker takes
    while fewer groups than SMs are active, and the autotuner may choose)
    tracks exactly as with 8 warps."""
    from paper_1505_00383_gb300 import learned
    s = synth.config_system("learned_n16_d")
    gam = synth.random_gamma(5)
    net = _net(ht, learned.init_params(9))
    out = {}
    for tw in (8, 16):
        prm = ht.ht_default_params(1, h_min=1e-9, team_warps=tw)
        out[tw] = learned.track(s, 1, gam, 96, prm, net=net)
    assert np.array_equal(out[8]["x_end"], out[16]["x_end"]) and np.array_equal(out[8]["status"], out[16]["status"])
    assert out[8]["stats"]["newton"] == out[16]["stats"]["newton"]
