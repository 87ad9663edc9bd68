"""Parity of the CUDA tracker stages and of whole-path tracking with the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from certify import certify_roots
from match import match_sets, to_complex
from parity import TOL, cerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ht():
    from paper_1505_00383_gb300 import _build, ht as binding
    _build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return binding


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


# ---------------------------------------------------------------- stages
@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("degrees", [[2, 2, 2], [3, 2], [5, 3, 4]])
def test_start_solutions_match_oracle(ht, L, degrees):
    count = int(np.prod(degrees))
    x = torch.full((len(degrees), 2, L, count), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_start_solutions(len(degrees), degrees, L, 0, count, x)
    ref = oracle.start_solutions(degrees, 0, count, L)
    e = cerr(x.cpu().numpy(), ref)
    assert np.max(e) <= {1: 4e-16, 2: 1e-31, 4: 1e-62}[L], np.max(e)


@pytest.mark.parametrize("L,variant", [(1, 0), (2, 0), (4, 0), (2, 2), (4, 2)])
@pytest.mark.parametrize("rows,cols", [(6, 6), (12, 12), (9, 5), (1, 1)])
def test_mgs_solve_matches_oracle(ht, L, variant, rows, cols):
    """Both arithmetics against the oracle's MGS, within the conditioning
    bound at the variant's unit (2^-53L; for QD integer limbs the 204 bits a
    product keeps)."""
    _mgs_case(ht, L, variant, rows, cols, 37)  # a full warp of systems and a ragged tail


@pytest.mark.parametrize("L,variant", [(1, 0), (2, 2), (4, 2)])
def test_mgs_solve_at_the_integer_row_limit(ht, L, variant):
    """64 x 64, the largest system the integer variant takes (33 systems: a
    warp and a ragged tail); 65 rows are refused with HT_EUNSUPPORTED."""
    _mgs_case(ht, L, variant, 64, 64, 33)
    if variant == 2:
        buf = torch.zeros((65, 66, 2, L, 1), dtype=torch.float64, device="cuda")
        with pytest.raises(ht.HTError) as e:
            ht.ht_mgs_solve_ex(L, 2, 65, 65, 1, buf, buf, buf)
        assert e.value.code == ht.HT_EUNSUPPORTED


def _mgs_case(ht, L, variant, rows, cols, n_sys):
    rng = synth.SplitMix64(300 + rows * 7 + cols + L)
    re, im = synth.unit_circle(rng, n_sys * rows * (cols + 1))
    mag = rng.uniform(re.size) + 0.5
    Ab = np.zeros((rows, cols + 1, 2, L, n_sys))
    Ab[:, :, 0] = synth.random_tails(rng, (re * mag).reshape(rows, cols + 1, n_sys), L).transpose(1, 2, 0, 3)
    Ab[:, :, 1] = synth.random_tails(rng, (im * mag).reshape(rows, cols + 1, n_sys), L).transpose(1, 2, 0, 3)
    A_or = np.ascontiguousarray(Ab[:, :cols].transpose(4, 0, 1, 2, 3))
    b_or = np.ascontiguousarray(Ab[:, cols].transpose(3, 0, 1, 2))
    ref = oracle.mgs_solve(A_or, b_or)  # [n_sys][cols][2][L]
    dAb = dev(Ab)
    dR = torch.empty((cols, cols + 1, 2, L, n_sys), dtype=torch.float64, device="cuda")
    dx = torch.empty((cols, 2, L, n_sys), dtype=torch.float64, device="cuda")
    ht.ht_mgs_solve_ex(L, variant, rows, cols, n_sys, dAb, dR, dx)
    torch.cuda.synchronize()
    got = dx.cpu().numpy()
    unit = 2.0 ** (-53 * L) if variant == 0 else 2.0 ** -min(53 * L, 29 * ({2: 5, 4: 8}[L] - 1) + 1)
    refv = np.ascontiguousarray(ref.transpose(1, 2, 3, 0))
    for s in range(n_sys):
        Ad = Ab[:, :cols, 0, 0, s] + 1j * Ab[:, :cols, 1, 0, s]
        cond = np.linalg.cond(Ad)
        scale = np.max(np.abs(refv[:, 0, 0, s] + 1j * refv[:, 1, 0, s]))
        e = np.max(cerr(got[..., s:s + 1], refv[..., s:s + 1]))
        assert e <= 64 * cond * cond * unit * scale * rows, (s, e, cond)


def test_compaction_table_tabjobidx(ht):
    g = json.load(open(os.path.join(GOLDEN, "tabjobidx.json")))
    st = dev(np.array(g["status"], np.int8))
    idx = torch.full((5,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((1,), dtype=torch.int32, device="cuda")
    ht.ht_compact(st, 5, idx, cnt)
    c = int(cnt.item())
    assert c == g["active_count"]
    assert idx[:c].cpu().tolist() == g["path_idx"]


@pytest.mark.parametrize("m", [1, 31, 1024, 1025, 70000])
def test_compaction_random_matches_oracle(ht, m):
    rng = synth.SplitMix64(m)
    st = (rng.integers(0, 3, m) - 1).astype(np.int8)
    idx = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((1,), dtype=torch.int32, device="cuda")
    ht.ht_compact(dev(st), m, idx, cnt)
    _, ref = oracle.compact(st)
    c = int(cnt.item())
    assert c == ref.size and np.array_equal(idx[:c].cpu().numpy(), ref)


# ---------------------------------------------------------------- tracking
def _oracle_params(L, **over):
    return oracle.default_params(L, **over)


def _gpu_params(ht, L, **over):
    return ht.ht_default_params(L, **over)


def track_gpu(ht, system, L, m, first=0, start_deg=None, gamma=(0.6, 0.8), eval_variant=None, **over):
    n = system.n_vars
    deg = system.degrees() if start_deg is None else np.asarray(start_deg, np.int32)
    hs = ht.system_from(system, L)
    if eval_variant is not None:
        ht.ht_set_eval_config(hs, eval_variant, 0)
    x = torch.full((n, 2, L, m), np.nan, dtype=torch.float64, device="cuda")
    status = torch.full((m,), 9, dtype=torch.int8, device="cuda")
    t = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    steps = torch.zeros((m,), dtype=torch.int32, device="cuda")
    stats = ht.ht_stats()
    ht.ht_track_paths(hs, deg, gamma, m, first, None, _gpu_params(ht, L, **over), x, status, t, steps, stats)
    torch.cuda.synchronize()
    return dict(x_end=x.cpu().numpy(), status=status.cpu().numpy(), t_end=t.cpu().numpy(),
                steps=steps.cpu().numpy(), stats=stats.as_dict())


def track_oracle(system, L, ids, start_deg=None, gamma=(0.6, 0.8), **over):
    deg = system.degrees() if start_deg is None else np.asarray(start_deg, np.int32)
    return oracle.track(system, deg, gamma, np.asarray(ids, np.int64), L, _oracle_params(L, **over))


def assert_same_outcome(g, o, tol=1e-10):
    """Equal counts of converged, failed and diverged paths; the converged
    endpoints agree as sets to tol (relative to max(1, |x|))."""
    for code in (1, -1, -2):
        assert int(np.sum(g["status"] == code)) == int(np.sum(o["status"] == code)), (code, g["status"], o["status"])
    conv_g = to_complex(g["x_end"])[g["status"] == 1]
    conv_o = to_complex(o["x_end"])[o["status"] == 1]
    ok, worst = match_sets(conv_g, conv_o, tol)
    assert ok, worst


@pytest.mark.parametrize("L", [1, 2, 4])
def test_diagonal_system_closed_form(ht, L):
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    exps, coef = [], []
    for i, ci in enumerate(c):
        a = [0, 0, 0]
        a[i] = 2
        exps += [a, [0, 0, 0]]
        coef += [[1.0, 0.0], [-ci.real, -ci.imag]]
    s = synth.System(3, 3, np.full(3, 2, np.int32), np.array(exps, np.int8), np.array(coef))
    g = track_gpu(ht, s, L, 8)
    assert np.all(g["status"] == 1) and np.all(g["t_end"] == 1.0)
    r = np.sqrt(c)
    expect = np.array([[r[0] * (1 - 2 * ((p >> 0) & 1)), r[1] * (1 - 2 * ((p >> 1) & 1)),
                        r[2] * (1 - 2 * ((p >> 2) & 1))] for p in range(8)])
    ok, worst = match_sets(to_complex(g["x_end"]), expect, 1e-13)
    assert ok, worst
    o = track_oracle(s, L, np.arange(8))
    assert_same_outcome(g, o)
    # per path, the same endpoint as the oracle to working precision
    e = cerr(g["x_end"], o["x_end"])
    assert np.max(e) <= {1: 1e-13, 2: 1e-26, 4: 1e-50}[L]


@pytest.mark.parametrize("h_min", [0.01, 1e-6])
def test_plain_tracker_n6_matches_oracle(ht, h_min):
    """64 paths of the n = 6 total-degree homotopy in complex double, with the
    step range 0.01-0.1 of the workload and with a small step floor."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    g = track_gpu(ht, s, 1, 64, gamma=gam, h_min=h_min)
    o = track_oracle(s, 1, np.arange(64), gamma=gam, h_min=h_min)
    assert_same_outcome(g, o)
    assert np.array_equal(g["status"], o["status"])
    assert np.array_equal(g["steps"], o["steps"])
    st = g["stats"]
    assert st["converged"] == np.sum(o["status"] == 1) and st["steps"] == int(np.sum(o["steps"]))
    assert st["newton"] == int(np.sum(o["newton"])) and st["rejects"] == int(np.sum(o["rejects"]))


def test_team_size_and_launch_shape_do_not_change_results(ht):
    """Every team size splits the same arithmetic differently over warps but
    in the same order, so results are bitwise identical."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    base = track_gpu(ht, s, 1, 64, gamma=gam, team_warps=1, iters_per_launch=1, rounds_per_sync=2)
    for tw, it, rs in ((2, 4, 8), (4, 3, 4), (8, 7, 6), (0, 0, 0)):
        r = track_gpu(ht, s, 1, 64, gamma=gam, team_warps=tw, iters_per_launch=it, rounds_per_sync=rs)
        for k in ("x_end", "status", "t_end", "steps"):
            assert np.array_equal(r[k], base[k], equal_nan=True), (tw, it, rs, k)


@pytest.mark.parametrize("L", [2, 4])
def test_team_size_does_not_change_integer_evaluation_results(ht, L):
    """With f on the integer pipe each lane's arithmetic is the same for any
    split of polynomials and MGS columns over the team's warps."""
    s = synth.config_system("stress_n10_qd" if L == 4 else "batched_n12_dd")
    gam = synth.random_gamma(1)
    base = track_gpu(ht, s, L, 96, gamma=gam, team_warps=1, iters_per_launch=2, rounds_per_sync=2)
    for tw in (2, 8) + ((16,) if L == 2 else ()):  # 16 warps: the wide instantiation (D and DD)
        r = track_gpu(ht, s, L, 96, gamma=gam, team_warps=tw)
        for k in ("x_end", "status", "t_end", "steps"):
            assert np.array_equal(r[k], base[k], equal_nan=True), (tw, k)


def test_sharded_path_ranges_union_equals_full_run(ht):
    """Paths are independent (Section 1): tracking path ranges separately (as
    separate GPUs would) gives the full run's results."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    full = track_gpu(ht, s, 1, 64, gamma=gam, h_min=1e-6)
    parts = [track_gpu(ht, s, 1, 24, first=0, gamma=gam, h_min=1e-6),
             track_gpu(ht, s, 1, 40, first=24, gamma=gam, h_min=1e-6)]
    x = np.concatenate([p["x_end"] for p in parts], axis=-1)
    st = np.concatenate([p["status"] for p in parts])
    assert np.array_equal(x, full["x_end"]) and np.array_equal(st, full["status"])


@pytest.mark.parametrize("name,L,m,sample,ev", [("batched_n12_dd", 2, 4096, 48, None), ("batched_n12_dd", 2, 4096, 24, 1),
                                              ("stress_n10_qd", 4, 1024, 16, None), ("stress_n10_qd", 4, 512, 8, 1)])
def test_batched_tracker_sampled_paths_match_oracle(ht, name, L, m, sample, ev):
    """The batched tracker on the workload shape (all 4,096 DD paths; 1,024 of
    the QD paths), with f evaluated on the integer pipe (the default for DD
    and QD) or on the FP64 pipe (ev = 1); a seeded sample of paths is
    re-tracked one by one by the oracle and must end with the same status and
    endpoint."""
    s = synth.config_system(name)
    gam = synth.random_gamma(synth.CONFIGS[name]["seed"])
    g = track_gpu(ht, s, L, m, gamma=gam, h_min=1e-6, eval_variant=ev)
    assert set(np.unique(g["status"])) <= {1, -1, -2}
    assert g["stats"]["converged"] + g["stats"]["failed"] + g["stats"]["diverged"] == m
    rng = synth.SplitMix64(7)
    ids = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m - 1, sample)]))
    o = track_oracle(s, L, ids, gamma=gam, h_min=1e-6)
    sub = dict(x_end=g["x_end"][..., ids], status=g["status"][ids])
    assert np.array_equal(sub["status"], o["status"]), (sub["status"], o["status"])
    conv = o["status"] == 1
    e = cerr(sub["x_end"][..., conv], o["x_end"][..., conv])
    scale = np.maximum(1.0, np.max(np.abs(to_complex(o["x_end"][..., conv])), axis=1))
    assert np.all(np.max(e, axis=0) / scale <= 1e-10)


@pytest.mark.parametrize("name,L", [("batched_n12_dd", 2), ("learned_n16_d", 1), ("stress_n10_qd", 4)])
def test_full_workload_ends_at_all_roots(ht, name, L):
    """Every path of the workload (4,096 DD, 65,536 D, 59,049 QD), in the
    tracker's default launch shape at the step floor 1e-9: all converge, and
    the GPU's endpoints carry a Kantorovich certificate of prod(d_i) distinct
    isolated roots -- by Bezout all the roots, one per path."""
    cfg = synth.CONFIGS[name]
    s = synth.config_system(name)
    m = cfg["degree"] ** cfg["n"]
    g = track_gpu(ht, s, L, m, gamma=synth.random_gamma(cfg["seed"]), h_min=1e-9)
    assert np.all(g["status"] == 1) and g["stats"]["converged"] == m
    assert np.all(g["t_end"] == 1.0)
    cert = certify_roots(s, to_complex(g["x_end"]))
    assert cert["distinct_roots"] == m, cert


@pytest.mark.parametrize("n", [20, 32, 33])
def test_tracker_at_the_integer_evaluation_limit(ht, n):
    """n = 32 is the largest system whose DD and QD tracking evaluates on
    integer limbs (QD also solves on them, and DD asks for exactly 48 KB of
    dynamic shared memory); n = 33 switches to the FP64 bodies; at n = 20 the
    QD kernel's dynamic shared memory is under 48 KB but, with its static
    shared memory, over the default limit.  The last 8
    of the 2^n paths (path indices past 2^32): DD against the oracle path by
    path; at n = 32, QD ends at the same roots with residuals at its own
    precision (the oracle's exact evaluation).  QD on FP64 bodies is covered
    at n = 10 (ev = 1 above); eight paths of it at n = 33 take minutes."""
    s = synth.total_degree_system(500 + n, n, 2, 4)
    m = 8
    first = 2 ** n - m
    gam = synth.random_gamma(n)
    g2 = track_gpu(ht, s, 2, m, first=first, gamma=gam, h_min=1e-6)
    o2 = track_oracle(s, 2, np.arange(first, first + m), gamma=gam, h_min=1e-6)
    assert np.array_equal(g2["status"], o2["status"]), (g2["status"], o2["status"])
    conv = o2["status"] == 1
    assert conv.sum() >= m // 2
    scale = np.maximum(1.0, np.max(np.abs(to_complex(o2["x_end"][..., conv])), axis=1))
    e = cerr(g2["x_end"][..., conv], o2["x_end"][..., conv])
    assert np.all(np.max(e, axis=0) / scale <= 1e-10)
    if n > 32:
        return
    g4 = track_gpu(ht, s, 4, m, first=first, gamma=gam, h_min=1e-6)
    assert np.array_equal(g4["status"], o2["status"])
    d = np.abs(to_complex(g4["x_end"])[conv] - to_complex(g2["x_end"])[conv])
    assert np.all(np.max(d, axis=1) / scale <= 1e-10)
    pts = np.nonzero(conv)[0]
    val, _ = oracle.eval_(s, g4["x_end"], pts=pts)
    mag, _ = oracle.eval_magnitude(s, g4["x_end"], pts=pts)
    res = np.hypot(val[:, 0, 0], val[:, 1, 0]) / mag
    assert np.max(res) <= 1e-40, np.max(res)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("h_max", [0.1, 0.005])
def test_deficient_system_matches_oracle_path_by_path(ht, L, h_max):
    """Bezout number 4, one finite root: paths that diverge past r_div, fail,
    or (with the default step cap) jump onto the root's path -- the same
    outcome as the oracle for every path, including where it ended."""
    s = synth.deficient_system()
    gam = synth.random_gamma(5)
    over = dict(r_div=1e4, h_min=1e-8, h_max=h_max)
    g = track_gpu(ht, s, L, 4, gamma=gam, **over)
    o = track_oracle(s, L, np.arange(4), gamma=gam, **over)
    assert np.array_equal(g["status"], o["status"]), (g["status"], o["status"])
    assert np.sum(g["status"] == 1) == (1 if h_max < 0.01 else 3)
    conv = o["status"] == 1
    e = cerr(g["x_end"][..., conv], o["x_end"][..., conv])
    assert np.max(e) <= 1e-10
    assert np.all(g["t_end"][~conv] > 0.999)  # the others leave near t = 1


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("case", ["growth", "update", "residual"])
def test_step_control_worked_examples(ht, L, case):
    """The step rule on the hand-derived examples of the oracle pins (linear
    homotopy g = x - 1, f = 2x - 3): 11 accepted steps without rejection;
    with one Newton round and tol_dx = 0.03, 2 steps with 1 rejection
    (tol_res = 1) or 8 steps with 7 rejections (tol_res = 1e-4)."""
    s = synth.System(1, 1, np.array([2], np.int32), np.array([[1], [0]], np.int8),
                     np.array([[2.0, 0.0], [-3.0, 0.0]]))
    over, want = {}, (1, 11, 0, 1.0)
    if case != "growth":
        tol_res, max_steps, rej = (1.0, 2, 1) if case == "update" else (1e-4, 8, 7)
        over = dict(newton_max=1, tol_dx=0.03, tol_res=tol_res, f_down=0.4, max_steps=max_steps)
        h = 0.05
        for _ in range(rej):
            h = 0.4 * h
        want = (-1, max_steps, rej, h)
    g = track_gpu(ht, s, L, 1, start_deg=[1], gamma=synth.random_gamma(8), **over)
    got = (int(g["status"][0]), int(g["steps"][0]), int(g["stats"]["rejects"]), float(g["t_end"][0]))
    assert got == want, (got, want)


def test_tracker_rejects_bad_arguments(ht):
    s = synth.config_system("plain_n6_d")
    hs = ht.system_from(s, 1)
    x = torch.zeros((6, 2, 1, 4), dtype=torch.float64, device="cuda")
    st = torch.zeros((4,), dtype=torch.int8, device="cuda")
    t = torch.zeros((4,), dtype=torch.float64, device="cuda")
    with pytest.raises(ht.HTError):  # zero gamma
        ht.ht_track_paths(hs, [2] * 6, (0.0, 0.0), 4, 0, None, None, x, st, t)
    with pytest.raises(ht.HTError):  # host output
        ht.ht_track_paths(hs, [2] * 6, (1.0, 0.0), 4, 0, None, None, x.cpu(), st, t)
    with pytest.raises(ht.HTError):  # odd rounds_per_sync
        ht.ht_track_paths(hs, [2] * 6, (1.0, 0.0), 4, 0, None, ht.ht_default_params(1, rounds_per_sync=3), x, st, t)
    with pytest.raises(ht.HTError):  # non-square system
        rect = synth.System(6, 5, s.n_terms[:5], s.exps[:40], s.coef[:40])
        ht.ht_track_paths(ht.system_from(rect, 1), [2] * 6, (1.0, 0.0), 4, 0, None, None, x, st, t)
    ht.ht_track_paths(hs, [2] * 6, (1.0, 0.0), 0, 0, None, None, x, st, t)  # no paths: no-op


@pytest.mark.parametrize("L", [2, 4])
def test_endpoint_check_in_higher_precision_matches_oracle(ht, L):
    """Complex double tracking, then Newton on f alone in DD / QD from the
    double endpoints (polish_only, x0 with one limb): every path gives the
    oracle's own DD / QD endpoint of that path to working precision, and the
    last update is at the precision's level."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    m = 64
    g = track_gpu(ht, s, 1, m, gamma=gam, h_min=1e-9)
    conv = g["status"] == 1
    hs = ht.system_from(s, L)
    x0 = dev(g["x_end"])
    x = torch.full((s.n_vars, 2, L, m), np.nan, dtype=torch.float64, device="cuda")
    st = torch.full((m,), 9, dtype=torch.int8, device="cuda")
    t = torch.zeros((m,), dtype=torch.float64, device="cuda")
    ldx = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    io = ht.ht_track_io(x0_limbs=1, polish_only=1, last_dx_out=ldx.data_ptr())
    ht.ht_track_paths_ex(hs, s.degrees(), gam, m, 0, x0, ht.ht_default_params(L, polish_max=6), x, st, t, None,
                         None, io)
    torch.cuda.synchronize()
    xc, sc, dxc = x.cpu().numpy(), st.cpu().numpy(), ldx.cpu().numpy()
    assert np.all(sc[conv] == 1) and np.all(t.cpu().numpy() == 1.0)
    assert np.max(dxc[conv]) <= {2: 1e-24, 4: 1e-48}[L]
    o = track_oracle(s, L, np.arange(m), gamma=gam, h_min=1e-9)
    # paths that reach the same root in the double run and the oracle's run
    both = conv & (o["status"] == 1)
    d = np.max(np.abs(to_complex(g["x_end"]) - to_complex(o["x_end"])), axis=1)
    same = both & (d <= 1e-8)
    assert same.sum() >= both.sum() - 2 and same.sum() > 0
    e = cerr(xc[..., same], o["x_end"][..., same])
    assert np.max(e) <= {2: 1e-26, 4: 1e-50}[L], np.max(e)


def test_narrow_start_points_are_widened(ht):
    """x0 given in one limb for a DD system: the missing limbs are zero, so
    the start solutions of x_i^2 - 1 (exactly +-1) give the same paths as the
    system's own start solutions."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    m = 64
    a = track_gpu(ht, s, 2, m, gamma=gam, h_min=1e-9)
    x0 = torch.empty((s.n_vars, 2, 1, m), dtype=torch.float64, device="cuda")
    ht.ht_start_solutions(s.n_vars, s.degrees(), 1, 0, m, x0)
    hs = ht.system_from(s, 2)
    x = torch.full((s.n_vars, 2, 2, m), np.nan, dtype=torch.float64, device="cuda")
    st = torch.full((m,), 9, dtype=torch.int8, device="cuda")
    t = torch.zeros((m,), dtype=torch.float64, device="cuda")
    ht.ht_track_paths_ex(hs, s.degrees(), gam, m, 0, x0, ht.ht_default_params(2, h_min=1e-9), x, st, t, None, None,
                         ht.ht_track_io(x0_limbs=1))
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), a["status"])
    assert np.array_equal(x.cpu().numpy(), a["x_end"], equal_nan=True)


def test_endpoint_check_rejects_bad_arguments(ht):
    s = synth.config_system("plain_n6_d")
    hs = ht.system_from(s, 2)
    m = 4
    x = torch.zeros((6, 2, 2, m), dtype=torch.float64, device="cuda")
    x1 = torch.zeros((6, 2, 1, m), dtype=torch.float64, device="cuda")
    st = torch.zeros((m,), dtype=torch.int8, device="cuda")
    t = torch.zeros((m,), dtype=torch.float64, device="cuda")
    p = ht.ht_default_params(2)
    with pytest.raises(ht.HTError):  # polish_only without start points
        ht.ht_track_paths_ex(hs, [2] * 6, (1.0, 0.0), m, 0, None, p, x, st, t, None, None, ht.ht_track_io(polish_only=1))
    with pytest.raises(ht.HTError):  # more limbs than the system
        ht.ht_track_paths_ex(hs, [2] * 6, (1.0, 0.0), m, 0, x1, p, x, st, t, None, None, ht.ht_track_io(x0_limbs=4))
    with pytest.raises(ht.HTError):  # widening in place
        ht.ht_track_paths_ex(hs, [2] * 6, (1.0, 0.0), m, 0, x, p, x, st, t, None, None, ht.ht_track_io(x0_limbs=1))
    with pytest.raises(ht.HTError):  # no polish rounds
        ht.ht_track_paths_ex(hs, [2] * 6, (1.0, 0.0), m, 0, x1, ht.ht_default_params(2, polish_max=0), x, st, t, None,
                             None, ht.ht_track_io(polish_only=1, x0_limbs=1))


def test_track_autotuner_picks_a_valid_shape_and_keeps_results(ht):
    """ht_tune_track times every launch shape on a path sample and keeps the
    fastest in the system; tracking with the tuned defaults gives the same
    bits as any explicit shape."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    hs = ht.system_from(s, 1)
    p = ht.ht_default_params(1, h_min=1e-9)
    team, iters, ms = ht.ht_tune_track(hs, s.degrees(), gam, 64, p)
    assert team in (1, 2, 4) and iters in (2, 4, 8) and ms > 0
    m = 64
    out = []
    for tw, it in ((0, 0), (2, 4)):
        x = torch.full((s.n_vars, 2, 1, m), np.nan, dtype=torch.float64, device="cuda")
        st = torch.full((m,), 9, dtype=torch.int8, device="cuda")
        t = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
        ht.ht_track_paths(hs, s.degrees(), gam, m, 0, None, ht.ht_default_params(1, h_min=1e-9, team_warps=tw,
                                                                                 iters_per_launch=it), x, st, t)
        torch.cuda.synchronize()
        out.append((x.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0], equal_nan=True) and np.array_equal(out[0][1], out[1][1])


def _golden_track(name):
    import sys
    sys.path.insert(0, GOLDEN)
    import make_track_oracle as M
    d = np.load(M.path(name))
    return M, {k: d[k] for k in d.files}


@pytest.mark.parametrize("name", ["batched_n12_dd", "stress_n10_qd"])
def test_full_workload_matches_oracle_on_1024_sampled_paths(ht, name):
    """All paths of the workload (4,096 DD; 59,049 QD) tracked at once in the
    launch shape the benchmark times (DD: the built-in shape; QD: the
    autotuner's choice on 1,024 paths), against the oracle's one-by-one
    tracking of 1,024 seeded path indices (tests/golden, written by a script
    that calls only the oracle): the same status for every sampled path and
    the same endpoint to 1e-10 relative to max(1, |x|_inf)."""
    M, gold = _golden_track(name)
    L, h_min = M.CASES[name][0], M.CASES[name][1]
    cfg = synth.CONFIGS[name]
    s = synth.config_system(name)
    gam = synth.random_gamma(cfg["seed"])
    m = cfg["degree"] ** cfg["n"]
    hs = ht.system_from(s, L)
    prm = ht.ht_default_params(L, h_min=h_min)
    if name == "stress_n10_qd":
        team, iters, _ = ht.ht_tune_track(hs, s.degrees(), gam, 1024, prm)
        prm.team_warps, prm.iters_per_launch = team, iters
    n = s.n_vars
    x = torch.full((n, 2, L, m), np.nan, dtype=torch.float64, device="cuda")
    st = torch.full((m,), 9, dtype=torch.int8, device="cuda")
    t = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_track_paths(hs, s.degrees(), gam, m, 0, None, prm, x, st, t, None, None)
    torch.cuda.synchronize()
    ids = gold["ids"]
    assert ids.size == 1024 and ids[0] == 0 and ids[-1] == m - 1
    sg = st.cpu().numpy()[ids]
    assert np.array_equal(sg, gold["status"]), np.flatnonzero(sg != gold["status"])[:10]
    conv = gold["status"] == 1
    xg = x.cpu().numpy()[:, :, 0, :][..., ids]
    zg = (xg[:, 0] + 1j * xg[:, 1]).T[conv]
    zo = (gold["x_lead"][:, 0] + 1j * gold["x_lead"][:, 1]).T[conv]
    scale = np.maximum(1.0, np.max(np.abs(zo), axis=1))
    err = np.max(np.maximum(np.abs(zg.real - zo.real), np.abs(zg.imag - zo.imag)), axis=1) / scale
    assert np.all(err <= 1e-10), (np.max(err), ids[conv][np.argmax(err)])
    assert np.all(t.cpu().numpy()[ids][conv] == 1.0)


# ---- tangent predictors (Euler, cubic Hermite on J v = -dh/dt)
@pytest.mark.parametrize("pred", [1, 2])
def test_tangent_predictors_n6_match_oracle_path_by_path(ht, pred):
    """64 paths of the n = 6 system with the Euler (1) and Hermite (2)
    predictors: the same status, number of steps and endpoint as the oracle's
    tracker with the same predictor, path by path."""
    s = synth.config_system("plain_n6_d")
    gam = synth.random_gamma(0)
    g = track_gpu(ht, s, 1, 64, gamma=gam, h_min=1e-6, predictor=pred)
    o = track_oracle(s, 1, np.arange(64), gamma=gam, h_min=1e-6, predictor=pred)
    assert_same_outcome(g, o)
    assert np.array_equal(g["status"], o["status"])
    assert np.array_equal(g["steps"], o["steps"])


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("pred", [1, 2])
def test_tangent_predictors_diagonal_closed_form(ht, L, pred):
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    exps, coef = [], []
    for i, ci in enumerate(c):
        a = [0, 0, 0]
        a[i] = 2
        exps += [a, [0, 0, 0]]
        coef += [[1.0, 0.0], [-ci.real, -ci.imag]]
    s = synth.System(3, 3, np.full(3, 2, np.int32), np.array(exps, np.int8), np.array(coef))
    g = track_gpu(ht, s, L, 8, predictor=pred)
    assert np.all(g["status"] == 1)
    o = track_oracle(s, L, np.arange(8), predictor=pred)
    assert_same_outcome(g, o)
    e = cerr(g["x_end"], o["x_end"])
    assert np.max(e) <= {1: 1e-13, 2: 1e-26, 4: 1e-50}[L]


@pytest.mark.parametrize("name,L,m,sample", [("batched_n12_dd", 2, 4096, 16), ("stress_n10_qd", 4, 512, 4)])
def test_hermite_predictor_batched_sampled_paths_match_oracle(ht, name, L, m, sample):
    """The Hermite predictor on the workload shapes (integer-pipe evaluation;
    QD also solves both right-hand sides on the integer pipe): a seeded
    sample of paths tracked by the oracle ends with the same status and
    endpoint."""
    s = synth.config_system(name)
    gam = synth.random_gamma(synth.CONFIGS[name]["seed"])
    g = track_gpu(ht, s, L, m, gamma=gam, h_min=1e-6, predictor=2)
    rng = synth.SplitMix64(8)
    ids = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m - 1, sample)]))
    o = track_oracle(s, L, ids, gamma=gam, h_min=1e-6, predictor=2)
    assert np.array_equal(g["status"][ids], o["status"])
    conv = o["status"] == 1
    e = cerr(g["x_end"][..., ids][..., conv], o["x_end"][..., conv])
    scale = np.maximum(1.0, np.max(np.abs(to_complex(o["x_end"][..., conv])), axis=1))
    assert np.all(np.max(e, axis=0) / scale <= 1e-10)


@pytest.mark.parametrize("L", [1, 4])
def test_hermite_results_do_not_depend_on_the_launch_shape(ht, L):
    """Both right-hand sides are dealt to the team's warps; any team size
    gives the same bits."""
    s = synth.config_system("stress_n10_qd" if L == 4 else "plain_n6_d")
    gam = synth.random_gamma(1)
    base = track_gpu(ht, s, L, 96 if L == 4 else 64, gamma=gam, team_warps=1, iters_per_launch=2,
                     rounds_per_sync=2, predictor=2)
    for tw in (2, 8):
        r = track_gpu(ht, s, L, 96 if L == 4 else 64, gamma=gam, team_warps=tw, predictor=2)
        for k in ("x_end", "status", "t_end", "steps"):
            assert np.array_equal(r[k], base[k], equal_nan=True), (tw, k)


def test_wide_teams_give_the_same_bits_in_double(ht):
    """16-warp teams (the wide instantiation the tracker picks while fewer
    groups than SMs are active) against one-warp teams on the n = 16 double
    workload; QD refuses them."""
    s = synth.config_system("learned_n16_d")
    gam = synth.random_gamma(3)
    base = track_gpu(ht, s, 1, 64, gamma=gam, team_warps=1, iters_per_launch=3, rounds_per_sync=2)
    for tw in (16, 0):  # 0: the automatic choice, 16 here (2 groups)
        r = track_gpu(ht, s, 1, 64, gamma=gam, team_warps=tw)
        for k in ("x_end", "status", "t_end", "steps"):
            assert np.array_equal(r[k], base[k], equal_nan=True), (tw, k)
    q = synth.config_system("stress_n10_qd")
    with pytest.raises(ht.HTError) as e:
        track_gpu(ht, q, 4, 32, team_warps=16)
    assert e.value.code == ht.HT_EINVAL
