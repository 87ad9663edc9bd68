"""Pins for the oracle tracker (Section 2) on systems whose solutions are known
in closed form or from a textbook routine."""
import numpy as np
import pytest

import synth
from certify import certify_roots
from exact import Cx, cx_from, fr, poly_value
from fractions import Fraction as Fr
from match import match_sets, to_complex


def _diag_system(cvals):
    n = len(cvals)
    exps = []
    coef = []
    for i, c in enumerate(cvals):
        a = [0] * n
        a[i] = 2
        exps += [a, [0] * n]
        coef += [[1.0, 0.0], [-c.real, -c.imag]]
    return synth.System(n, n, np.full(n, 2, np.int32), np.array(exps, np.int8), np.array(coef))


@pytest.mark.parametrize("L", [1, 2, 4])
def test_diagonal_system_closed_form(oracle_lib, L):
    """f_i = x_i^2 - c_i: the 2^n endpoints are all sign choices of sqrt(c_i)."""
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    s = _diag_system(c)
    out = oracle_lib.track(s, [2, 2, 2], synth.random_gamma(1), np.arange(8), L)
    assert np.all(out["status"] == 1)
    r = np.sqrt(c)
    expect = np.array([[r[0] * (1 - 2 * ((p >> 0) & 1)), r[1] * (1 - 2 * ((p >> 1) & 1)),
                        r[2] * (1 - 2 * ((p >> 2) & 1))] for p in range(8)])
    ok, worst = match_sets(to_complex(out["x_end"]), expect, 1e-13)
    assert ok, worst
    # residual of every endpoint, exactly
    for p in range(8):
        for i in range(3):
            z = cx_from(out["x_end"][i, :, :, p])
            res = z * z - Cx(Fr(c[i].real), Fr(c[i].imag))
            assert res.absf() <= {1: 1e-14, 2: 1e-28, 4: 1e-55}[L]


def test_univariate_roots_match_companion_matrix(oracle_lib):
    s = synth.total_degree_system(77, 1, 6, 7)  # dense univariate of degree 6
    out = oracle_lib.track(s, [6], synth.random_gamma(2), np.arange(6), 1)
    assert np.all(out["status"] == 1)
    coeffs = np.zeros(7, complex)
    for a, cf in zip(s.exps[:, 0], s.coef):
        coeffs[6 - a] += cf[0] + 1j * cf[1]
    roots = np.roots(coeffs)
    ok, worst = match_sets(to_complex(out["x_end"]), roots[:, None], 1e-10)
    assert ok, worst


def _dense(seed, n, d):
    from math import comb
    return synth.total_degree_system(seed, n, d, comb(n + d, d))


@pytest.mark.slow
def test_dense_generic_system_reaches_bezout_and_precisions_agree(oracle_lib):
    """All monomials of degree <= 2 present with random coefficients: all 2^n
    paths converge (the Bezout number is attained); D, DD and QD endpoint sets
    agree to 1e-10; every QD endpoint has an exact residual below 1e-40."""
    s = _dense(5, 3, 2)
    ends = {}
    for L in (1, 2, 4):
        out = oracle_lib.track(s, [2, 2, 2], synth.random_gamma(3), np.arange(8), L)
        assert np.all(out["status"] == 1), (L, out["status"])
        ends[L] = out
    for L in (2, 4):
        ok, worst = match_sets(to_complex(ends[1]["x_end"]), to_complex(ends[L]["x_end"]), 1e-10)
        assert ok, (L, worst)
    coefs = [Cx(Fr(c[0]), Fr(c[1])) for c in s.coef]
    m = s.n_terms[0]
    for p in range(8):
        xp = [cx_from(ends[4]["x_end"][i, :, :, p]) for i in range(3)]
        for j in range(3):
            r = poly_value(coefs[j * m:(j + 1) * m], s.exps[j * m:(j + 1) * m], xp)
            assert r.absf() <= 1e-40


def test_plain_n6_shape_runs_and_converged_endpoints_are_solutions(oracle_lib):
    s = synth.config_system("plain_n6_d")
    out = oracle_lib.track(s, [2] * 6, synth.random_gamma(0), np.arange(64), 1,
                           oracle_lib.default_params(1, h_min=1e-6))
    assert np.all(out["status"] == 1)  # with a small step floor every path converges
    X = to_complex(out["x_end"])
    # distinct endpoints: no two paths ended at the same solution
    ok, _ = match_sets(X, X, 0)
    D = np.max(np.abs(X[:, None] - X[None]), axis=2) + np.eye(64) * 1e9
    assert D.min() > 1e-6
    val, _ = oracle_lib.eval_(s, out["x_end"])
    assert np.max(np.abs(val[:, 0, 0] + 1j * val[:, 1, 0])) < 1e-10
    assert certify_roots(s, X)["distinct_roots"] == 64


def test_certificate_catches_duplicates_and_non_roots(oracle_lib):
    """The Kantorovich certificate accepts the closed-form roots of
    x_i^2 = c_i, and refuses a list with a root twice (two paths on one root)
    or with a point that is not near a root."""
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    s = _diag_system(c)
    r = np.sqrt(c)
    X = np.array([[r[0] * (1 - 2 * ((p >> 0) & 1)), r[1] * (1 - 2 * ((p >> 1) & 1)),
                   r[2] * (1 - 2 * ((p >> 2) & 1))] for p in range(8)])
    good = certify_roots(s, X)
    assert good["distinct_roots"] == 8 and good["h"] < 1e-12
    dup = X.copy()
    dup[5] = dup[2]
    assert certify_roots(s, dup)["distinct_roots"] == 0
    off = X.copy()
    off[3] = [0.1, 0.1j, 0.05]
    bad = certify_roots(s, off)
    assert bad["distinct_roots"] == 0 and bad["h"] > 0.5
    near = X + 1e-7  # still certifies the same roots: each lies within 2 eta
    assert certify_roots(s, near)["distinct_roots"] == 8


@pytest.mark.parametrize("name", ["batched_n12_dd",
                                  pytest.param("stress_n10_qd", marks=pytest.mark.slow),
                                  pytest.param("learned_n16_d", marks=pytest.mark.slow)])
def test_workload_systems_have_bezout_many_roots(oracle_lib, name):
    """Pins the converged/failed/diverged split of the tracking workloads.
    Tracked in double with the step floor 1e-9, every path converges, and the
    endpoints carry a Kantorovich certificate of prod(d_i) distinct isolated
    roots.  Bezout bounds the isolated roots by prod(d_i), so these are all of
    them: every path of the total-degree homotopy ends at a finite regular
    root, which is the split the tracker must report in every precision."""
    cfg = synth.CONFIGS[name]
    s = synth.config_system(name)
    m = cfg["degree"] ** cfg["n"]
    out = oracle_lib.track(s, [cfg["degree"]] * cfg["n"], synth.random_gamma(cfg["seed"]), np.arange(m), 1,
                           oracle_lib.default_params(1, h_min=1e-9))
    assert np.all(out["status"] == 1)
    cert = certify_roots(s, to_complex(out["x_end"]))
    assert cert["distinct_roots"] == m, cert



@pytest.mark.parametrize("L", [1, 2, 4])
def test_deficient_system_one_root_and_paths_to_infinity(oracle_lib, L):
    """With the step cap 0.005 exactly one path converges, to (1, 1), and the
    other three do not (diverged past r_div or failed), as the root count
    demands.  With the default cap 0.1 two more paths jump onto the root's
    path and report it as their endpoint; the certificate refuses those
    endpoints as distinct roots."""
    s = synth.deficient_system()
    gam = synth.random_gamma(5)
    tight = oracle_lib.track(s, [2, 2], gam, np.arange(4), L,
                             oracle_lib.default_params(L, r_div=1e4, h_min=1e-8, h_max=0.005))
    st = tight["status"]
    assert np.sum(st == 1) == 1 and np.all(np.isin(st, (1, -1, -2))) and np.sum(st == -2) >= 1
    X = to_complex(tight["x_end"])[st == 1]
    assert np.max(np.abs(X - 1.0)) <= {1: 1e-12, 2: 1e-28, 4: 1e-55}[L]
    loose = oracle_lib.track(s, [2, 2], gam, np.arange(4), L, oracle_lib.default_params(L, r_div=1e4, h_min=1e-8))
    conv = to_complex(loose["x_end"])[loose["status"] == 1]
    assert conv.shape[0] == 3 and np.max(np.abs(conv - 1.0)) < 1e-10
    assert certify_roots(s, conv)["distinct_roots"] == 0
    assert certify_roots(s, conv[:1])["distinct_roots"] == 1


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_predictor_is_exact_on_polynomial_paths(oracle_lib, L, m):
    """Extrapolation through m points reproduces every path that is a
    polynomial of degree m - 1 in t: complex polynomials with small integer
    coefficients at dyadic times, so the data are exact doubles and the
    expected point is known exactly; the error is rounding only."""
    from fractions import Fraction as F
    rng = synth.SplitMix64(900 + 10 * m + L)
    n = 3
    ts = [F(k, 16) for k in (0, 2, 3, 5, 6)[:m]]
    t1 = ts[-1] + F(3, 32)
    coef = rng.integers(-5, 5, 2 * n * m).reshape(n, 2, m)
    def p(i, c, t):
        return sum(F(int(coef[i, c, e])) * t ** e for e in range(m))
    xs = np.zeros((m, n, 2, L))
    for j, t in enumerate(ts):
        for i in range(n):
            for c in range(2):
                v = p(i, c, t)
                xs[j, i, c, 0] = float(v)
                assert F(xs[j, i, c, 0]) == v  # exact data
    out = oracle_lib.predict(np.array([float(t) for t in ts]), xs, float(t1))
    for i in range(n):
        for c in range(2):
            err = abs(fr(out[i, c]) - p(i, c, t1))
            scale = max(1, max(abs(p(i, c, t)) for t in ts))
            assert err <= 2.0 ** (-53 * L + 12) * scale, (i, c, float(err))


@pytest.mark.parametrize("L", [1, 2, 4])
def test_homotopy_special_cases_and_affinity_in_t(oracle_lib, L):
    """h(x, t) = gamma (1 - t) g(x) + t f(x) with g_i = x_i^d_i - 1, checked
    without restating it: it vanishes at the start solutions at t = 0, where
    its Jacobian is gamma d_i x_i^(d_i - 1) = gamma d_i conj(x_i) on the
    diagonal (x_i a root of unity) and zero elsewhere; at t = 1 it is f and
    f's Jacobian (the pinned evaluation); and h and J are affine in t."""
    s = synth.config_system("stress_n10_qd")
    n = s.n_vars
    deg = s.degrees()
    gam = synth.random_gamma(4)
    G = Cx(Fr(gam[0]), Fr(gam[1]))
    u = 2.0 ** (-53 * L)
    x0 = oracle_lib.start_solutions(deg, 5, 7, L)
    h0, J0 = oracle_lib.homotopy(s, deg, gam, 0.0, x0)
    for q in range(7):
        for i in range(n):
            assert cx_from(h0[i, :, :, q]).absf() <= 64 * u
            for j in range(n):
                got = cx_from(J0[i, j, :, :, q])
                if i != j:
                    assert got.abs2() == 0
                    continue
                xi = cx_from(x0[i, :, :, q])
                want = G * Cx(xi.re, -xi.im) * int(deg[i])
                assert (got - want).absf() <= 64 * u * int(deg[i])
    x = synth.unit_points(31 + L, n, 5, L)
    h1, J1 = oracle_lib.homotopy(s, deg, gam, 1.0, x)
    fv, fj = oracle_lib.eval_(s, x)
    assert np.array_equal(h1, fv) and np.array_equal(J1, fj)
    hz, Jz = oracle_lib.homotopy(s, deg, gam, 0.0, x)
    t = Fr(3, 8)
    ht, Jt = oracle_lib.homotopy(s, deg, gam, float(t), x)
    for q in range(5):
        for i in range(n):
            a, b, c = cx_from(hz[i, :, :, q]), cx_from(h1[i, :, :, q]), cx_from(ht[i, :, :, q])
            want = a * (1 - t) + b * t
            assert (c - want).absf() <= 2 ** 8 * u * (a.absf() + b.absf() + 1)
            for j in range(n):
                a, b, c = (cx_from(Jz[i, j, :, :, q]), cx_from(J1[i, j, :, :, q]), cx_from(Jt[i, j, :, :, q]))
                want = a * (1 - t) + b * t
                assert (c - want).absf() <= 2 ** 8 * u * (a.absf() + b.absf() + 1)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_step_control_worked_example(oracle_lib, L):
    """g = x - 1, f = 2x - 3 (one variable, degree 1): the homotopy is linear
    in x, so Newton's method lands on the path in one round and no step is
    rejected; the step sequence then follows from the step rule alone.  With
    h0 = 0.05, growth 1.5 and cap 0.1 the accepted steps end at t = 0.05,
    0.125 (h = 0.075), 0.225, 0.325, ..., 0.925 (h capped at 0.1), and the
    last step is clamped to t = 1: 11 steps, ending at x = 3/2."""
    s = synth.System(1, 1, np.array([2], np.int32), np.array([[1], [0]], np.int8),
                     np.array([[2.0, 0.0], [-3.0, 0.0]]))
    out = oracle_lib.track(s, [1], synth.random_gamma(8), np.arange(1), L)
    assert out["status"][0] == 1 and out["t_end"][0] == 1.0
    assert out["steps"][0] == 11 and out["rejects"][0] == 0
    z = cx_from(out["x_end"][0, :, :, 0])
    assert (z - Cx(Fr(3, 2))).absf() <= 4 * 2.0 ** (-53 * L)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("case", ["update", "residual"])
def test_rejection_worked_example(oracle_lib, L, case):
    """The same linear homotopy with one Newton round per step, cut off by
    max_steps.  From x = 1 (order-0 prediction) the update is exactly
    x(t1) - 1 = t1 / (gamma (1 - t1) + 2 t1), of modulus in
    [t1 / 1.05, t1 / 0.85] for |gamma| = 1 and t1 <= 0.05, and the residual
    at the predicted point is |h(1, t1)| = t1.  With tol_dx = 0.03:
      update:   tol_res = 1.  t1 = 0.05 is rejected (update >= 0.047), then
                h = 0.4 * 0.05 and t1 = 0.02 is accepted: 2 steps, 1 rejection.
      residual: tol_res = 1e-4.  Every t1 = 0.05 * 0.4^k above 1.0003e-4 fails
                the residual test; k = 7 (8.19e-5) passes: 8 steps, 7
                rejections, t = 0.05 * 0.4^7."""
    s = synth.System(1, 1, np.array([2], np.int32), np.array([[1], [0]], np.int8),
                     np.array([[2.0, 0.0], [-3.0, 0.0]]))
    gam = synth.random_gamma(8)
    tol_res, max_steps, rejects = (1.0, 2, 1) if case == "update" else (1e-4, 8, 7)
    prm = oracle_lib.default_params(L, newton_max=1, tol_dx=0.03, tol_res=tol_res, f_down=0.4, max_steps=max_steps)
    out = oracle_lib.track(s, [1], gam, np.arange(1), L, prm)
    h = 0.05
    for _ in range(rejects):
        h = 0.4 * h
    assert out["status"][0] == -1  # stopped by max_steps
    assert out["steps"][0] == max_steps and out["rejects"][0] == rejects
    assert out["t_end"][0] == h
    t = Fr(h)
    G = Cx(Fr(gam[0]), Fr(gam[1]))
    xt = (G * (1 - t) + Cx(3 * t)) / (G * (1 - t) + Cx(2 * t))
    assert (cx_from(out["x_end"][0, :, :, 0]) - xt).absf() <= 8 * 2.0 ** (-53 * L)


# ---- tangent predictor (Section 2's predictor stage, from J v = -dh/dt)
def _diag_system(c):
    n = len(c)
    exps, coef = [], []
    for i, ci in enumerate(c):
        a = [0] * n
        a[i] = 2
        exps += [a, [0] * n]
        coef += [[1.0, 0.0], [-ci.real, -ci.imag]]
    return synth.System(n, n, np.full(n, 2, np.int32), np.array(exps, np.int8), np.array(coef))


@pytest.mark.parametrize("L", [1, 2, 4])
def test_tangent_of_the_diagonal_system_in_closed_form(oracle_lib, L):
    """h_i = gamma (1 - t)(x_i^2 - 1) + t (x_i^2 - c_i): J = diag(2 x_i (gamma
    (1 - t) + t)) and dh_i/dt = (x_i^2 - c_i) - gamma (x_i^2 - 1), so the
    tangent at ANY point is v_i = -dh_i/dt / J_ii -- computed exactly with
    rationals from the same doubles."""
    from exact import Cx
    from fractions import Fraction as F
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    s = _diag_system(c)
    gam = (0.6, 0.8)
    rng = synth.SplitMix64(17 + L)
    for t in (0.0, 0.25, 0.625, 1.0):
        x = synth.unit_points(40 + L, 3, 4, L)
        x[:, :, 0, :] *= 0.5 + rng.uniform(12).reshape(3, 1, 4)  # off the path, |x| in (0.5, 1.5)
        x[:, :, 1:, :] = 0.0
        v = oracle_lib.tangent(s, [2, 2, 2], gam, t, x)
        G = Cx(F(gam[0]), F(gam[1]))
        T = F(t)
        for p in range(4):
            for i in range(3):
                xi = Cx(F(x[i, 0, 0, p]), F(x[i, 1, 0, p]))
                x2 = xi * xi
                ht = (x2 - Cx(F(c[i].real), F(c[i].imag))) - G * (x2 - Cx(1))
                Jii = Cx(2) * xi * (G * Cx(1 - T) + Cx(T))
                want = Cx(0) - ht / Jii
                got_re = sum(F(float(u)) for u in v[i, 0, :, p])
                got_im = sum(F(float(u)) for u in v[i, 1, :, p])
                err = float(abs(got_re - want.re) + abs(got_im - want.im))
                assert err <= 2.0 ** (-53 * L + 10) * max(1.0, want.absf()), (t, p, i, err)


def test_tangent_is_the_derivative_of_the_path(oracle_lib):
    """On the diagonal system's path x_i(t)^2 = (gamma (1 - t) + t c_i) /
    (gamma (1 - t) + t), the tangent equals the path's derivative (central
    differences of the closed form)."""
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    s = _diag_system(c)
    g = 0.6 + 0.8j
    xt = lambda t: np.sqrt((g * (1 - t) + t * c) / (g * (1 - t) + t))
    for t in (0.1, 0.5, 0.9):
        z = xt(t)
        x = np.zeros((3, 2, 1, 1))
        x[:, 0, 0, 0], x[:, 1, 0, 0] = z.real, z.imag
        v = oracle_lib.tangent(s, [2, 2, 2], (0.6, 0.8), t, x)
        vz = v[:, 0, 0, 0] + 1j * v[:, 1, 0, 0]
        h = 1e-5
        fd = (xt(t + h) - xt(t - h)) / (2 * h)
        assert np.max(np.abs(vz - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd))), (t, vz, fd)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_tangent_predictors_are_exact_on_polynomial_paths(oracle_lib, L):
    """Euler reproduces paths linear in t, the cubic Hermite predictor paths
    cubic in t, from exact dyadic data (values and derivatives)."""
    from fractions import Fraction as F
    from exact import fr
    rng = synth.SplitMix64(700 + L)
    n = 3
    s0, s1, t1 = F(1, 8), F(3, 8), F(9, 16)
    for mode, deg in ((1, 1), (2, 3)):
        coef = rng.integers(-6, 6, 2 * n * (deg + 1)).reshape(n, 2, deg + 1)
        p = lambda i, c, t: sum(F(int(coef[i, c, e])) * t ** e for e in range(deg + 1))
        dp = lambda i, c, t: sum(e * F(int(coef[i, c, e])) * t ** (e - 1) for e in range(1, deg + 1))
        arr = lambda f, t: np.array([[[float(f(i, c, t))] + [0.0] * (L - 1) for c in range(2)] for i in range(n)])
        out = oracle_lib.predict_tangent(mode, float(s0), arr(p, s0), arr(dp, s0), float(s1), arr(p, s1),
                                         arr(dp, s1), float(t1))
        for i in range(n):
            for c in range(2):
                err = abs(fr(out[i, c]) - p(i, c, t1))
                assert err <= 2.0 ** (-53 * L + 12) * 64, (mode, i, c, float(err))
        # at s1 the predictor returns x1; a path one degree higher is missed
        # by exactly its top coefficient times the predictor's known error
        # factor (Euler: (t1 - s1)^2; Hermite: (t1 - s0)^2 (t1 - s1)^2)
        out_s1 = oracle_lib.predict_tangent(mode, float(s0), arr(p, s0), arr(dp, s0), float(s1), arr(p, s1),
                                            arr(dp, s1), float(s1))
        assert np.array_equal(out_s1[:, :, 0], arr(p, s1)[:, :, 0])
        q = lambda i, c, t: p(i, c, t) + t ** (deg + 1)
        dq = lambda i, c, t: dp(i, c, t) + (deg + 1) * t ** deg
        out_q = oracle_lib.predict_tangent(mode, float(s0), arr(q, s0), arr(dq, s0), float(s1), arr(q, s1),
                                           arr(dq, s1), float(t1))
        miss = (t1 - s1) ** 2 if mode == 1 else (t1 - s0) ** 2 * (t1 - s1) ** 2
        for i in range(n):
            err = fr(out_q[i, 0]) - q(i, 0, t1)
            assert abs(err + miss) <= 2.0 ** (-53 * L + 12) * 64, (mode, float(err), float(miss))


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("pred", [1, 2])
def test_tangent_predictors_track_the_diagonal_system(oracle_lib, L, pred):
    """Every path of x_i^2 = c_i ends at its closed-form root with either
    tangent predictor, in D, DD and QD."""
    c = np.array([0.3 + 0.8j, -1.1 + 0.2j, 0.5 - 0.9j])
    s = _diag_system(c)
    o = oracle_lib.track(s, [2, 2, 2], (0.6, 0.8), np.arange(8), L, oracle_lib.default_params(L, predictor=pred))
    assert np.all(o["status"] == 1)
    r = np.sqrt(c)
    z = (o["x_end"][:, 0, 0, :] + 1j * o["x_end"][:, 1, 0, :]).T
    for p in range(8):
        want = [r[i] * (1 - 2 * ((p >> i) & 1)) for i in range(3)]
        assert np.max(np.abs(z[p] - want)) <= 1e-13, (p, z[p], want)


def test_hermite_takes_fewer_steps_than_euler(oracle_lib):
    """Both tangent predictors reach the same endpoints of the n = 6 system;
    the third-order Hermite predictor needs fewer steps than first-order
    Euler."""
    s = synth.config_system("plain_n6_d")
    g = synth.random_gamma(0)
    res = {}
    for pred in (1, 2):
        res[pred] = oracle_lib.track(s, s.degrees(), g, np.arange(16), 1,
                                     oracle_lib.default_params(1, h_min=1e-6, predictor=pred))
    assert np.all(res[1]["status"] == 1) and np.all(res[2]["status"] == 1)
    za = (res[1]["x_end"][:, 0, 0, :] + 1j * res[1]["x_end"][:, 1, 0, :]).T
    zb = (res[2]["x_end"][:, 0, 0, :] + 1j * res[2]["x_end"][:, 1, 0, :]).T
    assert np.max(np.abs(za - zb)) <= 1e-10
    assert res[2]["steps"].sum() < res[1]["steps"].sum()
