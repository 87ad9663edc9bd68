"""CPU tests of the library's multi-limb integer complex arithmetic
(csrc/ht_mpi.cuh, compiled for the host): conversions, products and
fixed-point accumulation against the oracle's exact L-limb arithmetic."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("mpi") / "libmpi_shim.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", out, os.path.join(HERE, "mpi_shim.cpp")])
    L = ctypes.CDLL(out)
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    L.mpi_roundtrip.argtypes = [ctypes.c_int, I64, P, P]
    L.mpi_product.argtypes = [ctypes.c_int, I64, P, P, ctypes.c_int, P]
    L.mpi_dot.argtypes = [ctypes.c_int, I64, ctypes.c_int, P, P, P, ctypes.c_int, P]
    L.mpi_dot_fast.argtypes = [ctypes.c_int, I64, ctypes.c_int, P, P, P, ctypes.c_int, P]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _complex(seed, n, L, spread=30):
    rng = synth.SplitMix64(seed)
    re, im = synth.unit_circle(rng, n)
    scale = 2.0 ** rng.integers(-spread, spread, n).astype(np.float64)
    out = np.empty((n, 2, L))
    out[:, 0, :] = synth.random_tails(rng, re * scale, L).T
    out[:, 1, :] = synth.random_tails(rng, im * scale, L).T
    out[:7, 1, :] = 0.0  # purely real values
    out[7:12, 0, :] = -out[7:12, 0, :]
    return np.ascontiguousarray(out)


def _cerr(oracle_lib, got, ref):
    d = [oracle_lib.value_diff(got[:, c, :], ref[:, c, :]) for c in (0, 1)]
    return np.hypot(d[0], d[1])


@pytest.mark.parametrize("L", [2, 4])
def test_conversion_round_trip(oracle_lib, shim, L):
    x = _complex(1 + L, 500, L)
    out = np.empty_like(x)
    assert shim.mpi_roundtrip(L, x.shape[0], _p(x), _p(out)) == 0
    mag = np.hypot(x[:, 0, 0], x[:, 1, 0])
    err = _cerr(oracle_lib, out, x)
    assert np.all(err <= 2.0 ** (-53 * L + 3) * mag), np.max(err / mag)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("e", [1, 3])
def test_product_against_oracle(oracle_lib, shim, L, e):
    """e * (a * b) against the oracle's complex product (each real operation
    rounded to L limbs) within a few units of 2^(-53 L) of |a| |b|."""
    n = 400
    a = _complex(10 + L, n, L)
    b = _complex(20 + L, n, L)
    out = np.empty_like(a)
    assert shim.mpi_product(L, n, _p(a), _p(b), e, _p(out)) == 0
    ar, ai = a[:, 0, :], a[:, 1, :]
    br, bi = b[:, 0, :], b[:, 1, :]
    mul = lambda u, v: oracle_lib.real_op("mul", u, v)
    add = lambda u, v: oracle_lib.real_op("add", u, v)
    sub = lambda u, v: oracle_lib.real_op("sub", u, v)
    ref = np.empty_like(a)
    ref[:, 0, :] = sub(mul(ar, br), mul(ai, bi))
    ref[:, 1, :] = add(mul(ar, bi), mul(ai, br))
    ee = np.zeros((n, L))
    ee[:, 0] = e
    ref[:, 0, :] = mul(ref[:, 0, :], ee)
    ref[:, 1, :] = mul(ref[:, 1, :], ee)
    scale = e * np.hypot(ar[:, 0], ai[:, 0]) * np.hypot(br[:, 0], bi[:, 0])
    err = _cerr(oracle_lib, out, ref)
    assert np.all(err <= 2.0 ** (-53 * L + 5) * scale), np.max(err / scale)


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("L", [2, 4])
def test_fixed_point_sums_with_cancellation(oracle_lib, shim, L, fast):
    """sum_j e_j a_j b_j in one fixed-point frame, with headroom bits, against
    the oracle: error relative to sum_j e_j |a_j b_j| (condition-aware)."""
    n, k = 60, 24
    a = _complex(30 + L, n * k, L, spread=8).reshape(n, k, 2, L)
    b = _complex(40 + L, n * k, L, spread=8).reshape(n, k, 2, L)
    a[:, 1] = -a[:, 0] * 1.0  # strong cancellation between the first two terms
    b[:, 1] = b[:, 0]
    e = np.array([1 + (j % 3) for j in range(k)], dtype=np.int32)
    out = np.empty((n, 2, L))
    fn = shim.mpi_dot_fast if fast else shim.mpi_dot
    assert fn(L, n, k, _p(np.ascontiguousarray(a)), _p(np.ascontiguousarray(b)), _p(e), 6, _p(out)) == 0
    mul = lambda u, v: oracle_lib.real_op("mul", u, v)
    add = lambda u, v: oracle_lib.real_op("add", u, v)
    sub = lambda u, v: oracle_lib.real_op("sub", u, v)
    ref = np.zeros((n, 2, L))
    absum = np.zeros(n)
    for j in range(k):
        ar, ai, br, bi = a[:, j, 0], a[:, j, 1], b[:, j, 0], b[:, j, 1]
        ee = np.zeros((n, L))
        ee[:, 0] = e[j]
        tr = mul(sub(mul(ar, br), mul(ai, bi)), ee)
        ti = mul(add(mul(ar, bi), mul(ai, br)), ee)
        ref[:, 0] = add(ref[:, 0], tr)
        ref[:, 1] = add(ref[:, 1], ti)
        absum += e[j] * np.hypot(ar[:, 0], ai[:, 0]) * np.hypot(br[:, 0], bi[:, 0])
    err = _cerr(oracle_lib, out, ref)
    assert np.all(err <= 2.0 ** (-53 * L + 12) * absum), np.max(err / absum)


@pytest.mark.parametrize("e", [3, 1, -3, 4, -5, 127])
@pytest.mark.parametrize("L", [2, 4])
def test_shift_accumulation_equals_generic(shim, L, e):
    """The single-shift accumulation gives the same limbs as the generic
    per-limb one for right and left shifts (frames slightly above the
    accumulator's included) wherever its precondition holds: the term times
    its factor below the top limb's bit 28 (for DD, whose accumulator has one
    limb fewer than a term, that rules out every left shift).  Factors up to
    3 in magnitude take the 32-bit sums, larger ones the 64-bit sums."""
    shim.mpi_compare_acc.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int]
    shim.mpi_compare_acc.restype = ctypes.c_int64
    x = _complex(77 + L, 200, L, spread=3)
    worst = shim.mpi_compare_acc(L, x.shape[0], _p(x), -20, 29 * 9, e)
    # the single shift truncates the term before the factor (at most |e| units
    # of the last limb); the generic routine truncates each of the W <= 8
    # shifted limbs of e z
    assert 0 <= worst <= abs(e) + 8, worst


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("name", ["plain_n6_d", "batched_n12_dd", "stress_n10_qd", "evaldiff_n32", "edge", "spread",
                                  "extreme"])
def test_integer_evaluation_matches_oracle(oracle_lib, shim, L, name):
    """The integer evaluation path (bounds, fixed-point frame, reverse-mode
    sweep, conversion; the device kernel runs this code per lane) against the
    oracle at the evaluation tolerance, relative to the sum of term moduli."""
    from parity import TOL, rel_err
    shim.mpi_eval.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int64] + [ctypes.c_void_p] * 3
    if name == "edge":
        nv = 12
        exps = np.zeros((5, nv), np.int8)
        exps[1, :] = 1
        exps[2, 3] = 9
        exps[3, [0, 5, 11]] = [2, 3, 1]
        exps[4, 7] = 1
        coef = np.array([[0.5, -0.25], [1.0, 0.0], [-0.3, 0.7], [0.2, 0.2], [0.0, 1.0]])
        s = synth.System(nv, 2, np.array([3, 2], np.int32), exps, coef)
        x = synth.unit_points(8, nv, 6, L)
        rng = synth.SplitMix64(4)
        x *= 2.0 ** rng.integers(-20, 20, nv * 6).reshape(nv, 1, 1, 6).astype(np.float64)
        x[2, :, :, 5] = 0.0
    elif name == "extreme":  # 64 variables, a 64-variable support, exponent 127
        s = synth.extreme_system(77, 64, 3)
        x = synth.unit_points(17 + L, 64, 3, L)
    elif name == "spread":  # points over 60 binades
        s = synth.config_system("stress_n10_qd")
        x = synth.unit_points(91 + L, s.n_vars, 8, L)
        rng = synth.SplitMix64(12)
        x *= 2.0 ** rng.integers(-30, 30, s.n_vars * 8).reshape(s.n_vars, 1, 1, 8).astype(np.float64)
    else:
        s = synth.config_system(name)
        x = synth.unit_points(55 + L, s.n_vars, 2 if name == "evaldiff_n32" else 5, L)
    n = x.shape[-1]
    nt = np.ascontiguousarray(s.n_terms, np.int32)
    ex = np.ascontiguousarray(s.exps, np.int8)
    cf = np.ascontiguousarray(s.coef_limbs(L))
    val = np.empty((s.n_polys, 2, L, n))
    jac = np.empty((s.n_polys, s.n_vars, 2, L, n))
    assert shim.mpi_eval(L, s.n_vars, s.n_polys, _p(nt), _p(ex), _p(cf), n, _p(np.ascontiguousarray(x)), _p(val),
                         _p(jac)) == 0
    ov, oj = oracle_lib.eval_(s, x)
    mv, mj = oracle_lib.eval_magnitude(s, x)
    ev, ej = rel_err(val, ov, mv), rel_err(jac, oj, mj)
    assert ev <= TOL[L] and ej <= TOL[L], (ev, ej)


def _unit(L):
    """Relative precision of a floating limb string: the L-double target or
    the 29 (W - 1) + 1 bits the W limbs guarantee, whichever is coarser."""
    W = {1: 3, 2: 5, 4: 8}[L]
    return 2.0 ** -min(53 * L, 29 * (W - 1) + 1)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_general_sums_against_oracle(oracle_lib, shim, L):
    """sum_j e_j z_j with signed small e_j (the adds and subtracts of MGS),
    error relative to sum_j |e_j| |z_j|, including exact cancellation."""
    shim.mpi_sum.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p]
    n, k = 200, 5
    z = _complex(300 + L, n * k, L, spread=10).reshape(n, k, 2, L)
    z[:, 1] = z[:, 0]  # e = (1, -1, ...): exact cancellation of the first two
    e = np.array([1, -1, 2, -3, 1], dtype=np.int32)
    out = np.empty((n, 2, L))
    assert shim.mpi_sum(L, n, k, _p(np.ascontiguousarray(z)), _p(e), _p(out)) == 0
    add = lambda u, v: oracle_lib.real_op("add", u, v)
    mul = lambda u, v: oracle_lib.real_op("mul", u, v)
    ref = np.zeros((n, 2, L))
    absum = np.zeros(n)
    for j in range(k):
        ee = np.zeros((n, L))
        ee[:, 0] = e[j]
        ref[:, 0] = add(ref[:, 0], mul(z[:, j, 0], ee))
        ref[:, 1] = add(ref[:, 1], mul(z[:, j, 1], ee))
        absum += abs(e[j]) * np.hypot(z[:, j, 0, 0], z[:, j, 1, 0])
    err = _cerr(oracle_lib, out, ref)
    assert np.all(err <= _unit(L) * 64 * absum), np.max(err / absum)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_inverse_square_root_against_oracle(oracle_lib, shim, L):
    shim.mpi_invsqrt.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    rng = synth.SplitMix64(500 + L)
    lead = rng.uniform(300) * 2.0 ** rng.integers(-40, 40, 300).astype(np.float64) + 1e-3
    v = np.ascontiguousarray(synth.random_tails(rng, lead, L).T)
    out = np.empty_like(v)
    assert shim.mpi_invsqrt(L, v.shape[0], _p(v), _p(out)) == 0
    ref = oracle_lib.real_op("div", np.tile(np.eye(1, L), (v.shape[0], 1)), oracle_lib.real_op("sqrt", v))
    d = oracle_lib.value_diff(out, ref)
    assert np.all(np.abs(d) <= _unit(L) * 32 * np.abs(ref[:, 0])), np.max(np.abs(d) / np.abs(ref[:, 0]))


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("rows,cols", [(6, 6), (12, 12), (9, 5), (1, 1), (64, 64)])
def test_least_squares_on_limb_strings_matches_oracle(oracle_lib, shim, L, rows, cols):
    """Modified Gram-Schmidt with every dot product and norm as one exact
    fixed-point sum, 1/sqrt by Newton: the solution of [A | b] against the
    oracle's MGS within the conditioning bound of the GPU test."""
    shim.mpi_mgs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    rng = synth.SplitMix64(300 + rows * 7 + cols + L)
    n_sys = 12 if rows < 64 else 3  # 64 rows: the largest the integer variant takes
    re, im = synth.unit_circle(rng, n_sys * rows * (cols + 1))
    mag = rng.uniform(re.size) + 0.5
    Ab = np.zeros((n_sys, rows, cols + 1, 2, L))
    Ab[..., 0, :] = synth.random_tails(rng, (re * mag), L).T.reshape(n_sys, rows, cols + 1, L)
    Ab[..., 1, :] = synth.random_tails(rng, (im * mag), L).T.reshape(n_sys, rows, cols + 1, L)
    x = np.empty((n_sys, cols, 2, L))
    assert shim.mpi_mgs(L, rows, cols, n_sys, _p(np.ascontiguousarray(Ab)), _p(x)) == 0
    ref = oracle_lib.mgs_solve(np.ascontiguousarray(Ab[:, :, :cols]), np.ascontiguousarray(Ab[:, :, cols]))
    for s in range(n_sys):
        Ad = Ab[s, :, :cols, 0, 0] + 1j * Ab[s, :, :cols, 1, 0]
        cond = np.linalg.cond(Ad)
        r = ref[s, :, 0, 0] + 1j * ref[s, :, 1, 0]
        scale = np.max(np.abs(r))
        e = np.max(_cerr(oracle_lib, x[s], ref[s]))
        assert e <= 64 * cond * cond * _unit(L) * scale * rows, (s, e, cond)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_scaled_conversion_is_the_truncated_exact_product(shim, L):
    """s a for a fixed-point string a and a double s, converted to L doubles:
    the doubles' exact sum is the exact product a s truncated to the leading
    53 L bits (so it lies within 2^(1 - 53 L) |a s| below |a s|), and for s = 1
    the doubles are those of the plain conversion.  Exact rationals on the
    Python side; strings with a negative top limb and scales of every sign
    and binade included."""
    from fractions import Fraction
    WA = {1: 2, 2: 4, 4: 8}[L]
    F = -29 * (WA - 1) - 3
    rng = np.random.default_rng(500 + L)
    n = 400
    a = rng.integers(0, 1 << 29, size=(n, WA)).astype(np.int32)
    a[:, -1] = rng.integers(-(1 << 27), 1 << 27, size=n)
    a[::7, :-1] = 0  # sparse strings: a single top limb
    s = rng.uniform(-1.0, 1.0, n) * np.exp2(rng.integers(-60, 60, n))
    s[:5] = [1.0, -1.0, 0.5, 1.0 - 2.0 ** -53, 0.0]
    out = np.zeros((n, L))
    plain = np.zeros((n, L))
    shim.mpi_scaled_convert.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    assert shim.mpi_scaled_convert(L, n, _p(a), F, _p(s), _p(out), _p(plain)) == 0
    for q in range(n):
        val = sum(Fraction(int(a[q, k])) * Fraction(2) ** (29 * k) for k in range(WA)) * Fraction(2) ** F
        exact = val * Fraction(float(s[q]))
        got = sum(Fraction(float(d)) for d in out[q])
        assert abs(got) <= abs(exact)  # truncation toward zero
        assert abs(exact - got) <= abs(exact) * Fraction(2) ** (1 - 53 * L), (q, float(exact), float(got))
        if s[q] == 1.0:
            assert np.array_equal(out[q], plain[q])


@pytest.mark.parametrize("L", [2, 4])
def test_scaled_limb_string_is_the_exact_product_cut_to_w_limbs(shim, L):
    """s (ar + i ai) for fixed-point strings and a double s, as a limb string
    (the tracker's Jacobian rows scaled by t): each component of the string's
    value lies within one unit of its last limb of the exact product (the
    string keeps the W limbs from the highest nonzero one of either
    component), its lower limbs are digits in [0, 2^29), and the top limbs
    stay below 2^28 in magnitude.  Exact rationals on the Python side."""
    from fractions import Fraction
    WA, W = {2: (4, 5), 4: (8, 8)}[L]
    F = -29 * (WA - 1) - 3
    rng = np.random.default_rng(700 + L)
    n = 300
    ar = rng.integers(0, 1 << 29, size=(n, WA)).astype(np.int32)
    ai = rng.integers(0, 1 << 29, size=(n, WA)).astype(np.int32)
    ar[:, -1] = rng.integers(-(1 << 27), 1 << 27, size=n)
    ai[:, -1] = rng.integers(-(1 << 27), 1 << 27, size=n)
    ai[::5] = 0  # real values
    ar[::11, :-2] = 0  # short strings
    s = rng.uniform(0.0, 1.0, n)
    s[:4] = [1.0, 0.5, 2.0 ** -40, 1.0 - 2.0 ** -53]
    out = np.zeros((n, 2 * W + 1), dtype=np.int32)
    shim.mpi_scaled_fz.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p]
    assert shim.mpi_scaled_fz(L, n, _p(ar), _p(ai), F, _p(s), _p(out)) == 0
    two = Fraction(2)
    for q in range(n):
        f = int(out[q, 0])
        for comp, a in ((0, ar[q]), (1, ai[q])):
            limbs = out[q, 1 + comp * W:1 + (comp + 1) * W]
            assert np.all(limbs[:-1] >= 0) and np.all(limbs[:-1] < (1 << 29))
            assert abs(int(limbs[-1])) < (1 << 28)
            exact = sum(Fraction(int(a[k])) * two ** (29 * k) for k in range(WA)) * two ** F * Fraction(float(s[q]))
            got = sum(Fraction(int(limbs[k])) * two ** (29 * k) for k in range(W)) * two ** f
            assert abs(exact - got) <= two ** (f + 1), (q, comp)
