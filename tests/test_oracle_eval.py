"""Pins for the oracle's evaluation and differentiation (Table tabcpugpu,
Table tabmoneval, Table tabtranspose)."""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from exact import Cx, cx_from, fr, poly_partial_by_interpolation, poly_value

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_system(seed, n=3, m=5, emax=3):
    rng = synth.SplitMix64(seed)
    exps = rng.integers(0, emax, n * m * n).reshape(n * m, n).astype(np.int8)
    exps[::m] = 0  # one constant term per polynomial
    re, im = synth.unit_circle(rng, n * m)
    return synth.System(n, n, np.full(n, m, np.int32), exps, np.stack([re, im], 1))


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("method", ["naive", "speelpenning"])
def test_eval_against_exact_brute_force(oracle_lib, L, method):
    """Values from an exact rational sum of terms; derivatives by exact
    polynomial interpolation along each coordinate (no product rule)."""
    s = _tiny_system(11 + L)
    x = synth.unit_points(21, s.n_vars, 3, L)
    val, jac = oracle_lib.eval_(s, x, method=method)
    mval, mjac = oracle_lib.eval_magnitude(s, x)
    coefs = [Cx(Fr(c[0]), Fr(c[1])) for c in s.coef]
    deg = int(s.exps.astype(int).sum(1).max())
    u = Fr(2) ** (-53 * L)
    for p in range(3):
        xp = [cx_from(x[i, :, :, p]) for i in range(s.n_vars)]
        for j in range(s.n_polys):
            sl = slice(j * 5, (j + 1) * 5)
            ex = poly_value(coefs[sl], s.exps[sl], xp)
            got = cx_from(val[j, :, :, p])
            assert (got - ex).absf() <= 64 * deg * float(u) * mval[j, p] + 1e-300
            for i in range(s.n_vars):
                exd = poly_partial_by_interpolation(coefs[sl], s.exps[sl], xp, i, deg)
                gotd = cx_from(jac[j, i, :, :, p])
                assert (gotd - exd).absf() <= 64 * deg * float(u) * mjac[j, i, p] + 1e-300, (j, i, p)


def test_magnitude_scale_is_the_sum_of_term_moduli(oracle_lib):
    """The tolerance scale sum |term| of each output: with positive real
    coefficients and positive real points every term is a positive real, so
    the scale equals the exact value and exact derivative; for complex inputs
    it bounds the exact value from above (triangle inequality)."""
    s = _tiny_system(71)
    rng = synth.SplitMix64(72)
    pos = synth.System(s.n_vars, s.n_polys, s.n_terms, s.exps,
                       np.stack([rng.uniform(s.exps.shape[0]) + 0.25, np.zeros(s.exps.shape[0])], 1))
    x = np.zeros((s.n_vars, 2, 1, 4))
    x[:, 0, 0, :] = 0.5 + 1.5 * rng.uniform(s.n_vars * 4).reshape(s.n_vars, 4)  # moduli in [0.5, 2)
    mval, mjac = oracle_lib.eval_magnitude(pos, x)
    coefs = [Cx(Fr(c[0]), Fr(c[1])) for c in pos.coef]
    deg = int(pos.exps.astype(int).sum(1).max())
    for p in range(4):
        xp = [cx_from(x[i, :, :, p]) for i in range(s.n_vars)]
        for j in range(s.n_polys):
            sl = slice(j * 5, (j + 1) * 5)
            ex = float(poly_value(coefs[sl], pos.exps[sl], xp).re)
            assert abs(mval[j, p] - ex) <= 1e-13 * ex
            for i in range(s.n_vars):
                exd = float(poly_partial_by_interpolation(coefs[sl], pos.exps[sl], xp, i, deg).re)
                assert abs(mjac[j, i, p] - exd) <= 1e-13 * max(exd, 1e-300)
    x = synth.unit_points(73, s.n_vars, 4, 1) * 1.7
    mval, _ = oracle_lib.eval_magnitude(s, x)
    coefs = [Cx(Fr(c[0]), Fr(c[1])) for c in s.coef]
    for p in range(4):
        xp = [cx_from(x[i, :, :, p]) for i in range(s.n_vars)]
        for j in range(s.n_polys):
            sl = slice(j * 5, (j + 1) * 5)
            assert poly_value(coefs[sl], s.exps[sl], xp).absf() <= mval[j, p] * (1 + 1e-13)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_naive_and_reverse_mode_agree(oracle_lib, L):
    """The product rule and the reverse mode are two different computations of
    the same derivatives; on both workload families they agree to rounding."""
    u = 2.0 ** (-53 * L)
    for s, npts in ((synth.config_system("plain_n6_d"), 4), (synth.config_system("evaldiff_n32"), 1 if L == 4 else 2)):
        x = synth.unit_points(3, s.n_vars, npts, L)
        v1, j1 = oracle_lib.eval_(s, x, method="naive")
        v2, j2 = oracle_lib.eval_(s, x, method="speelpenning")
        mv, mj = oracle_lib.eval_magnitude(s, x)
        for a, b, m in ((v1, v2, mv), (j1, j2, mj)):
            d = np.hypot(oracle_lib.value_diff(np.moveaxis(a[..., 0, :, :], -2, -1),
                                               np.moveaxis(b[..., 0, :, :], -2, -1)),
                         oracle_lib.value_diff(np.moveaxis(a[..., 1, :, :], -2, -1),
                                               np.moveaxis(b[..., 1, :, :], -2, -1)))
            assert np.all(d <= 200 * 24 * u * m), np.max(d / m)


def test_tabmoneval_slots(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "tabmoneval.json")))
    k = g["k"]
    for L in (1, 2, 4):
        x = synth.unit_points(5 + L, k, 1, L)[:, :, :, 0]
        slots, nmul = oracle_lib.speelpenning_slots(x)
        assert nmul == g["multiplications"] == 3 * k - 5
        xe = [cx_from(x[i]) for i in range(k)]
        for row in g["rows_in_execution_order"]:
            ex = Cx(1)
            for v in row["product_of"]:
                ex = ex * xe[v - 1]
            got = cx_from(slots[row["slot"]])
            assert (got - ex).absf() <= 8 * 2.0 ** (-53 * L)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6, 7, 8])
def test_reverse_mode_counts_and_values(oracle_lib, k):
    """3k - 5 multiplications for k >= 2; value and every derivative exact to rounding."""
    for L in (1, 2):
        x = synth.unit_points(40 + k, k, 1, L)[:, :, :, 0]
        slots, nmul = oracle_lib.speelpenning_slots(x)
        assert nmul == (3 * k - 5 if k >= 2 else 0)
        xe = [cx_from(x[i]) for i in range(k)]
        full = Cx(1)
        for z in xe:
            full = full * z
        assert (cx_from(slots[2 * k - 1 if k > 1 else 0]) - full).absf() <= 4 * k * 2.0 ** (-53 * L)


def test_tabtranspose_layout(oracle_lib):
    """Each evaluated quantity of all paths is contiguous, path index fastest."""
    g = json.load(open(os.path.join(GOLDEN, "tabtranspose.json")))
    s = synth.System(3, 1, np.array([1], np.int32), np.array([g["monomial_exponents"]], np.int8),
                     np.array([[1.0, 0.0]]))
    npts = 3
    x = synth.unit_points(8, 3, npts, 1)
    val, jac = oracle_lib.eval_(s, x)
    flat = np.concatenate([val[0, 0, 0], jac[0, :, 0, 0].reshape(-1)])  # real parts, quantity-major
    for q, quant in enumerate(g["quantities"]):
        for p in range(npts):
            ex = Cx(1)
            for v in quant["product_of"]:
                ex = ex * cx_from(x[v, :, :, p])
            assert abs(flat[q * npts + p] - float(ex.re)) <= 1e-15
