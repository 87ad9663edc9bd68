"""Pins for the oracle's L-limb arithmetic: every operation is checked against
exact rational arithmetic (Python fractions), with the error bound of a
correctly rounded L-limb result."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from exact import fr


def _rand(rng, n, L, spread=20):
    lead = (rng.uniform(n) * 2 - 1) * 2.0 ** rng.integers(-spread, spread, n).astype(np.float64)
    lead[lead == 0] = 1.0
    return np.ascontiguousarray(synth.random_tails(rng, lead, L).T)


def _exact(op, A, B):
    return {"add": A + B, "sub": A - B, "mul": A * B, "div": A / B}[op]


BOUND_BITS = {"add": 1, "sub": 1, "mul": 1, "div": 2}


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_real_op_against_exact_rationals(oracle_lib, L, op):
    rng = synth.SplitMix64(1234 + 17 * L)
    n = 400
    a = _rand(rng, n, L)
    b = _rand(rng, n, L)
    # adversarial pairs: heavy cancellation in add/sub, tiny/huge magnitudes
    b[:50] = -a[:50]
    b[:50, L - 1] += np.ldexp(1.0, -60 * L)
    b[50:100] *= 2.0 ** -40
    out = oracle_lib.real_op(op, a, b)
    for i in range(n):
        A, B, Z = fr(a[i]), fr(b[i]), fr(out[i])
        ex = _exact(op, A, B)
        assert abs(Z - ex) <= Fr(2) ** (-53 * L + BOUND_BITS[op]) * abs(ex), (op, L, i)


@pytest.mark.parametrize("L", [2, 4])
def test_real_op_limbs_are_canonical(oracle_lib, L):
    """Each limb is the correctly rounded remainder: |limb j+1| <= ulp(limb j) / 2."""
    rng = synth.SplitMix64(99)
    a, b = _rand(rng, 200, L), _rand(rng, 200, L)
    for op in ("add", "mul"):
        out = oracle_lib.real_op(op, a, b)
        for j in range(L - 1):
            assert np.all(np.abs(out[:, j + 1]) <= np.abs(np.spacing(out[:, j])) / 2)


def test_double_is_ieee(oracle_lib):
    """L = 1 is plain IEEE double arithmetic."""
    rng = synth.SplitMix64(7)
    a, b = _rand(rng, 1000, 1), _rand(rng, 1000, 1)
    for op, f in (("add", np.add), ("sub", np.subtract), ("mul", np.multiply), ("div", np.divide)):
        assert np.array_equal(oracle_lib.real_op(op, a, b)[:, 0], f(a[:, 0], b[:, 0]))
    assert np.array_equal(oracle_lib.real_op("sqrt", np.abs(a))[:, 0], np.sqrt(np.abs(a[:, 0])))


@pytest.mark.parametrize("L", [2, 4])
def test_sqrt_against_exact(oracle_lib, L):
    rng = synth.SplitMix64(4242 + L)
    a = np.abs(_rand(rng, 200, L))
    out = oracle_lib.real_op("sqrt", a)
    for i in range(a.shape[0]):
        A, Z = fr(a[i]), fr(out[i])
        # |Z^2 - A| / A ~ 2 |relative error of Z|
        assert abs(Z * Z - A) <= Fr(2) ** (-53 * L + 4) * A


@pytest.mark.parametrize("L", [2, 4])
def test_value_diff_is_exact_difference(oracle_lib, L):
    rng = synth.SplitMix64(5)
    a = _rand(rng, 100, L)
    b = a.copy()
    b[:, L - 1] += np.spacing(a[:, L - 1]) * 3
    d = oracle_lib.value_diff(a, b)
    for i in range(100):
        assert d[i] == float(fr(a[i]) - fr(b[i]))


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("op", ["add", "mul"])
def test_real_op_is_rounded_limb_by_limb(oracle_lib, L, op):
    """The oracle's stated semantics: the exact result rounded limb by limb, so
    the error is at most half an ulp of the last limb."""
    rng = synth.SplitMix64(555 + L)
    n = 400
    a = _rand(rng, n, L, spread=3)
    b = _rand(rng, n, L, spread=3)
    out = oracle_lib.real_op(op, a, b)
    for i in range(n):
        ex = _exact(op, fr(a[i]), fr(b[i]))
        half_ulp = Fr(abs(float(np.spacing(out[i, L - 1])))) / 2
        assert abs(fr(out[i]) - ex) <= half_ulp, (op, L, i)
