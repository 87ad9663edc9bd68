"""The comparison helpers of the parity tests reject what they must: a
helper that always agreed would make every parity test pass."""
import numpy as np

from match import match_sets
from parity import TOL, cerr, rel_err


def test_match_sets_is_a_one_to_one_pairing():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 3)) + 1j * rng.standard_normal((6, 3))
    perm = A[[3, 0, 5, 1, 4, 2]]
    ok, worst = match_sets(A, perm, 0.0)
    assert ok and worst == 0.0
    dup = A.copy()
    dup[4] = dup[1]  # two paths on one endpoint, one endpoint missing
    assert not match_sets(A, dup, 1e-3)[0]
    near = A + 1e-11
    assert match_sets(A, near, 1e-10)[0] and not match_sets(A, near, 1e-12)[0]
    assert not match_sets(A, A[:5], 1.0)[0]  # different counts never match
    big = A * 1e6  # distances scale with max(1, |x|_inf)
    assert match_sets(big, big + 1e-5, 1e-10)[0]


def test_cerr_sees_the_last_limb_and_ignores_the_representation():
    L, n = 4, 5
    rng = np.random.default_rng(1)
    x = np.zeros((3, 2, L, n))
    x[:, :, 0] = rng.standard_normal((3, 2, n))
    for l in range(1, L):
        x[:, :, l] = x[:, :, l - 1] * 2.0 ** -54 * rng.uniform(-1, 1, (3, 2, n))
    assert np.all(cerr(x, x) == 0.0)
    y = x.copy()
    ulp = np.abs(np.spacing(x[1, 1, L - 1, 2]))
    y[1, 1, L - 1, 2] += ulp  # one unit in the last limb of one imaginary part
    e = cerr(y, x)
    assert e[1, 2] == ulp and np.count_nonzero(e) == 1
    z = x.copy()  # the same value with its first two limbs merged where exact
    z[:, :, 0] = 3.0
    z[:, :, 1] = 2.0 ** -60
    w = z.copy()
    w[:, :, 0] = 3.0 + 2.0 ** -51
    w[:, :, 1] = 2.0 ** -60 - 2.0 ** -51
    assert np.all(cerr(w, z) == 0.0)


def test_rel_err_is_relative_to_the_scale():
    L, n = 2, 3
    x = np.zeros((2, 2, L, n))
    x[:, :, 0] = 1.0
    y = x.copy()
    y[0, 0, 1, 1] = 1e-20
    mag = np.full((2, n), 4.0)
    assert rel_err(y, x, mag) == 1e-20 / 4.0
    assert rel_err(y, x, mag) > TOL[2]
    assert rel_err(x, x, mag) == 0.0
