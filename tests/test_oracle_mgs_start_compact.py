"""Pins for least squares by modified Gram-Schmidt, the total-degree start
solutions and the scan compaction of Table tabjobidx."""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth
from exact import Cx, cx_from, cx_pow

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_complex(rng, shape, L):
    re, im = synth.unit_circle(rng, int(np.prod(shape)))
    mag = rng.uniform(re.size) + 0.5
    re, im = re * mag, im * mag
    out = np.empty(shape + (2, L))
    out[..., 0, :] = synth.random_tails(rng, re, L).T.reshape(shape + (L,))
    out[..., 1, :] = synth.random_tails(rng, im, L).T.reshape(shape + (L,))
    return out


@pytest.mark.parametrize("rows,cols", [(6, 6), (12, 12), (9, 5)])
def test_mgs_matches_lstsq_in_double(oracle_lib, rows, cols):
    rng = synth.SplitMix64(rows * 100 + cols)
    A = _rand_complex(rng, (8, rows, cols), 1)
    b = _rand_complex(rng, (8, rows), 1)
    x = oracle_lib.mgs_solve(A, b)
    for s in range(8):
        Ac = A[s, :, :, 0, 0] + 1j * A[s, :, :, 1, 0]
        bc = b[s, :, 0, 0] + 1j * b[s, :, 1, 0]
        ref = np.linalg.lstsq(Ac, bc, rcond=None)[0]
        got = x[s, :, 0, 0] + 1j * x[s, :, 1, 0]
        cond = np.linalg.cond(Ac)
        assert np.max(np.abs(got - ref)) <= 1e-14 * cond * max(1, np.max(np.abs(ref)))


def _exact_solve(A, b):
    """Exact rational solution of the normal equations A^H A x = A^H b."""
    rows, cols = len(A), len(A[0])
    N = [[Cx(0) for _ in range(cols)] for _ in range(cols)]
    r = [Cx(0) for _ in range(cols)]
    for i in range(cols):
        for j in range(cols):
            for k in range(rows):
                N[i][j] = N[i][j] + Cx(A[k][i].re, -A[k][i].im) * A[k][j]
        for k in range(rows):
            r[i] = r[i] + Cx(A[k][i].re, -A[k][i].im) * b[k]
    for c in range(cols):  # Gauss-Jordan (exact, no pivoting problems for SPD)
        piv = N[c][c]
        for j in range(c, cols):
            N[c][j] = N[c][j] / piv
        r[c] = r[c] / piv
        for i in range(cols):
            if i != c:
                f = N[i][c]
                for j in range(c, cols):
                    N[i][j] = N[i][j] - f * N[c][j]
                r[i] = r[i] - f * r[c]
    return r


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("rows,cols", [(3, 3), (5, 3)])
def test_mgs_against_exact_solution(oracle_lib, L, rows, cols):
    rng = synth.SplitMix64(77 + L + rows)
    A = _rand_complex(rng, (2, rows, cols), L)
    b = _rand_complex(rng, (2, rows), L)
    x = oracle_lib.mgs_solve(A, b)
    for s in range(2):
        Ae = [[cx_from(A[s, i, j]) for j in range(cols)] for i in range(rows)]
        be = [cx_from(b[s, i]) for i in range(rows)]
        ex = _exact_solve(Ae, be)
        Ad = A[s, :, :, 0, 0] + 1j * A[s, :, :, 1, 0]
        cond = np.linalg.cond(Ad)
        scale = max(e.absf() for e in ex)
        for j in range(cols):
            err = (cx_from(x[s, j]) - ex[j]).absf()
            assert err <= 100 * cond * cond * 2.0 ** (-53 * L) * scale, (j, err)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("degrees", [[2, 2, 2], [3, 2], [5, 3], [3, 3, 3, 3]])
def test_start_solutions_are_the_roots_of_unity(oracle_lib, L, degrees):
    count = int(np.prod(degrees))  # Bezout number of paths
    x = oracle_lib.start_solutions(degrees, 0, count, L)
    pts = set()
    for p in range(count):
        for i, d in enumerate(degrees):
            z = cx_from(x[i, :, :, p])
            r = cx_pow(z, d) - Cx(1)
            assert r.absf() <= 16 * d * 2.0 ** (-53 * L)
            if d == 2:  # +-1 exactly
                assert z.im == 0 and abs(z.re) == 1
        pts.add(tuple(np.round(x[:, :, 0, p].ravel(), 12)))
    assert len(pts) == count  # all distinct
    # digit of variable 0 varies fastest
    if degrees[0] == 2:
        assert x[0, 0, 0, 0] == 1.0 and x[0, 0, 0, 1] == -1.0


def test_compaction_table_tabjobidx(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "tabjobidx.json")))
    scan, idx = oracle_lib.compact(np.array(g["status"], np.int8))
    assert scan.tolist() == g["scan_for_0"]
    assert idx.tolist() == g["path_idx"]
    assert scan[-1] == g["active_count"]
    job = [int(scan[i]) if st == 0 else None for i, st in enumerate(g["status"])]
    assert job == g["job_idx"]


def test_compaction_random(oracle_lib):
    rng = synth.SplitMix64(3)
    st = (rng.integers(0, 3, 10000) - 1).astype(np.int8)
    scan, idx = oracle_lib.compact(st)
    assert np.array_equal(scan, np.cumsum(st == 0))
    assert np.array_equal(idx, np.nonzero(st == 0)[0])
