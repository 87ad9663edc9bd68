"""The synthetic stand-ins have the shapes the paper reports for its three
applications (Section 4.2, Table tabsumchar): dimension, monomials per
polynomial and their degrees; the oracle's two evaluation methods agree on
them (no GPU needed)."""
import numpy as np
import pytest

import synth

# Table tabsumchar: dimension and number of monomials
TABSUMCHAR = {"cyclic10_shape": (10, 92), "nash8_shape": (8, 1040), "pieri44_shape": (16, 3936)}


@pytest.mark.parametrize("name", list(TABSUMCHAR))
def test_shapes_follow_table_tabsumchar(name):
    s = synth.config_system(name)
    dim, mons = TABSUMCHAR[name]
    assert s.n_vars == s.n_polys == dim and s.n_monomials == mons
    deg = s.exps.astype(int).sum(axis=1)
    off = np.concatenate([[0], np.cumsum(s.n_terms)])
    for j in range(s.n_polys):
        rows = [tuple(r) for r in s.exps[off[j]:off[j + 1]]]
        assert len(set(rows)) == len(rows)  # distinct monomials
        d = deg[off[j]:off[j + 1]]
        if name == "cyclic10_shape":  # polynomial k of degree k; the last has two terms
            if j < dim - 1:
                assert s.n_terms[j] == 10 and np.all(d == j + 1)
            else:
                assert s.n_terms[j] == 2 and sorted(d.tolist()) == [0, dim]
        elif name == "nash8_shape":  # 130 monomials of degrees 1..7
            assert s.n_terms[j] == 130 and d.min() >= 1 and d.max() <= 7
        else:  # 246 monomials of degree 4
            assert s.n_terms[j] == 246 and np.all(d == 4)
    assert np.allclose(np.hypot(s.coef[:, 0], s.coef[:, 1]), 1.0, atol=1e-15)
    # the same seed gives the same system
    t = synth.config_system(name)
    assert np.array_equal(s.exps, t.exps) and np.array_equal(s.coef, t.coef)


@pytest.mark.parametrize("name", list(TABSUMCHAR))
def test_oracle_methods_agree_on_the_stand_ins(oracle_lib, name):
    s = synth.config_system(name)
    x = synth.unit_points(3, s.n_vars, 5, 2)
    v0, j0 = oracle_lib.eval_(s, x, method="naive")
    v1, j1 = oracle_lib.eval_(s, x, method="speelpenning")
    mv, mj = oracle_lib.eval_magnitude(s, x)
    assert np.all(np.abs(v0 - v1).max(axis=(1, 2)) <= 1e-28 * mv)
    assert np.all(np.abs(j0 - j1).max(axis=(2, 3)) <= 1e-28 * mj)
