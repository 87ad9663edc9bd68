"""Mixed-precision tracking (ht_track_refined; the "quality up" of Sections 1
and 4.4): track in double, refine in double double or quad double, track the
failures again in the high precision.  Its endpoints are compared with a
pure high-precision run and checked with the oracle's residuals."""
import numpy as np
import pytest

import oracle
import synth
from match import to_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ht():
    from paper_1505_00383_gb300 import _build, ht as binding
    _build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return binding


def _buffers(n, L, m):
    x = torch.full((n, 2, L, m), np.nan, dtype=torch.float64, device="cuda")
    st = torch.full((m,), 9, dtype=torch.int8, device="cuda")
    t = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    return x, st, t


def _runs(ht, name, Lh, m, h_min):
    s = synth.config_system(name)
    gam = synth.random_gamma(synth.CONFIGS[name]["seed"])
    lo, hi = ht.system_from(s, 1), ht.system_from(s, Lh)
    pl, ph = ht.ht_default_params(1, h_min=h_min), ht.ht_default_params(Lh, h_min=h_min)
    xr, sr, tr = _buffers(s.n_vars, Lh, m)
    rs = ht.ht_refine_stats()
    ht.ht_track_refined(lo, hi, s.degrees(), gam, m, 0, pl, ph, xr, sr, tr, rs)
    xh, sh, th = _buffers(s.n_vars, Lh, m)
    ht.ht_track_paths(hi, s.degrees(), gam, m, 0, None, ph, xh, sh, th)
    xl, sl, tl = _buffers(s.n_vars, 1, m)
    ht.ht_track_paths(lo, s.degrees(), gam, m, 0, None, pl, xl, sl, tl)
    torch.cuda.synchronize()
    cpu = lambda *a: [v.cpu().numpy() for v in a]
    return s, cpu(xr, sr, tr), cpu(xh, sh, th), cpu(xl, sl, tl), rs.as_dict()


def _same_sets(A, B, tol=1e-10):
    """One-to-one nearest-neighbour pairing of two endpoint sets ([m][n]
    complex) within tol max(1, |a|_inf)."""
    from scipy.spatial import cKDTree
    if A.shape != B.shape:
        return False
    emb = lambda X: np.concatenate([X.real, X.imag], axis=1)
    d, j = cKDTree(emb(B)).query(emb(A), k=1, p=np.inf)
    scale = np.maximum(1.0, np.max(np.abs(A), axis=1))
    return bool(np.all(d <= tol * scale) and np.unique(j).size == j.size)


def _residual_ok(s, x, L, ids, tol):
    """|f(x)| of the refined endpoints by the oracle, relative to the sum of
    the term moduli, at most tol."""
    val, _ = oracle.eval_(s, np.ascontiguousarray(x[..., ids]))
    mag, _ = oracle.eval_magnitude(s, np.ascontiguousarray(x[..., ids]))
    r = np.hypot(val[:, 0, 0, :], val[:, 1, 0, :]) / np.maximum(mag, 1e-300)
    return float(np.max(r)) <= tol, float(np.max(r))


@pytest.mark.parametrize("name,Lh,m,h_min", [("batched_n12_dd", 2, 4096, 1e-6), ("stress_n10_qd", 4, 1024, 1e-9)])
def test_refined_run_equals_the_high_precision_run(ht, name, Lh, m, h_min):
    s, (xr, sr, tr), (xh, sh, th), (xl, sl, tl), rs = _runs(ht, name, Lh, m, h_min)
    for code in (1, -1, -2):
        assert np.sum(sr == code) == np.sum(sh == code), (code, rs)
    assert rs["converged"] == np.sum(sr == 1) and rs["lo_converged"] == np.sum(sl == 1)
    conv = sr == 1
    assert _same_sets(to_complex(xr)[conv], to_complex(xh)[sh == 1])
    assert np.all(tr[conv] == 1.0)
    # the refined endpoints carry the high precision's accuracy: residuals at
    # the working precision's scale on a sample (checked by the oracle)
    ids = np.flatnonzero(conv)[:: max(1, int(conv.sum()) // 48)]
    tol = {2: 1e-20, 4: 1e-40}[Lh]  # refinement stops at updates of 1e-24 / 1e-48 relative
    ok, r = _residual_ok(s, xr, Lh, ids, tol)
    assert ok, r
    # the double endpoints alone are only accurate to double precision
    # (residuals evaluated in the high precision)
    xl_hi = np.zeros(xl.shape[:2] + (Lh,) + xl.shape[3:])
    xl_hi[:, :, 0, :] = xl[:, :, 0, :]
    okd, rd = _residual_ok(s, xl_hi, Lh, ids, tol)
    assert not okd and 1e-18 < rd < 1e-12, rd


def test_failed_paths_are_tracked_again_like_the_high_precision_run(ht):
    """n = 6 with the step floor 0.01: most paths fail in double.  Those are
    tracked again in double double from their start points and equal the
    pure double double run's paths bit for bit."""
    s, (xr, sr, tr), (xh, sh, th), (xl, sl, tl), rs = _runs(ht, "plain_n6_d", 2, 64, 0.01)
    again = sl != 1
    assert again.sum() > 0 and rs["retracked"] >= again.sum()
    assert np.array_equal(sr[again], sh[again])
    assert np.array_equal(xr[..., again], xh[..., again], equal_nan=True)
    assert np.array_equal(tr[again], th[again])
    kept = ~again & (sh == 1)
    d = np.max(np.abs(to_complex(xr)[kept] - to_complex(xh)[kept]), axis=1)
    assert np.all(d <= 1e-10 * np.maximum(1.0, np.max(np.abs(to_complex(xh)[kept]), axis=1)))


def test_refined_rejects_mismatched_systems(ht):
    a = ht.system_from(synth.config_system("plain_n6_d"), 1)
    b = ht.system_from(synth.config_system("batched_n12_dd"), 2)
    c = ht.system_from(synth.config_system("plain_n6_d"), 1)
    x, st, t = _buffers(6, 2, 4)
    for lo, hi in ((a, b), (a, c)):
        with pytest.raises(ht.HTError) as e:
            ht.ht_track_refined(lo, hi, [2] * 6, (1.0, 0.0), 4, 0, None, None, x, st, t)
        assert e.value.code == ht.HT_EINVAL
