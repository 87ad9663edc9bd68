"""Parity of the CUDA evaluation kernel (ht_eval_diff) with the oracle.

Tolerance: relative 1e-12 (D), 1e-26 (DD), 1e-55 (QD), relative to the sum of
the moduli of each output's terms (condition-aware: a plain |value| scale
would punish the cancellation every random system has)."""
import numpy as np
import pytest

import oracle
import synth
from parity import TOL, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ht():
    from paper_1505_00383_gb300 import _build, ht as binding
    _build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return binding


def _run(ht, system, x, L, host=False):
    nv, _, _, n = x.shape
    hs = ht.system_from(system, L)
    if host:
        val = np.empty((system.n_polys, 2, L, n))
        jac = np.empty((system.n_polys, nv, 2, L, n))
        ht.ht_eval_diff_host(hs, n, np.ascontiguousarray(x), val, jac)
        return val, jac
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    val = torch.full((system.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    jac = torch.full((system.n_polys, nv, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_eval_diff(hs, n, xd, val, jac)
    torch.cuda.synchronize()
    return val.cpu().numpy(), jac.cpu().numpy()


def _check(system, x, L, val, jac, pts=None):
    ov, oj = oracle.eval_(system, x, pts=pts)
    mv, mj = oracle.eval_magnitude(system, x, pts=pts)
    if pts is not None:
        val, jac = val[..., pts], jac[..., pts]
    assert np.all(np.isfinite(val)) and np.all(np.isfinite(jac))
    ev, ej = rel_err(val, ov, mv), rel_err(jac, oj, mj)
    assert ev <= TOL[L] and ej <= TOL[L], (L, ev, ej)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("name", ["plain_n6_d", "batched_n12_dd", "stress_n10_qd", "evaldiff_n32"])
def test_evaldiff_matches_oracle_several_tiles_and_ragged_tail(ht, name, L):
    s = synth.config_system(name)
    n = 32 * 3 + 5  # three full warps of points and a ragged tail of 5
    if name == "evaldiff_n32" and L == 4:
        n = 32 + 3
    x = synth.unit_points(101 + L, s.n_vars, n, L)
    val, jac = _run(ht, s, x, L)
    _check(s, x, L, val, jac)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_evaldiff_full_size_sampled(ht, L):
    """The 65,536-point sweep in the launch configuration the benchmark times,
    checked on sampled points (first, last, and random ones)."""
    s = synth.config_system("evaldiff_n32")
    n = 65536
    x = synth.unit_points(1000 + L, s.n_vars, n, L)
    val, jac = _run(ht, s, x, L)
    rng = synth.SplitMix64(9 + L)
    pts = np.unique(np.concatenate([[0, 31, 32, n - 1], rng.integers(0, n - 1, {1: 12, 2: 6, 4: 2}[L])]))
    _check(s, x, L, val, jac, pts=pts)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_edge_cases_wide_supports_constants_high_degree(ht, L):
    """A constant term, a monomial on 12 variables (the runtime-bounded path),
    exponents up to 9, a single point."""
    nv = 12
    exps = np.zeros((5, nv), np.int8)
    exps[1, :] = 1                       # all 12 variables
    exps[2, 3] = 9                       # x3^9
    exps[3, [0, 5, 11]] = [2, 3, 1]
    exps[4, 7] = 1
    coef = np.array([[0.5, -0.25], [1.0, 0.0], [-0.3, 0.7], [0.2, 0.2], [0.0, 1.0]])
    s = synth.System(nv, 2, np.array([3, 2], np.int32), exps, coef)
    for n in (1, 40):
        x = synth.unit_points(7, nv, n, L)
        val, jac = _run(ht, s, x, L)
        _check(s, x, L, val, jac)


def test_zero_points_is_a_noop_and_bad_args_are_rejected(ht):
    s = synth.config_system("plain_n6_d")
    hs = ht.system_from(s, 1)
    x = torch.zeros((6, 2, 1, 4), dtype=torch.float64, device="cuda")
    val = torch.zeros((6, 2, 1, 4), dtype=torch.float64, device="cuda")
    jac = torch.zeros((6, 6, 2, 1, 4), dtype=torch.float64, device="cuda")
    ht.ht_eval_diff(hs, 0, x, val, jac)
    with pytest.raises(ht.HTError) as e:
        ht.ht_eval_diff(hs, 4, x.cpu(), val, jac)  # host pointer for a device argument
    assert e.value.code == ht.HT_EINVAL
    with pytest.raises(ht.HTError):
        ht.ht_eval_diff(hs, -1, x, val, jac)
    with pytest.raises(ht.HTError):
        ht.ht_eval_diff(hs, 4, x, x, jac)  # overlapping input and output
    with pytest.raises(ht.HTError):
        ht.ht_create_system(0, 1, [1], np.zeros((1, 0), np.int8), np.zeros((1, 2, 1)), 1)
    with pytest.raises(ht.HTError):
        ht.ht_create_system(2, 1, [1], np.zeros((1, 2), np.int8), np.zeros((1, 2, 3)), 3)


@pytest.mark.parametrize("name,L,n,variant", [("batched_n12_dd", 1, 70, -1), ("batched_n12_dd", 4, 70, 2),
                                              ("batched_n12_dd", 2, 2 * 4096 + 37, 2), ("plain_n6_d", 1, 333, -1),
                                              ("evaldiff_n32", 1, 8 * 4096 + 5, -1), ("evaldiff_n32", 4, 1000, 2),
                                              ("evaldiff_n32", 2, 517, 3)])
def test_host_buffer_entry_point_matches(ht, name, L, n, variant):
    """The host entry evaluates blocks of polynomials (12 polynomials: blocks
    of 8 and 4; 32: four blocks of 8; 6: one block; the three-kernel variant:
    one block) and copies each block's rows back: the device entry's bits."""
    s = synth.config_system(name)
    x = synth.unit_points(55, s.n_vars, n, L)
    hs = ht.system_from(s, L)
    ht.ht_set_eval_config(hs, variant, 256 if variant == 2 else 0)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    v1 = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    j1 = torch.full((s.n_polys, s.n_vars, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_eval_diff(hs, n, xd, v1, j1)
    torch.cuda.synchronize()
    v2 = np.full((s.n_polys, 2, L, n), np.nan)
    j2 = np.full((s.n_polys, s.n_vars, 2, L, n), np.nan)
    ht.ht_eval_diff_host(hs, n, np.ascontiguousarray(x), v2, j2)
    assert np.array_equal(v1.cpu().numpy(), v2) and np.array_equal(j1.cpu().numpy(), j2)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_every_kernel_configuration_gives_identical_results(ht, L):
    """Compact and unrolled monomial bodies, 64/128/256 threads: the same
    operations in the same order, so bitwise identical outputs; the autotuner
    then keeps one of them (at these few points often the three kernels,
    bitwise the same too)."""
    s = synth.config_system("evaldiff_n32")
    n = 32 * 5 + 7
    x = synth.unit_points(3 + L, s.n_vars, n, L)
    hs = ht.system_from(s, L)
    xd = torch.from_numpy(x).cuda()
    ref = None
    for variant in (1, 0):
        for threads in (64, 128, 256):
            ht.ht_set_eval_config(hs, variant, threads)
            val = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
            jac = torch.full((s.n_polys, s.n_vars, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
            ht.ht_eval_diff(hs, n, xd, val, jac)
            out = (val.cpu().numpy(), jac.cpu().numpy())
            if ref is None:
                ref = out
            else:
                assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), (variant, threads)
    val = torch.empty((s.n_polys, 2, L, n), dtype=torch.float64, device="cuda")
    jac = torch.empty((s.n_polys, s.n_vars, 2, L, n), dtype=torch.float64, device="cuda")
    v, t, ms = ht.ht_tune_eval(hs, n, xd, val, jac, reps=1)
    assert v in (0, 1, 2, 3) and t in (64, 128, 256) and ms > 0
    if v in (0, 1, 3):  # the three kernels (3) take the FP64 bodies' operations in their order
        assert np.array_equal(val.cpu().numpy(), ref[0]) and np.array_equal(jac.cpu().numpy(), ref[1])
    else:  # the integer variant: its own arithmetic, same accuracy contract
        _check(s, x, L, val.cpu().numpy(), jac.cpu().numpy())


def _run_variant(ht, system, x, L, variant, threads=0):
    nv, _, _, n = x.shape
    hs = ht.system_from(system, L)
    ht.ht_set_eval_config(hs, variant, threads)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    val = torch.full((system.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    jac = torch.full((system.n_polys, nv, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_eval_diff(hs, n, xd, val, jac)
    torch.cuda.synchronize()
    return val.cpu().numpy(), jac.cpu().numpy()


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("name", ["plain_n6_d", "batched_n12_dd", "stress_n10_qd", "evaldiff_n32"])
def test_integer_variant_matches_oracle(ht, name, L):
    """The integer-pipe evaluation (multi-limb integer complex arithmetic with
    fixed-point accumulation) meets the same tolerance against the oracle."""
    s = synth.config_system(name)
    n = 32 * 3 + 5
    if name == "evaldiff_n32" and L == 4:
        n = 32 + 3
    x = synth.unit_points(201 + L, s.n_vars, n, L)
    val, jac = _run_variant(ht, s, x, L, 2)
    _check(s, x, L, val, jac)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("name", ["plain_n6_d", "stress_n10_qd", "evaldiff_n32"])
def test_integer_block_organisation_is_bitwise_identical(ht, name, L):
    """Integer limbs per unit (128-thread CTAs: lane = point, local copies of
    the point) and per block of 32 points (256-thread CTAs: the block's points
    in shared memory, polynomials dealt to warps) add the same exact terms:
    the same bits, ragged last block included."""
    s = synth.config_system(name)
    n = 32 * 4 + 11 if L < 4 else 32 + 11
    x = synth.unit_points(91 + L, s.n_vars, n, L)
    a = _run_variant(ht, s, x, L, 2, 128)
    b = _run_variant(ht, s, x, L, 2, 256)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    _check(s, x, L, b[0], b[1])


@pytest.mark.parametrize("L", [1, 2, 4])
def test_integer_variant_full_size_sampled(ht, L):
    s = synth.config_system("evaldiff_n32")
    n = 65536
    x = synth.unit_points(3000 + L, s.n_vars, n, L)
    val, jac = _run_variant(ht, s, x, L, 2)
    rng = synth.SplitMix64(19 + L)
    pts = np.unique(np.concatenate([[0, 31, 32, n - 1], rng.integers(0, n - 1, {1: 12, 2: 6, 4: 2}[L])]))
    _check(s, x, L, val, jac, pts=pts)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_integer_variant_edge_cases(ht, L):
    """Constant terms, a 12-variable support, exponent 9, values spread over
    many binades and exact zeros among the inputs."""
    nv = 12
    exps = np.zeros((5, nv), np.int8)
    exps[1, :] = 1
    exps[2, 3] = 9
    exps[3, [0, 5, 11]] = [2, 3, 1]
    exps[4, 7] = 1
    coef = np.array([[0.5, -0.25], [1.0, 0.0], [-0.3, 0.7], [0.2, 0.2], [0.0, 1.0]])
    s = synth.System(nv, 2, np.array([3, 2], np.int32), exps, coef)
    x = synth.unit_points(8, nv, 40, L)
    rng = synth.SplitMix64(4)
    x *= 2.0 ** rng.integers(-20, 20, nv * 40).reshape(nv, 1, 1, 40).astype(np.float64)
    x[2, :, :, 5] = 0.0   # an exact zero variable at one point
    val, jac = _run_variant(ht, s, x, L, 2)
    _check(s, x, L, val, jac)
    vb, jb = _run_variant(ht, s, x, L, 2, 256)
    assert np.array_equal(val, vb) and np.array_equal(jac, jb)



@pytest.mark.parametrize("L", [1, 2, 4])
def test_maximum_sizes_integer_variant_limit(ht, L):
    """64 variables (the integer variant's largest system) with a 64-variable
    monomial and exponent 127: the compact and unrolled FP64 bodies and both
    integer organisations match the oracle, with one warp and a ragged tail
    of points; FP64 bodies agree bitwise, and so do the integer ones."""
    s = synth.extreme_system(77, 64, 3)
    n = 32 + 5
    x = synth.unit_points(17 + L, 64, n, L)
    outs = {}
    for variant, threads in ((1, 128), (0, 128), (2, 128), (2, 256)):
        val, jac = _run_variant(ht, s, x, L, variant, threads)
        _check(s, x, L, val, jac)
        outs[(variant, threads)] = (val, jac)
    for a, b in (((1, 128), (0, 128)), ((2, 128), (2, 256))):
        assert np.array_equal(outs[a][0], outs[b][0]) and np.array_equal(outs[a][1], outs[b][1]), (a, b)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_maximum_sizes_255_variables(ht, L):
    """255 variables, the largest system: the FP64 bodies match the oracle;
    the integer variant (at most 64 variables) is refused with
    HT_EUNSUPPORTED and the system keeps evaluating with its FP64 bodies."""
    s = synth.extreme_system(78, 255, 4)
    n = 32 + 3
    x = synth.unit_points(27 + L, 255, n, L)
    a = _run_variant(ht, s, x, L, 1, 128)
    _check(s, x, L, *a)
    hs = ht.system_from(s, L)
    with pytest.raises(ht.HTError) as e:
        ht.ht_set_eval_config(hs, 2, 0)
    assert e.value.code == ht.HT_EUNSUPPORTED
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    val = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    jac = torch.full((s.n_polys, 255, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_eval_diff(hs, n, xd, val, jac)
    assert np.array_equal(val.cpu().numpy(), a[0]) and np.array_equal(jac.cpu().numpy(), a[1])


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("name", ["cyclic10_shape", "nash8_shape", "pieri44_shape"])
def test_paper_shaped_systems_match_oracle(ht, name, variant, L):
    """The stand-ins shaped like the paper's three applications (Section 4.2,
    Table tabsumchar), at the largest point count of its evaluation tables
    (3,000 points) on sampled points, and at the smallest (10 points) on all,
    with the FP64 bodies (variant 1) and the integer limbs (variant 2)."""
    s = synth.config_system(name)
    for n, sample in ((3000, {1: 12, 2: 6, 4: 3}[L]), (10, None)):
        x = synth.unit_points(500 + L + n, s.n_vars, n, L)
        hs = ht.system_from(s, L)
        ht.ht_set_eval_config(hs, variant, 256 if variant == 2 else 0)
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        val = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
        jac = torch.full((s.n_polys, s.n_vars, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
        ht.ht_eval_diff(hs, n, xd, val, jac)
        torch.cuda.synchronize()
        pts = None
        if sample is not None:
            rng = synth.SplitMix64(77 + L)
            pts = np.unique(np.concatenate([[0, 31, n - 1], rng.integers(0, n - 1, sample)]))
        _check(s, x, L, val.cpu().numpy(), jac.cpu().numpy(), pts=pts)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("name", ["evaldiff_n32", "cyclic10_shape", "nash8_shape", "stress_n10_qd"])
def test_unfused_three_kernels_equal_the_fused_kernel(ht, name, L):
    """The paper's coeff / mon / sum organisation over a device workspace
    (ht_eval_diff_unfused) takes the fused FP64 bodies' operations in their
    order: bitwise the same values and Jacobian, on three warps of points and
    a ragged tail; and within the oracle's tolerance."""
    s = synth.config_system(name)
    n = 32 * 3 + 5
    x = synth.unit_points(211 + L, s.n_vars, n, L)
    hs = ht.system_from(s, L)
    ht.ht_set_eval_config(hs, 1, 0)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = []
    for unfused in (False, True):
        val = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
        jac = torch.full((s.n_polys, s.n_vars, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
        if unfused:
            st = ht.ht_unfused_stats()
            ht.ht_eval_diff_unfused(hs, n, xd, val, jac, st)
            d = st.as_dict()
            assert d["ms_mon"] > 0 and d["bytes_mon"] > d["bytes_coeff"] > 0 and d["bytes_sum"] > 0
        else:
            ht.ht_eval_diff(hs, n, xd, val, jac)
        torch.cuda.synchronize()
        out.append((val.cpu().numpy(), jac.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    _check(s, x, L, out[1][0], out[1][1])
    # the same organisation as ht_eval_diff's variant 3
    ht.ht_set_eval_config(hs, 3, 0)
    val = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    jac = torch.full((s.n_polys, s.n_vars, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
    ht.ht_eval_diff(hs, n, xd, val, jac)
    torch.cuda.synchronize()
    assert np.array_equal(val.cpu().numpy(), out[0][0]) and np.array_equal(jac.cpu().numpy(), out[0][1])


def test_unfused_in_chunks_at_full_size(ht):
    """65,536 points in QD need 29 workspace chunks of 2,304 points: points
    at chunk edges and in the last chunk against the fused kernel, bit for
    bit."""
    s = synth.config_system("evaldiff_n32")
    n, L = 65536, 4
    x = torch.from_numpy(synth.unit_points(1004, s.n_vars, n, L)).cuda()
    hs = ht.system_from(s, L)
    ht.ht_set_eval_config(hs, 1, 0)
    res = []
    for unfused in (False, True):
        val = torch.full((s.n_polys, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
        jac = torch.full((s.n_polys, s.n_vars, 2, L, n), np.nan, dtype=torch.float64, device="cuda")
        (ht.ht_eval_diff_unfused if unfused else ht.ht_eval_diff)(hs, n, x, val, jac)
        torch.cuda.synchronize()
        pts = torch.tensor([0, 2303, 2304, 40000, 64511, 64512, n - 1], device="cuda")
        res.append((val[..., pts].cpu().numpy(), jac[..., pts].cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
