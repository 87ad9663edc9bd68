"""Planted mistakes in the oracle, on the CPU.

Each entry copies the oracle's source with one plausible mistake (a dropped
term, a wrong sign, a wrong index or constant), compiles the copy with the
oracle's own flags, and runs one pin against it: the pin must fail.  This
checks that the pins would catch such mistakes in the oracle, not only that
the oracle passes them.  The mistakes are planted in the oracle only; the
CUDA library is not involved.
"""
import os
import re
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import test_oracle_arith as A
import test_oracle_eval as E
import test_oracle_mgs_start_compact as M
import test_oracle_mlp as N
import test_oracle_track as T

# name: (original line, planted mistake, the pin that must fail)
MUTANTS = {
    "accumulator drops the rounding error of a sum": (
        "double lo = y - (hi - x);", "double lo = 0.0 * (y - (hi - x));",
        lambda o: A.test_real_op_against_exact_rationals(o, 2, "add")),
    "Dekker product drops the low-by-low term": (
        "e = ((ah * bh - p) + ah * bl + al * bh) + al * bl;", "e = ((ah * bh - p) + ah * bl + al * bh);",
        lambda o: A.test_real_op_against_exact_rationals(o, 2, "mul")),
    "division stops after one quotient digit": (
        "for (int it = 0; it < L + 2; ++it) {", "for (int it = 0; it < 1; ++it) {",
        lambda o: A.test_real_op_against_exact_rationals(o, 2, "div")),
    "square root takes one Newton step": (
        "for (int it = 0; it < L; ++it) y = rmul<L>", "for (int it = 0; it < 1; ++it) y = rmul<L>",
        lambda o: A.test_sqrt_against_exact(o, 4)),
    "product rule keeps the differentiated exponent": (
        "int e = a[l] - (l == i ? 1 : 0);", "int e = a[l] - (l == i ? 0 : 0);",
        lambda o: E.test_eval_against_exact_brute_force(o, 1, "naive")),
    "reverse mode takes the wrong forward product": (
        "slots[out] = cmul<L>(slots[j - 2], slots[k - 1]);", "slots[out] = cmul<L>(slots[j - 1], slots[k - 1]);",
        lambda o: E.test_tabmoneval_slots(o)),
    "common factor misses one power": (
        "for (int e = 1; e < a[i]; ++e) cf = cmul<L>(cf, x[i]);", "for (int e = 2; e < a[i]; ++e) cf = cmul<L>(cf, x[i]);",
        lambda o: E.test_eval_against_exact_brute_force(o, 1, "speelpenning")),
    "derivative not scaled by the exponent": (
        "C<L> scaled = cscale<L>(cf, rfrom<L>((double)ex[r]));", "C<L> scaled = cf;",
        lambda o: E.test_eval_against_exact_brute_force(o, 1, "speelpenning")),
    "tolerance scale keeps the differentiated exponent": (
        "dd *= std::pow(ax[l], (double)(a[l] - (l == i ? 1 : 0)));", "dd *= std::pow(ax[l], (double)(a[l]));",
        lambda o: E.test_magnitude_scale_is_the_sum_of_term_moduli(o)),
    "tolerance scale squares the exponent factor": (
        "double dd = c * a[i];", "double dd = c * a[i] * a[i];",
        lambda o: E.test_magnitude_scale_is_the_sum_of_term_moduli(o)),
    "exact difference adds instead of subtracting": (
        "s.add(-b[i * L + l]);", "s.add(b[i * L + l]);",
        lambda o: A.test_value_diff_is_exact_difference(o, 2)),
    "Gram-Schmidt projection without the conjugate": (
        "r = cadd<L>(r, cconjmul<L>(M[(size_t)i * W + q], M[(size_t)i * W + j]));",
        "r = cadd<L>(r, cmul<L>(M[(size_t)i * W + q], M[(size_t)i * W + j]));",
        lambda o: M.test_mgs_matches_lstsq_in_double(o, 6, 6)),
    "back substitution adds instead of subtracting": (
        "acc = csub<L>(acc, cmul<L>(Rm[(size_t)q * W + j], xk[j]));",
        "acc = cadd<L>(acc, cmul<L>(Rm[(size_t)q * W + j], xk[j]));",
        lambda o: M.test_mgs_matches_lstsq_in_double(o, 6, 6)),
    "roots of unity at half the angle": (
        "double th = 2.0 * pi * (double)k / (double)d;", "double th = pi * (double)k / (double)d;",
        lambda o: M.test_start_solutions_are_the_roots_of_unity(o, 1, [5, 3])),
    "path digits in the wrong radix": (
        "    r /= deg[i];\n", "    r /= 2;\n",
        lambda o: M.test_start_solutions_are_the_roots_of_unity(o, 1, [3, 2])),
    "roots of unity left at double precision": (
        "for (int it = 0; it < 3; ++it) {\n      C<L> zd1", "for (int it = 0; it < 0; ++it) {\n      C<L> zd1",
        lambda o: M.test_start_solutions_are_the_roots_of_unity(o, 2, [5, 3])),
    "complex division without the conjugate": (
        "C<L> num = cconjmul<L>(b, a);  // conj(b) a", "C<L> num = cmul<L>(b, a);  // conj(b) a",
        lambda o: M.test_start_solutions_are_the_roots_of_unity(o, 2, [5, 3])),
    "start system derivative on the wrong column": (
        "if (j == i) v = cadd<L>(v, cmul<L>(gs, dg));", "if (j == (i + 1) % n) v = cadd<L>(v, cmul<L>(gs, dg));",
        lambda o: T.test_homotopy_special_cases_and_affinity_in_t(o, 1)),
    "Adam without bias correction of the first moment": (
        "double c1 = 1.0 - std::pow(b1, step)", "double c1 = 1.0",
        lambda o: N.test_adam_first_step_moves_each_weight_by_lr(o)),
    "compaction keeps finished paths": (
        "if (status[i] == 0) path_idx[c++] = (int32_t)i;", "if (status[i] >= 0) path_idx[c++] = (int32_t)i;",
        lambda o: M.test_compaction_table_tabjobidx(o)),
    "homotopy weights g by t instead of 1 - t": (
        "C<L> gs = cscale<L>(H.gamma, omt);", "C<L> gs = cscale<L>(H.gamma, tt);",
        lambda o: T.test_homotopy_special_cases_and_affinity_in_t(o, 2)),
    "start system derivative d x^(d-1) off by one": (
        "C<L> dg = cscale<L>(xd1, rfrom<L>((double)H.d[i]));", "C<L> dg = cscale<L>(xd1, rfrom<L>((double)H.d[i] - 1.0));",
        lambda o: T.test_homotopy_special_cases_and_affinity_in_t(o, 2)),
    "predictor weights with the wrong sign": (
        "den = rmul<L>(den, rsub<L>(rfrom<L>(ht[base + j]), rfrom<L>(ht[base + i])));",
        "den = rmul<L>(den, rsub<L>(rfrom<L>(ht[base + i]), rfrom<L>(ht[base + j])));",
        lambda o: T.test_predictor_is_exact_on_polynomial_paths(o, 2, 4)),  # (-1)^(m-1): even m
    "step never grows after an accepted step": (
        "h = std::min(hmax, fup * h);", "h = std::min(hmax, h);",
        lambda o: T.test_step_control_worked_example(o, 1)),
    "step grows past its cap": (
        "h = std::min(hmax, fup * h);", "h = fup * h;",
        lambda o: T.test_step_control_worked_example(o, 1)),
    "rejection ignores the shrink factor": (
        "h = fdown * h;", "h = 0.5 * h;",
        lambda o: T.test_rejection_worked_example(o, 1, "update")),
    "acceptance ignores the residual": (
        "if (ndx <= tol_dx * sx && nres <= lim) {", "if (ndx <= tol_dx * sx) {",
        lambda o: T.test_rejection_worked_example(o, 1, "residual")),
    "acceptance ignores the update": (
        "if (ndx <= tol_dx * sx && nres <= lim) {", "if (nres <= lim) {",
        lambda o: T.test_rejection_worked_example(o, 1, "update")),
    "Newton step subtracts the update": (
        "for (int i = 0; i < n; ++i) x[i] = cadd<L>(x[i], dx[i]);", "for (int i = 0; i < n; ++i) x[i] = csub<L>(x[i], dx[i]);",
        lambda o: T.test_diagonal_system_closed_form(o, 1)),
    "divergence test never fires": (
        "if (norm_inf<L>(x.data(), n) > rdiv_) {", "if (norm_inf<L>(x.data(), n) > 1e300) {",
        lambda o: T.test_deficient_system_one_root_and_paths_to_infinity(o, 1)),
    "error bound takes every first-layer ReLU mask as certain": (
        "        dz1[i] = z1[i] > 0 ? g1[i] : 0.0;\n        edz1[i] = std::fabs(g1[i]) + eg1[i];",
        "        dz1[i] = z1[i] > 0 ? g1[i] : 0.0;\n        edz1[i] = eg1[i];",
        lambda o: N.test_error_bound_covers_the_reduced_precision_model(o)),
    "error bound without the rounding of the hidden activations": (
        "eh1[o] = rnd(h1[o], ez1[o], u_act);", "eh1[o] = ez1[o];",
        lambda o: N.test_error_bound_covers_the_reduced_precision_model(o)),
    "error bound accumulates at the activations' precision": (
        "const double acc = std::ldexp(1.0, -23), u32", "const double acc = std::ldexp(1.0, -8), u32",
        lambda o: N.test_error_bound_without_rounding_is_the_accumulation_error(o)),
    "error bound takes every ReLU mask as uncertain": (
        "      if (z2[i] > ez2[i]) {", "      if (z2[i] > 1e300) {",
        lambda o: N.test_error_bound_catches_planted_gradient_mistakes(o)),
    "tangent with the sign of dh/dt flipped": (
        "if (ht) ht[i] = csub<L>(fv[i], cmul<L>(H.gamma, g));", "if (ht) ht[i] = cadd<L>(fv[i], cmul<L>(H.gamma, g));",
        lambda o: T.test_tangent_of_the_diagonal_system_in_closed_form(o, 1)),
    "back substitution solves the first right-hand side twice": (
        "C<L> acc = Rm[(size_t)q * W + cols + k];", "C<L> acc = Rm[(size_t)q * W + cols];",
        lambda o: T.test_tangent_of_the_diagonal_system_in_closed_form(o, 2)),
    "Hermite predictor forgets to scale the first tangent by the interval": (
        "const R<L> b0 = rmul<L>(radd<L>(rsub<L>(u3, rmul<L>(two, u2)), u), d);",
        "const R<L> b0 = radd<L>(rsub<L>(u3, rmul<L>(two, u2)), u);",
        lambda o: T.test_tangent_predictors_are_exact_on_polynomial_paths(o, 1)),
    "network forward pass without the first ReLU": (
        "h1[o] = a > 0 ? a : 0;", "h1[o] = a;",
        lambda o: N.test_forward_is_a_relu_layer_stack(o)),
    "network backward pass without the ReLU mask": (
        "dz2[i] = z2[i] > 0 ? dh2[i] : 0;", "dz2[i] = dh2[i];",
        lambda o: N.test_gradient_matches_central_differences(o)),
}


def _slug(name):
    return re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = oracle.source()
    d = tmp_path_factory.mktemp("oracle_mutants")

    def build(item):
        name, (old, new, _) = item
        assert src.count(old) == 1, name  # the planted line is unambiguous
        return name, oracle.compile_variant(src.replace(old, new), str(d / (_slug(name) + ".so")))

    with ThreadPoolExecutor(max_workers=max(1, min(len(MUTANTS), os.cpu_count() or 1))) as ex:
        return dict(ex.map(build, MUTANTS.items()))


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_its_pin(oracle_lib, mutant_libs, name):
    pin = MUTANTS[name][2]
    with oracle.loaded_from(mutant_libs[name]):
        with pytest.raises(AssertionError):
            pin(oracle)
