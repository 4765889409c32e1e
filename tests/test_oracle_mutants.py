"""The oracle's pins catch plausible mistakes.  Each case copies oracle/ to a
temporary directory, plants one slip in the copy of oracle.cpp (a flipped
sign, a dropped term, a transposed operand, a wrong constant or index),
builds that copy and runs against it the pins that should notice; at least
one of them must fail.  The planted copies live only in the test's
temporary directory."""
import importlib.util
import shutil
import sys
import uuid
from pathlib import Path

import pytest

from paper_2003_12861_gb300 import workloads as W
import test_oracle_binned as PB
import test_oracle_expr as PE
import test_oracle_extended as PX
import test_oracle_fit_pins as PF
import test_oracle_mlp as PM
import test_oracle_pins as P

ORACLE = Path(__file__).resolve().parent.parent / "oracle"


def load_mutant(tmp_path, old, new, file="oracle.cpp"):
    d = tmp_path / "oracle_mutant"
    shutil.copytree(ORACLE, d, ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    src = (d / file).read_text()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    (d / file).write_text(src.replace(old, new))
    name = f"oracle_mutant_{uuid.uuid4().hex}"
    spec = importlib.util.spec_from_file_location(name, d / "__init__.py", submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def leaf_cases(kind):
    return [c for c in P.LEAF_CASES if c[0] == kind]


def norm_pins(kind):
    return [lambda m, c=c: P.test_leaf_norm_matches_quadrature(m, *c) for c in leaf_cases(kind)]


def dnorm_pins(kind):
    return [lambda m, c=c: P.test_leaf_norm_derivative_matches_richardson(m, *c) for c in leaf_cases(kind)]


CONV_PARAMS = [([1.5, 0.0, 0.05], 0.01), ([1.5, 0.0, 0.05], 0.3), ([0.4, 0.3, 0.2], 1.0)]

MUTANTS = {
    # GAUSSEXP: d A / d tau with the sign of its first term flipped
    "gaussexp_dA_dtau_sign": (
        "{-sigma * sigma / (tau * tau * tau) + (t - mu) / (tau * tau), 1.0 / tau, sigma / (tau * tau)}",
        "{sigma * sigma / (tau * tau * tau) + (t - mu) / (tau * tau), 1.0 / tau, sigma / (tau * tau)}",
        lambda: dnorm_pins("gaussexp") + [lambda m: P.test_gradient_richardson(m, "decay_model")]),
    # GAUSSEXP: d z / d sigma without its 1/tau term
    "gaussexp_dz_dsigma_dropped_term": (
        "(1.0 / tau + (t - mu) / (sigma * sigma)) / kSqrt2}",
        "((t - mu) / (sigma * sigma)) / kSqrt2}",
        lambda: dnorm_pins("gaussexp") + [lambda m: P.test_gradient_richardson(m, "decay_model")]),
    # GAUSSEXP: the erfc argument with its operands transposed
    "gaussexp_z_transposed": (
        "  const double z = (s - u) / kSqrt2;\n  const double g = std::exp(-0.5 * u * u);",
        "  const double z = (u - s) / kSqrt2;\n  const double g = std::exp(-0.5 * u * u);",
        lambda: [lambda m, a=a: P.test_gaussexp_shape_is_the_convolution(m, *a) for a in CONV_PARAMS]),
    # erfcx: the continued fraction's partial numerators one index off
    "erfcx_continued_fraction_index": (
        "for (int k = 400; k >= 1; --k) t = z + (0.5 * k) / t;",
        "for (int k = 400; k >= 1; --k) t = z + (0.5 * (k + 1)) / t;",
        lambda: [lambda m, a=a: P.test_gaussexp_shape_is_the_convolution(m, *a)
                 for a in (([1.0, 0.5, 0.1], -0.4), ([1.0, 0.5, 0.05], -0.2))]),
    # EXP: the series of the truncated exponential's mean with 1/6 for 1/12
    "exp_mean_series_coefficient": (
        "return 0.5 + y / 12.0 - y * y * y / 720.0;", "return 0.5 + y / 6.0 - y * y * y / 720.0;",
        lambda: dnorm_pins("exp")),
    # EXPR quadrature: Gauss-Legendre weights without their factor 2
    "gauss_legendre_weights": (
        "w[i] = 2.0 / ((1.0 - z * z) * dp * dp);", "w[i] = 1.0 / ((1.0 - z * z) * dp * dp);",
        lambda: [lambda m, a=a: PE.test_expr_normalisation_closed_form(m, a) for a in (0.0, 0.7)]),
    # CHEB: the integral of T_k with 1 + k^2 for 1 - k^2
    "cheb_integral_sign": (
        "2.0 / (1.0 - (double)k * k)", "2.0 / (1.0 + (double)k * k)",
        lambda: norm_pins("cheb")),
    # POLY: the power rule divided by k instead of k + 1
    "poly_integral_power": (
        "(std::pow(b, k + 1) - std::pow(a, k + 1)) / (k + 1);", "(std::pow(b, k + 1) - std::pow(a, k + 1)) / k;",
        lambda: norm_pins("poly") + [P.test_worked_example_gauss_poly1]),
    # GAUSS: the normal mass on a range right of the mean with its ends swapped
    "normal_mass_ends_swapped": (
        "if (alpha >= 0) return 0.5 * (std::erfc(alpha / kSqrt2) - std::erfc(beta / kSqrt2));",
        "if (alpha >= 0) return 0.5 * (std::erfc(beta / kSqrt2) - std::erfc(alpha / kSqrt2));",
        lambda: norm_pins("gauss")),
    # GAUSS: d log g / d sigma as u / sigma instead of u^2 / sigma
    "gauss_dsigma_power": (
        "df[1] = *f * u * u / q[1];", "df[1] = *f * u / q[1];",
        lambda: [lambda m: P.test_gradient_richardson(m, "gauss_poly1_model")]),
    # SUM: the last component weighted by the sum of the others' fractions
    "sum_last_fraction": (
        "const double fl = 1.0 - frac_sum;", "const double fl = frac_sum;",
        lambda: [P.test_sum_prod_special_cases, lambda m: P.test_nll_brute_force_mpmath(m, "gauss_poly1_model")]),
    # SUM: the fraction's derivative with its sign flipped
    "sum_fraction_derivative_sign": (
        "if (fi >= 0) r.d[fi] += val[n.in[j]].v - last.v;", "if (fi >= 0) r.d[fi] += last.v - val[n.in[j]].v;",
        lambda: [lambda m: P.test_gradient_richardson(m, "gauss_poly1_model")]),
    # Philox: one bit of a round multiplier
    "philox_multiplier": (
        "(uint64_t)0xD2511F53u * c[0]", "(uint64_t)0xD2511F52u * c[0]",
        lambda: [lambda m, k=k: P.test_philox_known_answers(m, *k) for k in P.PHILOX_KAT]),
    # histogram: bins shifted by half a bin
    "hist64_offset": (
        "double t = (x[i] - lo) * scale;", "double t = (x[i] - lo) * scale + 0.5;",
        lambda: [P.test_hist64_matches_numpy]),
    # accept-reject with the comparison reversed
    "accept_reject_reversed": (
        "if (y < factor_density(m, nm, theta, fac[j], xv, val)) {",
        "if (y > factor_density(m, nm, theta, fac[j], xv, val)) {",
        lambda: [lambda m: P.test_generator_matches_pdf_histogram(m, "gauss_poly1_model")]),
    # EXPR: the quotient rule with the sign of the divisor's term flipped
    "expr_quotient_rule_sign": (
        "for (int k = 0; k < np; ++k) a.d[k] = (a.d[k] - v * b.d[k]) / b.v;",
        "for (int k = 0; k < np; ++k) a.d[k] = (a.d[k] + v * b.d[k]) / b.v;",
        lambda: [lambda m: PE.test_expr_gaussian_equals_the_builtin_gaussian(m, W.GAUSS_POLY1_TRUE)]),
    # EXPR: the power's derivative without its factor a^b
    "expr_pow_derivative_factor": (
        "a.d[k] = v * (b.d[k] * la + b.v * a.d[k] / a.v);", "a.d[k] = (b.d[k] * la + b.v * a.d[k] / a.v);",
        lambda: [lambda m, a=a: PE.test_expr_normalisation_closed_form(m, a) for a in (0.7, 2.3)]),
    # POISSON: the derivative of its mass with lambda's sign flipped
    "poisson_norm_derivative_sign": (
        "ds.add(pk * (k / lam - 1.0));", "ds.add(pk * (k / lam + 1.0));",
        lambda: [PX.test_poisson_gradient_and_mle]),
    # EXTEND: the extended term's log with the wrong sign
    "extended_term_sign": (
        "ext = nu - (double)N * std::log(nu);", "ext = nu + (double)N * std::log(nu);",
        lambda: [PX.test_extended_term_and_closed_form_mle]),
    # EXTEND: the yield's derivative with N / nu added instead of subtracted
    "extended_derivative_sign": (
        "sg[fi].add(-(1.0 - (double)N / nu));", "sg[fi].add(-(1.0 + (double)N / nu));",
        lambda: [PX.test_extended_term_and_closed_form_mle]),
    # covariance: the central difference of the gradient without its 2
    "covariance_difference_step": (
        "Hs[j * P + k] = (gp[j] - gm[j]) / (2.0 * hstep);", "Hs[j * P + k] = (gp[j] - gm[j]) / hstep;",
        lambda: [PF.test_decay_fit_minimum_and_covariance]),
    # generation: an accept-reject bound below the density's maximum
    "generation_bound_too_low": (
        "bounds[j] = 1.2 * mx;", "bounds[j] = 0.6 * mx;",
        lambda: [lambda m: P.test_generator_matches_pdf_histogram(m, "decay_model")]),
    # fitter: the bound transform mapping onto half of the range
    "fit_bound_transform_scale": (
        "th[k] = bounded[k] ? lo[k] + (hi[k] - lo[k]) * (std::sin(x[k]) + 1.0) * 0.5 : x[k];",
        "th[k] = bounded[k] ? lo[k] + (hi[k] - lo[k]) * (std::sin(x[k]) + 1.0) * 0.25 : x[k];",
        lambda: [P.test_fraction_only_fit_matches_bounded_scalar_minimiser, P.test_gaussian_mle_closed_form]),
}


# Slips in the Python oracles (binned likelihood, MLP): the pins' modules
# import those oracles by name, so the case points that name at the copy.
PY_MUTANTS = {
    # binned: linear extrapolation of g beyond one sigma shifted by 2
    "binned_extrapolation_offset": (
        "binned.py", "return 2.0 * abs(alpha) - 1.0, 2.0 if alpha > 0 else -2.0",
        "return 2.0 * abs(alpha) + 1.0, 2.0 if alpha > 0 else -2.0", PB, "B",
        lambda: [PB.test_nominal_and_extrapolation] +
        [lambda a=a: PB.test_interpolation_is_continuously_differentiable(a) for a in (-1.0, 1.0)]),
    # binned: the normsys quadratic coefficient from the difference of the logs
    "binned_normsys_coefficient": (
        "binned.py", "b = 0.5 * (np.log(m.k_hi) + np.log(m.k_lo))", "b = 0.5 * (np.log(m.k_hi) - np.log(m.k_lo))",
        PB, "B", lambda: [lambda a=a: PB.test_interpolation_reaches_the_variations_at_one_sigma(a) for a in (1.0, -1.0)]),
    # binned: the histosys quadratic coefficient without the nominal subtracted
    "binned_histosys_coefficient": (
        "binned.py", "b = 0.5 * (np.asarray(m.h_hi) + np.asarray(m.h_lo)) - h",
        "b = 0.5 * (np.asarray(m.h_hi) + np.asarray(m.h_lo))",
        PB, "B", lambda: [lambda a=a: PB.test_interpolation_reaches_the_variations_at_one_sigma(a) for a in (1.0, -1.0)]),
    # binned: the Poisson term's derivative weight with n / nu added
    "binned_poisson_weight_sign": (
        "binned.py", "w = 1.0 - n / nu", "w = 1.0 + n / nu", PB, "B",
        lambda: [lambda th=th: PB.test_gradient_richardson(th) for th in ([1.3, 0.4, -0.7],)]),
    # binned: the constraint without its factor 1/2 in the NLL
    "binned_constraint_half": (
        "binned.py", "nll = terms.sum() + 0.5 * np.sum(theta[cons] ** 2)", "nll = terms.sum() + np.sum(theta[cons] ** 2)",
        PB, "B", lambda: [lambda th=th: PB.test_gradient_richardson(th) for th in ([1.3, 0.4, -0.7],)]),
    # MLP: GELU with sqrt(2) replaced by 2
    "mlp_gelu_scale": (
        "mlp.py", "return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))", "return 0.5 * z * (1.0 + erf(z / 2.0))",
        PM, "M", lambda: [PM.test_gelu_matches_torch]),
    # MLP: the backward pass through the weights with its columns reversed (a mis-indexed weight)
    "mlp_backward_transpose": (
        "mlp.py", "d = _r(dz, rounding) @ _r(W, rounding).T", "d = (_r(dz, rounding) @ _r(W, rounding).T)[:, ::-1]",
        PM, "M", lambda: [PM.test_backward_matches_finite_differences]),
    # MLP: Adam's first-moment bias correction with beta2
    "mlp_adam_bias_correction": (
        "mlp.py", "mh = m / (1 - b1 ** t)", "mh = m / (1 - b2 ** t)", PM, "M", lambda: [PM.test_adam_matches_torch]),
    # MLP: bfloat16 rounding that always rounds half up
    "mlp_bf16_ties": (
        "mlp.py", "r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16",
        PM, "M", lambda: [PM.test_bf16_rounding_matches_torch]),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_a_planted_mistake_in_the_python_oracles(tmp_path, monkeypatch, name):
    file, old, new, test_mod, attr, pins = PY_MUTANTS[name]
    mod = load_mutant(tmp_path, old, new, file=file)
    sub = importlib.import_module(f"{mod.__name__}.{file[:-3]}")
    monkeypatch.setattr(test_mod, attr, sub)
    failed = []
    for pin in pins():
        try:
            pin()
        except (AssertionError, RuntimeError, ValueError) as e:
            failed.append(type(e).__name__)
            break
    assert failed, f"no pin noticed the planted mistake '{name}'"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_a_planted_mistake(tmp_path, name):
    old, new, pins = MUTANTS[name]
    mod = load_mutant(tmp_path, old, new)
    failed = []
    for pin in pins():
        try:
            pin(mod)
        except (AssertionError, RuntimeError, ValueError) as e:
            failed.append(type(e).__name__)
            break
    assert failed, f"no pin noticed the planted mistake '{name}'"


def test_an_unplanted_copy_passes_the_same_pins(tmp_path):
    """The control: the copy without a planted mistake passes every pin the
    cases above run, so what they catch is the mistake, not the copy."""
    mod = load_mutant(tmp_path, "TEST INFRASTRUCTURE ONLY.", "TEST INFRASTRUCTURE ONLY.")
    for name, (_, _, pins) in sorted(MUTANTS.items()):
        for pin in pins():
            pin(mod)


def test_unplanted_python_oracles_pass_the_same_pins(tmp_path, monkeypatch):
    mod = load_mutant(tmp_path, "TEST INFRASTRUCTURE ONLY.", "TEST INFRASTRUCTURE ONLY.")
    for name, (file, _, _, test_mod, attr, pins) in sorted(PY_MUTANTS.items()):
        monkeypatch.setattr(test_mod, attr, importlib.import_module(f"{mod.__name__}.{file[:-3]}"))
        for pin in pins():
            pin()
