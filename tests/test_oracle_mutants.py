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

import test_oracle_pins as P

ORACLE = Path(__file__).resolve().parent.parent / "oracle"


def load_mutant(tmp_path, old, new):
    d = tmp_path / "oracle_mutant"
    shutil.copytree(ORACLE, d, ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    src = (d / "oracle.cpp").read_text()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    (d / "oracle.cpp").write_text(src.replace(old, new))
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
    # fitter: the bound transform mapping onto half of the range
    "fit_bound_transform_scale": (
        "th[k] = bounded[k] ? lo[k] + (hi[k] - lo[k]) * (std::sin(x[k]) + 1.0) * 0.5 : x[k];",
        "th[k] = bounded[k] ? lo[k] + (hi[k] - lo[k]) * (std::sin(x[k]) + 1.0) * 0.25 : x[k];",
        lambda: [P.test_fraction_only_fit_matches_bounded_scalar_minimiser, P.test_gaussian_mle_closed_form]),
}


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
