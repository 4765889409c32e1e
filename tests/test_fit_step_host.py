"""The fit's quasi-Newton state machine (csrc/fit_step.h), which the host
driver and the device step share, checked on the CPU: its own sine and
cosine against the C library, and whole fits whose minimum is known in
closed form (a quadratic, Rosenbrock's function under bounds, a minimum
beyond a bound), plus the domain and max_evals exits."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "fit_step_check.cpp")


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("fit_step") / "fit_step_check")
    cmd = [gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(ROOT, "paper_2003_12861_gb300", "csrc"), SRC, "-o", exe]
    subprocess.run(cmd, check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.splitlines())}


def test_sin_cos_against_the_c_library(results):
    # |x| <= 60 and small arguments down to 2^-40: within one unit of 1
    assert results["sin_abs_err"] <= 2.3e-16 and results["cos_abs_err"] <= 2.3e-16
    assert results["sin_rel_err_small"] <= 4.5e-16
    assert results["sin0"] == 0.0 and results["cos0"] == 1.0


def test_quadratic_minimum(results):
    # EDM < 1e-14 on a quadratic with Hessian eigenvalues 2..7: |x - a| ~ 1e-7
    assert results["quad_status"] == 0
    assert results["quad_err"] < 1e-6
    assert results["quad_evals"] < 40


def test_rosenbrock_under_bounds(results):
    assert results["rosen_status"] == 0
    assert results["rosen_err"] < 1e-6
    assert results["rosen_evals"] < 200


def test_minimum_beyond_a_bound_ends_on_the_bound(results):
    assert results["bound_status"] == 0
    assert abs(results["bound_theta"] - 2.0) < 1e-6


def test_domain_and_evaluation_cap(results):
    assert results["domain_status"] == 4 and results["domain_evals"] == 1  # RF_E_DOMAIN
    assert results["cap_status"] == 5 and results["cap_evals"] == 7  # RF_E_NOT_CONVERGED
