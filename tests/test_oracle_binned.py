"""Pins of the binned (HistFactory-style) oracle: the nominal point, the
interpolation definitions at alpha = +-1, scipy's Poisson log-pmf, the
closed-form MLE of a single normalisation factor, and the analytic gradient
against Richardson-extrapolated central differences."""
import math

import numpy as np
import pytest
from scipy import special, stats

from oracle import binned as B
from paper_2003_12861_gb300 import workloads as W


def small_model():
    h0 = np.array([5.0, 8.0, 3.0, 1.5])
    h1 = np.array([20.0, 15.0, 10.0, 7.0, 4.0, 2.0])
    mods = [B.Modifier(0, B.NORMFACTOR, 0),
            B.Modifier(0, B.NORMSYS, 1, 0.9, 1.12),
            B.Modifier(1, B.NORMSYS, 1, 0.95, 1.03),
            B.Modifier(1, B.HISTOSYS, 2, h_lo=h1 * 0.97, h_hi=h1 * np.linspace(1.01, 1.08, 6)),
            B.Modifier(0, B.HISTOSYS, 2, h_lo=h0 * 1.02, h_hi=h0 * 0.96)]
    return B.BinnedModel(6, [2, 0], [h0, h1], [False, True, True], mods)


def test_nominal_point_is_the_sum_of_histograms():
    m = small_model()
    nu, _ = m.expected([1.0, 0.0, 0.0])
    want = np.zeros(6)
    want[2:6] += m.nominal[0]
    want[0:6] += m.nominal[1]
    assert np.array_equal(nu, want)


@pytest.mark.parametrize("alpha", [1.0, -1.0])
def test_interpolation_reaches_the_variations_at_one_sigma(alpha):
    h = np.array([10.0, 20.0])
    lo, hi = h * 0.8, h * 1.3
    m = B.BinnedModel(2, [0], [h], [True, True], [B.Modifier(0, B.HISTOSYS, 0, h_lo=lo, h_hi=hi),
                                                   B.Modifier(0, B.NORMSYS, 1, 0.9, 1.2)])
    nu, _ = m.expected([alpha, 0.0])
    assert np.allclose(nu, hi if alpha > 0 else lo, rtol=1e-15)
    nu, _ = m.expected([0.0, alpha])
    assert np.allclose(nu, h * (1.2 if alpha > 0 else 0.9), rtol=1e-15)


def test_nll_is_minus_poisson_log_pmf():
    m = small_model()
    rng = np.random.Generator(np.random.PCG64(3))
    th = np.array([1.3, 0.4, -0.7])
    nu, _ = m.expected(th)
    n = rng.poisson(nu).astype(float)
    nll, g, scale = m.nll(th, n)
    want = -np.sum(stats.poisson.logpmf(n, nu)) - np.sum(special.gammaln(n + 1)) + 0.5 * (0.4 ** 2 + 0.7 ** 2)
    assert abs(nll - want) < 1e-12 * scale


def test_single_normfactor_mle_closed_form():
    h = np.array([3.0, 7.0, 11.0, 2.0])
    m = B.BinnedModel(4, [0], [h], [False], [B.Modifier(0, B.NORMFACTOR, 0)])
    n = np.array([5.0, 6.0, 15.0, 1.0])
    mu = n.sum() / h.sum()
    _, g, _ = m.nll([mu], n)
    assert abs(g[0]) < 1e-12 * n.sum()


@pytest.mark.parametrize("th", [[1.3, 0.4, -0.7], [0.6, -1.2, 0.9], [1.0, 0.0, 0.0]])
def test_gradient_richardson(th):
    m = small_model()
    n = np.array([22.0, 17.0, 19.0, 18.0, 9.0, 4.0])
    th = np.array(th)
    _, g, _ = m.nll(th, n)
    for k in range(3):
        def f(d):
            t = th.copy()
            t[k] += d
            return m.nll(t, n)[0]
        h = 1e-3
        c1 = (f(h) - f(-h)) / (2 * h)
        c2 = (f(h / 2) - f(-h / 2)) / h
        num = (4 * c2 - c1) / 3
        # g'' jumps at |alpha| = 1, where the extrapolation has a kink of
        # size O(h) in the second derivative only
        assert abs(num - g[k]) < 1e-6 * max(1.0, abs(g[k]))


@pytest.mark.parametrize("alpha", [-1.0, 0.0, 1.0])
def test_interpolation_is_continuously_differentiable(alpha):
    # value and first derivative agree from both sides at 0 and +-1
    h0, lo, hi = np.array([10.0]), np.array([7.0]), np.array([14.5])
    m = B.BinnedModel(1, [0], [h0], [True, True], [B.Modifier(0, B.HISTOSYS, 0, h_lo=lo, h_hi=hi),
                                                   B.Modifier(0, B.NORMSYS, 1, 0.8, 1.3)])
    for k in range(2):
        def nu(a):
            t = np.zeros(2)
            t[k] = a
            return m.expected(t)[0][0]
        e = 1e-7
        left = (nu(alpha) - nu(alpha - e)) / e
        right = (nu(alpha + e) - nu(alpha)) / e
        assert abs(left - right) < 1e-5 * max(1.0, abs(left))
        assert abs(nu(alpha + e) - nu(alpha - e)) < 1e-5


def test_nominal_and_extrapolation():
    h0, lo, hi = np.array([10.0, 4.0]), np.array([7.0, 5.0]), np.array([14.5, 3.0])
    m = B.BinnedModel(2, [0], [h0], [True, True], [B.Modifier(0, B.HISTOSYS, 0, h_lo=lo, h_hi=hi),
                                                   B.Modifier(0, B.NORMSYS, 1, 0.8, 1.3)])
    assert np.array_equal(m.expected([0.0, 0.0])[0], h0)
    # linear beyond +-1 sigma: at alpha = 2 the histosys gives h + 3 (h_hi - h) - (h_hi - h_lo) ... i.e.
    # delta(2) = a 2 + b 3 with a, b from the +-1 sigma points
    a, b = 0.5 * (hi - lo), 0.5 * (hi + lo) - h0
    assert np.allclose(m.expected([2.0, 0.0])[0], h0 + 2 * a + 3 * b, rtol=1e-15)
    # exponential beyond +-1 in log: eta(-2) = exp(-2 a + 3 b)
    an, bn = 0.5 * (np.log(1.3) - np.log(0.8)), 0.5 * (np.log(1.3) + np.log(0.8))
    assert np.allclose(m.expected([0.0, -2.0])[0], h0 * np.exp(-2 * an + 3 * bn), rtol=1e-15)


def test_nonpositive_expectation_is_infinite():
    h = np.array([1.0, 2.0])
    m = B.BinnedModel(2, [0], [h], [False], [B.Modifier(0, B.NORMFACTOR, 0)])
    assert math.isinf(m.nll([-1.0], [1.0, 1.0])[0])


def test_workload_shape():
    spec = W.binned_model()
    m = B.from_spec(spec)
    assert m.n_bins == 28 * 50 and m.n_params == 256 and len(m.nominal) == 28 * 8
    hists = len(m.nominal) + 2 * sum(1 for md in m.modifiers if md.kind == B.HISTOSYS)
    assert 9000 < hists < 12000  # the paper's example model has 10 832 histograms
    nu, _ = m.expected(np.concatenate([[1, 1, 1], np.zeros(253)]))
    assert np.all(nu > 0)
