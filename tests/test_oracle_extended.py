"""Oracle pins of the Poisson leaf and the extended likelihood (the next rows
after the decay workloads): closed forms of the regularised incomplete gamma
function, scipy's Poisson pmf, the identity dP(N <= n)/dlambda = -pmf(n),
brute-force normalisation, and the closed-form extended MLE nu = N."""
import math

import numpy as np
import pytest
from scipy import special, stats

from paper_2003_12861_gb300.workloads import Node


def poisson_leaf(a, b, lam, free=True, lo=1e-3, hi=1e3):
    return [Node("obs", (), 0.0, a, b), Node("param", (), lam, lo, hi, free), Node("poisson", (0, 1))]


@pytest.mark.parametrize("a,b,lam", [(0, 20, 3.0), (0, 60, 17.5), (2, 9, 4.2), (5, 400, 123.0), (0, 3, 0.2)])
def test_poisson_norm_is_the_incomplete_gamma_mass(oracle_mod, a, b, lam):
    m = oracle_mod.Model(poisson_leaf(a, b, lam), 2)
    I, dI = m.leaf_norm(2, [lam])
    # sum_{k=a}^{b-1} pmf(k) = P(N <= b-1) - P(N <= a-1), P(N <= n) = Q(n+1, lambda)
    want = special.gammaincc(b, lam) - (special.gammaincc(a, lam) if a > 0 else 0.0)
    # each term is exp(k log lambda - lambda - log k!): the exponent's rounding
    # error is a few ulp of its largest part
    tol = 4 * np.finfo(float).eps * (b * abs(math.log(lam)) + lam + math.lgamma(b + 1))
    assert abs(I - want) <= tol * max(want, 1e-300) + 1e-16
    # d/dlambda P(N <= n) = -pmf(n)
    dwant = -stats.poisson.pmf(b - 1, lam) + (stats.poisson.pmf(a - 1, lam) if a > 0 else 0.0)
    assert abs(dI[0] - dwant) <= 1e-12 * max(abs(dwant), stats.poisson.pmf(round(lam), lam))


def test_poisson_shape_is_the_pmf_of_the_floor(oracle_mod):
    a, b, lam = 0, 30, 6.5
    m = oracle_mod.Model(poisson_leaf(a, b, lam), 2)
    for x in [0.0, 0.3, 1.0, 5.999, 6.0, 17.2, 29.0, 29.9999, 30.0]:
        k = min(math.floor(x), b - 1)
        assert m.leaf_shape(2, [lam], x) == pytest.approx(stats.poisson.pmf(k, lam), rel=1e-13)


def test_poisson_density_integrates_to_one(oracle_mod):
    # The normalised step density over [a, b]: unit-width steps k = a..b-1.
    a, b, lam = 3, 25, 9.0
    m = oracle_mod.Model(poisson_leaf(a, b, lam), 2)
    mids = np.arange(a, b) + 0.5
    p = m.pdf([lam], [mids], node=2)
    assert abs(p.sum() - 1.0) < 1e-14


def test_poisson_gradient_and_mle(oracle_mod):
    # Full range (truncation < 1e-40): the MLE of lambda is the sample mean.
    a, b = 0, 80
    rng = np.random.Generator(np.random.PCG64(8))
    k = rng.poisson(7.3, 3000).astype(np.float64)
    m = oracle_mod.Model(poisson_leaf(a, b, 5.0, lo=0.5, hi=50.0), 2)
    lam_hat = k.mean()
    nll, g, al, ag, rc = m.nll([lam_hat], [k])
    assert rc == 0 and abs(g[0]) < 1e-11 * ag[0]
    # gradient = -(sum k / lambda - N) away from the MLE
    lam = 6.1
    nll, g, *_ = m.nll([lam], [k])
    assert abs(g[0] - (-(k.sum() / lam - len(k)))) < 1e-10 * len(k)
    # and the NLL is -sum log pmf (library routine)
    assert abs(nll + stats.poisson.logpmf(k, lam).sum()) < 1e-9 * abs(nll)
    r = m.fit([k])
    assert r["status"] == 0 and abs(r["theta"][0] - lam_hat) < 1e-4 * math.sqrt(lam_hat / len(k))


def extended_gauss(nu0=500.0):
    return [Node("obs", (), 0.0, -30.0, 30.0), Node("param", (), 0.2, -5, 5, True),
            Node("param", (), 1.3, 0.1, 5, True), Node("gauss", (0, 1, 2)),
            Node("param", (), nu0, 1.0, 1e7, True), Node("extend", (3, 4))]


def test_extended_term_and_closed_form_mle(oracle_mod):
    spec = extended_gauss()
    m = oracle_mod.Model(spec, 5)
    plain = oracle_mod.Model(spec[:4], 3)
    x = np.random.Generator(np.random.PCG64(4)).normal(0.3, 1.1, 777)
    th = [0.3, 1.1, 640.0]
    nll, g, al, ag, rc = m.nll(th, [x])
    nll0, g0, *_ = plain.nll(th[:2], [x])
    N = len(x)
    # NLL_ext = NLL + nu - N log nu; d/dnu = 1 - N/nu; the others unchanged
    assert abs(nll - (nll0 + 640.0 - N * math.log(640.0))) <= 1e-12 * al
    assert g[2] == pytest.approx(1.0 - N / 640.0, rel=1e-15)
    assert np.allclose(g[:2], g0, rtol=0, atol=1e-12 * max(abs(g0).max(), 1))
    # the extended MLE of nu is N exactly; mu, sigma as without extension
    r = m.fit([x])
    assert r["status"] == 0 and abs(r["theta"][2] - N) < 1e-4 * math.sqrt(N)
    assert abs(r["theta"][0] - x.mean()) < 1e-4 * x.std() / math.sqrt(N)
    # and its variance is N (inverse Hessian of nu - N log nu at nu = N)
    assert abs(r["cov"][2, 2] / N - 1) < 1e-3


def test_extended_domain_and_placement(oracle_mod):
    spec = extended_gauss()
    m = oracle_mod.Model(spec, 5)
    x = np.zeros(10)
    nll, g, al, ag, rc = m.nll([0.0, 1.0, -3.0], [x])
    assert rc == -2 and math.isinf(nll)
    # EXTEND only as the root
    bad = spec + [Node("prod", (5,))]
    with pytest.raises(ValueError):
        oracle_mod.Model(bad, 6)
    with pytest.raises(ValueError):
        oracle_mod.Model(poisson_leaf(0.5, 10, 2.0), 2)   # non-integer Poisson range


def test_poisson_generation_follows_the_pmf(oracle_mod):
    a, b, lam = 0, 25, 6.0
    m = oracle_mod.Model(poisson_leaf(a, b, lam), 2)
    x = m.generate([lam], 123, 0, 0, 20000)[0]
    k = np.floor(x).astype(int)
    assert k.min() >= a and k.max() <= b - 1
    obs = np.bincount(k, minlength=b)[a:b]
    pmf = stats.poisson.pmf(np.arange(a, b), lam)
    exp = 20000 * pmf / pmf.sum()
    keep = exp > 5
    chi2 = (((obs - exp) ** 2) / exp)[keep].sum()
    assert chi2 < stats.chi2.ppf(0.999, keep.sum() - 1)


def test_extended_model_generates_its_pdf(oracle_mod):
    spec = extended_gauss()
    m = oracle_mod.Model(spec, 5)
    x = m.generate([0.2, 1.3, 500.0], 5, 0, 0, 5000)[0]
    assert abs(x.mean() - 0.2) < 5 * 1.3 / math.sqrt(5000) and abs(x.std() - 1.3) < 0.05
