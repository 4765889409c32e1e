"""Pins of the CPU oracle against facts fixed outside it: quadrature of the
shapes, the convolution integral, closed-form maximum-likelihood estimates,
30-digit brute force of the definitions, Richardson-extrapolated finite
differences, special cases of SUM/PROD and published Philox vectors.

None of these re-types the oracle's closed forms."""
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate, stats

from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node, ModelSpec

import mp_defs


def single_leaf(kind, lo, hi, params, free=True):
    nodes = [Node("obs", (), 0.0, lo, hi)]
    for v in params:
        nodes.append(Node("param", (), v, -1e9, 1e9, free))
    nodes.append(Node(kind, tuple(range(len(nodes)))))
    return ModelSpec(nodes, len(nodes) - 1)


LEAF_CASES = [
    ("gauss", 0.0, 10.0, [5.0, 0.5]),
    ("gauss", 0.0, 10.0, [9.7, 2.0]),            # truncated on one side
    ("gauss", 5.2, 5.4, [5.28, 0.015]),
    ("gauss", 0.0, 1.0, [-3.0, 0.4]),            # far tail on the left (erfc branch)
    ("gauss", 0.0, 1.0, [4.0, 0.6]),             # far tail on the right
    ("exp", 0.0, 10.0, [-0.7]),
    ("exp", 0.0, 10.0, [0.0]),
    ("exp", 0.0, 10.0, [1e-5]),                  # series branch of the mean
    ("exp", -1.0, 2.0, [3.0]),
    ("gaussexp", 0.0, 10.0, [1.5, 0.0, 0.05]),
    ("gaussexp", 0.0, 10.0, [0.4, 0.3, 0.2]),
    ("gaussexp", 0.0, 10.0, [2.5, -0.4, 0.6]),
    ("gaussexp", -2.0, 3.0, [1.0, 0.5, 0.3]),
    ("cheb", 0.0, 10.0, [-0.2, 0.05]),
    ("cheb", 5.2, 5.4, [-0.3]),
    ("cheb", -1.0, 3.0, [0.1, -0.2, 0.05, 0.02]),
    ("poly", 0.0, 10.0, [-0.05]),
    ("poly", -1.0, 1.0, [0.1, 0.3]),
    ("poly", 1.0, 2.0, [0.2, -0.1, 0.03]),
]


@pytest.mark.parametrize("kind,lo,hi,params", LEAF_CASES)
def test_leaf_norm_matches_quadrature(oracle_mod, kind, lo, hi, params):
    s = single_leaf(kind, lo, hi, params)
    m = oracle_mod.Model(s.nodes, s.root)
    th = np.array(params, dtype=float)
    I, _ = m.leaf_norm(s.root, th)
    pts = [params[1]] if kind == "gaussexp" and lo < params[1] < hi else None
    if kind == "gauss" and lo < params[0] < hi:
        pts = [params[0]]
    Iq, err = integrate.quad(lambda x: m.leaf_shape(s.root, th, x), lo, hi, points=pts, epsabs=0, epsrel=1e-13,
                             limit=400)
    assert abs(I - Iq) <= 1e-11 * abs(Iq), (I, Iq)
    # and the normalised pdf integrates to one
    Pq, _ = integrate.quad(lambda x: m.pdf(th, [np.array([x])])[0], lo, hi, points=pts, epsabs=0, epsrel=1e-13,
                           limit=400)
    assert abs(Pq - 1.0) < 1e-11


@pytest.mark.parametrize("kind,lo,hi,params", LEAF_CASES)
def test_leaf_norm_derivative_matches_richardson(oracle_mod, kind, lo, hi, params):
    s = single_leaf(kind, lo, hi, params)
    m = oracle_mod.Model(s.nodes, s.root)
    th = np.array(params, dtype=float)
    _, dI = m.leaf_norm(s.root, th)
    for k in range(len(params)):
        width = params[1] if kind == "gauss" else params[2] if kind == "gaussexp" else 1.0
        h = 1e-3 * min(max(abs(th[k]), 0.1), width)  # small against the pdf's own width

        def D(h):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            return (m.leaf_norm(s.root, tp)[0] - m.leaf_norm(s.root, tm)[0]) / (2 * h)

        R = (4 * D(h / 2) - D(h)) / 3  # Richardson: cancels the h^2 term
        scale = max(abs(R), abs(m.leaf_norm(s.root, th)[0]) * 1e-3)
        assert abs(dI[k] - R) <= 1e-7 * scale, (k, dI[k], R)


@pytest.mark.parametrize("params,t", [([1.5, 0.0, 0.05], 0.01), ([1.5, 0.0, 0.05], 0.3), ([1.5, 0.0, 0.05], 4.0),
                                      ([0.4, 0.3, 0.2], 0.1), ([0.4, 0.3, 0.2], -0.5), ([2.5, -0.4, 0.6], 2.0),
                                      ([1.0, 0.5, 0.1], -0.4),   # z = 7.4: the continued-fraction branch
                                      ([1.0, 0.5, 0.05], -0.2)])  # z = 10
def test_gaussexp_shape_is_the_convolution(oracle_mod, params, t):
    s = single_leaf("gaussexp", -5.0, 10.0, params)
    m = oracle_mod.Model(s.nodes, s.root)
    got = m.leaf_shape(s.root, np.array(params), t)
    want = mp_defs.shape("gaussexp", t, [mp.mpf(p) for p in params], -5, 10)
    # In the far left tail (values ~1e-45) the 30-digit quadrature itself only
    # settles to ~5e-13; elsewhere it is good to well below 1e-13.
    tol = 1e-11 if float(want) < 1e-30 else 1e-13
    assert abs(got - float(want)) <= tol * float(want), (got, want)


def test_gaussexp_zero_resolution_limit(oracle_mod):
    # sigma -> 0: the convolution becomes the bare decay exp(-(t-mu)/tau) for t > mu.
    tau, mu = 1.3, 0.2
    s = single_leaf("gaussexp", 0.0, 10.0, [tau, mu, 1e-7])
    m = oracle_mod.Model(s.nodes, s.root)
    for t in [0.5, 1.0, 3.0, 7.0]:
        got = m.leaf_shape(s.root, np.array([tau, mu, 1e-7]), t)
        assert abs(got - math.exp(-(t - mu) / tau)) < 1e-9
    I, _ = m.leaf_norm(s.root, np.array([tau, mu, 1e-7]))
    assert abs(I - tau * (1 - math.exp(-(10 - mu) / tau))) < 1e-9


def test_worked_example_gauss_poly1(oracle_mod):
    # p(x=5) at mu=5, sigma=0.5, f=0.3, a1=-0.05 on [0,10]: the Gaussian's mass
    # outside the range is ~1e-23, so the Gauss part is 0.3/(0.5 sqrt(2 pi)) and
    # the Poly1 part is 0.7 (1 - 0.25)/(10 - 2.5) = 0.07.
    s = W.gauss_poly1_model()
    m = oracle_mod.Model(s.nodes, s.root)
    p = m.pdf(W.GAUSS_POLY1_TRUE, [np.array([5.0])])[0]
    assert abs(p - (0.3 / (0.5 * math.sqrt(2 * math.pi)) + 0.07)) < 1e-15
    # Chebychev2 normalisation of the decay model's background: 10 - 5 * 0.05 * 2/3
    d = W.decay_model()
    md = oracle_mod.Model(d.nodes, d.root)
    cheb = [i for i, n in enumerate(d.nodes) if n.kind == "cheb"][0]
    assert abs(md.leaf_norm(cheb, W.DECAY_TRUE)[0] - (10 - 5 * 0.05 * 2 / 3)) < 1e-13


def _events(model_spec, theta, n, seed, oracle_mod):
    m = oracle_mod.Model(model_spec.nodes, model_spec.root)
    return m, m.generate(theta, seed, 0, 0, n)


@pytest.mark.parametrize("which", ["gauss_poly1_model", "decay_model", "prod3_model"])
def test_nll_brute_force_mpmath(oracle_mod, which):
    spec = W.model_for(which)
    theta = {"gauss_poly1_model": W.GAUSS_POLY1_TRUE, "decay_model": W.DECAY_TRUE,
             "prod3_model": W.PROD3_TRUE}[which]
    m, cols = _events(spec, theta, 6, 99, oracle_mod)
    # move one parameter off its generating value so nothing is special
    theta = theta * (1 + 0.03 * np.cos(np.arange(len(theta))))
    nll, g, al, ag, rc = m.nll(theta, cols)
    assert rc == 0
    evs = list(zip(*[c.tolist() for c in cols]))
    want = mp_defs.nll(spec.nodes, spec.root, [mp.mpf(t) for t in theta], evs)
    assert abs(nll - float(want)) <= 1e-13 * al, (nll, want)
    # gradient: 30-digit central difference of the brute-force definition
    if which != "prod3_model":
        for k in range(len(theta)):
            h = mp.mpf("1e-8") * max(abs(theta[k]), 0.1)

            def F(v):
                tt = [mp.mpf(t) for t in theta]
                tt[k] = v
                return mp_defs.nll(spec.nodes, spec.root, tt, evs)

            gk = (F(mp.mpf(theta[k]) + h) - F(mp.mpf(theta[k]) - h)) / (2 * h)
            assert abs(g[k] - float(gk)) <= 1e-9 * max(ag[k], 1e-300), (k, g[k], gk)


@pytest.mark.parametrize("which", ["gauss_poly1_model", "decay_model", "prod3_model"])
def test_gradient_richardson(oracle_mod, which):
    spec = W.model_for(which)
    theta = {"gauss_poly1_model": W.GAUSS_POLY1_TRUE, "decay_model": W.DECAY_TRUE,
             "prod3_model": W.PROD3_TRUE}[which]
    m, cols = _events(spec, theta, 2000, 7, oracle_mod)
    th = theta * (1 + 0.02 * np.sin(np.arange(len(theta)) + 1))
    _, g, _, ag, rc = m.nll(th, cols)
    assert rc == 0
    for k in range(len(th)):
        h = 1e-4 * max(abs(th[k]), 0.01)

        def D(h):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            return (m.nll(tp, cols)[0] - m.nll(tm, cols)[0]) / (2 * h)

        R = (4 * D(h / 2) - D(h)) / 3
        assert abs(g[k] - R) <= 1e-7 * ag[k], (k, g[k], R)


def test_gaussian_mle_closed_form(oracle_mod):
    # Gaussian on a range of +-40 sigma: the MLE is the sample mean and the
    # 1/N sample standard deviation; the gradient there vanishes and the
    # covariance is diag(s^2/N, s^2/(2N)).
    nodes = [Node("obs", (), 0, -40.0, 40.0), Node("param", (), 0.3, -5, 5, True),
             Node("param", (), 1.4, 0.1, 5, True), Node("gauss", (0, 1, 2))]
    m = oracle_mod.Model(nodes, 3)
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.normal(0.1, 1.1, 5000)
    mean, sd = x.mean(), x.std()
    nll, g, al, ag, rc = m.nll([mean, sd], [x])
    assert abs(g[0]) < 1e-12 * ag[0] * 10 and abs(g[1]) < 1e-12 * ag[1] * 10
    r = m.fit([x])
    assert r["status"] == 0
    N = len(x)
    assert abs(r["theta"][0] - mean) < 1e-4 * sd / math.sqrt(N)
    assert abs(r["theta"][1] - sd) < 1e-4 * sd / math.sqrt(2 * N)
    assert abs(r["cov"][0, 0] / (sd * sd / N) - 1) < 1e-4
    assert abs(r["cov"][1, 1] / (sd * sd / (2 * N)) - 1) < 1e-4


def test_exponential_mle_closed_form(oracle_mod):
    # exp(c x) on [0, 2000]: the truncation is exp(-2000 |c|) ~ 0, so the MLE is c = -1/mean.
    nodes = [Node("obs", (), 0, 0.0, 2000.0), Node("param", (), -0.5, -10, -0.01, True), Node("exp", (0, 1))]
    m = oracle_mod.Model(nodes, 2)
    x = np.random.Generator(np.random.PCG64(11)).exponential(0.8, 4000)
    chat = -1.0 / x.mean()
    _, g, _, ag, _ = m.nll([chat], [x])
    assert abs(g[0]) < 1e-12 * ag[0] * 10
    r = m.fit([x])
    assert r["status"] == 0 and abs(r["theta"][0] - chat) < 1e-4 * abs(chat) / math.sqrt(len(x))


def test_fraction_only_fit_matches_bounded_scalar_minimiser(oracle_mod):
    from scipy.optimize import minimize_scalar

    spec = W.gauss_poly1_model()
    m0, cols = _events(spec, W.GAUSS_POLY1_TRUE, 3000, 3, oracle_mod)
    nodes = [Node(n.kind, n.inputs, n.value, n.lo, n.hi, n.free) for n in spec.nodes]
    fixed = dict(zip(["mu", "sigma", "a1"], [5.0, 0.5, -0.05]))
    idx = {n: i for i, n in enumerate(["x", "mu", "sigma", "f", "a1"])}
    for name, v in fixed.items():
        o = nodes[idx[name]]
        nodes[idx[name]] = Node("param", (), v, o.lo, o.hi, False)
    m = oracle_mod.Model(nodes, spec.root)
    r = m.fit(cols)
    res = minimize_scalar(lambda f: m.nll([f], cols)[0], bounds=(0.0, 1.0), method="bounded",
                          options={"xatol": 1e-10})
    assert abs(r["theta"][0] - res.x) < 1e-6


def test_sum_prod_special_cases(oracle_mod):
    x = np.linspace(0.05, 9.95, 50)
    # SUM with f = 1 equals its first component
    nodes = [Node("obs", (), 0, 0, 10), Node("param", (), 4.0, 0, 10, True), Node("param", (), 1.2, 0.1, 5, True),
             Node("gauss", (0, 1, 2)), Node("param", (), 0.1, -1, 1, True), Node("cheb", (0, 4)),
             Node("param", (), 1.0, 0, 1, False), Node("sum", (3, 5, 6)), Node("prod", (3,))]
    m = oracle_mod.Model(nodes, 7)
    th = np.array([4.0, 1.2, 0.1])
    assert np.allclose(m.pdf(th, [x], node=7), m.pdf(th, [x], node=3), rtol=1e-15, atol=0)
    # PROD with one factor equals that factor
    m8 = oracle_mod.Model(nodes, 8)
    assert np.array_equal(m8.pdf(th, [x]), m8.pdf(th, [x], node=3))


def test_invalid_models_rejected(oracle_mod):
    base = [Node("obs", (), 0, 0, 10), Node("param", (), 4.0, 0, 10, True), Node("param", (), 1.2, 0.1, 5, True),
            Node("gauss", (0, 1, 2))]
    with pytest.raises(ValueError):  # PROD of two factors in the same observable
        oracle_mod.Model(base + [Node("prod", (3, 3))], 4)
    with pytest.raises(ValueError):  # SUM components over different observables
        nodes = base + [Node("obs", (), 0, 0, 1), Node("poly", (4,)), Node("param", (), 0.5, 0, 1, True),
                        Node("sum", (3, 5, 6))]
        oracle_mod.Model(nodes, 7)
    with pytest.raises(ValueError):  # leaf with a pdf where a parameter belongs
        oracle_mod.Model(base + [Node("gauss", (0, 3, 2))], 4)


def _philox_kat():
    """Known-answer vectors from tests/golden/philox4x32_10_kat.txt (cited there)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(w, 16) for w in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


PHILOX_KAT = _philox_kat()


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answers(oracle_mod, ctr, key, out):
    assert oracle_mod.philox4x32_10(ctr, key) == out


@pytest.mark.parametrize("mu", [3.0, 25.0, 1000.0, 60000.0])
def test_poisson_moments(oracle_mod, mu):
    n = 20000
    k = np.array([oracle_mod.poisson(123, s, mu) for s in range(n)], dtype=float)
    assert abs(k.mean() - mu) < 5 * math.sqrt(mu / n)
    # variance of the sample variance of a Poisson ~ (mu + 2 mu^2)/n
    assert abs(k.var() - mu) < 5 * math.sqrt((mu + 2 * mu * mu) / n)
    if mu == 25.0:
        vals, cnt = np.unique(k, return_counts=True)
        lo, hi = 12, 40
        obs = np.array([cnt[vals < lo].sum()] + [cnt[vals == v].sum() for v in range(lo, hi)] + [cnt[vals >= hi].sum()])
        pmf = np.array([stats.poisson.cdf(lo - 1, mu)] + [stats.poisson.pmf(v, mu) for v in range(lo, hi)]
                       + [stats.poisson.sf(hi - 1, mu)])
        chi2 = ((obs - n * pmf) ** 2 / (n * pmf)).sum()
        assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4


@pytest.mark.parametrize("which", ["gauss_poly1_model", "decay_model"])
def test_generator_matches_pdf_histogram(oracle_mod, which):
    spec = W.model_for(which)
    theta = W.GAUSS_POLY1_TRUE if which == "gauss_poly1_model" else W.DECAY_TRUE
    m, cols = _events(spec, theta, 60000, 2024, oracle_mod)
    x = cols[0]
    edges = np.linspace(0, 10, 41)
    cnt, _ = np.histogram(x, edges)
    prob = np.array([integrate.quad(lambda t: m.pdf(theta, [np.array([t])])[0], a, b, epsrel=1e-10, limit=200)[0]
                     for a, b in zip(edges[:-1], edges[1:])])
    exp_ = len(x) * prob
    chi2 = ((cnt - exp_) ** 2 / exp_).sum()
    assert stats.chi2.sf(chi2, len(cnt) - 1) > 1e-4
    assert x.min() >= 0 and x.max() < 10


def test_generator_is_counter_based(oracle_mod):
    # events [i0, i1) generated alone equal the same slice of a longer run
    spec = W.decay_model()
    m = oracle_mod.Model(spec.nodes, spec.root)
    full = m.generate(W.DECAY_TRUE, 77, 3, 0, 500)[0]
    part = m.generate(W.DECAY_TRUE, 77, 3, 200, 300)[0]
    assert np.array_equal(full[200:300], part)
    other = m.generate(W.DECAY_TRUE, 77, 4, 0, 500)[0]
    assert not np.array_equal(full, other)


def test_hist64_matches_numpy(oracle_mod):
    x = np.random.Generator(np.random.PCG64(1)).uniform(0, 10, 100000)
    h = oracle_mod.hist64(x, 0.0, 10.0)
    ref, _ = np.histogram(x, np.linspace(0, 10, 65))
    assert np.allclose(h, ref / len(x), rtol=0, atol=2e-5)
    assert abs(h.sum() - 1) < 1e-6


# ------------------------------------------- generation under a PROD root

def _factor_density(m, theta, root_inputs, f, n_obs, col):
    """Normalised density of PROD factor f in its own observable (column
    col), the other observables held at fixed in-range values."""
    def dens(x):
        cols = [np.array([0.5 * (lo + hi)]) for lo, hi in _RANGES[n_obs]]
        cols[col] = np.array([x])
        return m.pdf(theta, cols, node=f)[0]
    return dens


_RANGES = {3: [(5.2, 5.4), (0.0, 10.0), (-1.0, 1.0)], 2: [(0.0, 30.0), (-5.0, 5.0)]}


def _chi2_p(cnt, exp_):
    keep = exp_ > 0
    chi2 = ((cnt[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


@pytest.mark.parametrize("which", ["prod3_model", "poisson_gauss_model"])
def test_prod_root_generation_follows_each_factor(oracle_mod, which):
    """Events of a product model are drawn factor by factor (each factor's
    observable by accept-reject against its own bound): every column's
    histogram must follow that factor's normalised density, and the columns
    must be independent (the joint density is the product, paper Sec. 1: a
    PROD node multiplies PDFs of disjoint observables)."""
    spec = W.model_for(which)
    theta = W.PROD3_TRUE if which == "prod3_model" else W.POISSON_GAUSS_TRUE
    m, cols = _events(spec, theta, 80000, 31337, oracle_mod)
    root = spec.nodes[spec.root]
    n_obs = len(cols)
    N = len(cols[0])
    probs = []
    for col, f in enumerate(root.inputs):
        lo, hi = _RANGES[n_obs][col]
        x = cols[col]
        assert x.min() >= lo and x.max() < hi
        if spec.nodes[f].kind == "poisson":
            # a step density of unit steps: k = floor(x) follows the pmf
            # renormalised on lo .. hi-1, and x - k is uniform on [0, 1)
            k = np.arange(int(lo), int(hi))
            fr = x - np.floor(x)
            fc, _ = np.histogram(fr, np.linspace(0, 1, 21))
            assert _chi2_p(fc.astype(float), np.full(20, N / 20)) > 1e-4
            cnt = np.bincount(np.floor(x).astype(int) - int(lo), minlength=len(k))[: len(k)].astype(float)
            pmf = stats.poisson.pmf(k, theta[0])
            prob = pmf / pmf.sum()
            edges = np.concatenate([k, [hi]]).astype(float)
        else:
            dens = _factor_density(m, theta, root.inputs, f, n_obs, col)
            edges = np.linspace(lo, hi, 41)
            cnt, _ = np.histogram(x, edges)
            prob = np.array([integrate.quad(dens, a, b, epsrel=1e-10, limit=200)[0]
                             for a, b in zip(edges[:-1], edges[1:])])
        assert abs(prob.sum() - 1.0) < 1e-8
        assert _chi2_p(cnt.astype(float), N * prob) > 1e-4, (which, col)
        probs.append((edges, prob))
    # independence: each pair of columns against the product of the marginals
    for c1 in range(n_obs):
        for c2 in range(c1 + 1, n_obs):
            e1, p1 = _coarse(*probs[c1])
            e2, p2 = _coarse(*probs[c2])
            joint, _, _ = np.histogram2d(cols[c1], cols[c2], [e1, e2])
            assert _chi2_p(joint.ravel(), N * np.outer(p1, p2).ravel()) > 1e-4, (which, c1, c2)


def _coarse(edges, prob, n=8):
    """Merge adjacent bins into about n groups of similar probability."""
    cum = np.concatenate([[0.0], np.cumsum(prob)])
    cut = sorted({int(np.searchsorted(cum, q)) for q in np.linspace(0, 1, n + 1)[1:-1]} - {0, len(prob)})
    idx = [0] + cut + [len(prob)]
    return edges[idx], np.array([prob[a:b].sum() for a, b in zip(idx[:-1], idx[1:])])


def test_prod_generation_detects_a_planted_dependence(oracle_mod):
    """The independence check above has power: pairing each mass value with
    a decay time sorted by the mass (a perfect rank correlation, both
    marginals unchanged) fails it."""
    spec = W.prod3_model()
    m, cols = _events(spec, W.PROD3_TRUE, 80000, 31337, oracle_mod)
    order = np.argsort(cols[0])
    t_sorted = np.sort(cols[1])
    planted = [cols[0][order], t_sorted, cols[2]]
    e1 = np.quantile(planted[0], np.linspace(0, 1, 9))
    e2 = np.quantile(planted[1], np.linspace(0, 1, 9))
    joint, _, _ = np.histogram2d(planted[0], planted[1], [e1, e2])
    p = np.full(8, 1 / 8)
    assert _chi2_p(joint.ravel(), len(planted[0]) * np.outer(p, p).ravel()) < 1e-10
