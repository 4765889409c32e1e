"""Pins of the oracle's EXPR leaf: a density given as a postfix program over
the observable and the node's parameters, normalised by the oracle's own
adaptive Gauss-Legendre quadrature (the paper's Sec. 5 fall-back evaluation
for PDFs that have no specialised batch code).  Each pin fixes the program
evaluation, its parameter derivatives and the quadrature by something other
than the oracle itself: the built-in Gaussian's analytic normalisation,
closed-form integrals, 30-digit brute force, finite differences."""
import mpmath as mp
import numpy as np
import pytest
from scipy import integrate, stats

from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node, expr_program

import mp_defs


@pytest.mark.parametrize("theta", [W.GAUSS_POLY1_TRUE, np.array([4.2, 1.3, 0.6, 0.02]),
                                   np.array([0.3, 0.05, 0.8, -0.05]), np.array([9.7, 2.5, 0.2, 0.3])])
def test_expr_gaussian_equals_the_builtin_gaussian(oracle_mod, theta):
    """exp(-((x - mu)/sigma)^2/2) as a program gives the built-in GAUSS node's
    likelihood and gradient: the program's values and derivatives, and the
    quadrature against the analytic erf normalisation, including a peak
    near the range's edge and a narrow one (sigma = 0.05 on [0, 10])."""
    ref = W.gauss_poly1_model()
    ex = W.expr_gauss_poly1_model()
    mr = oracle_mod.Model(ref.nodes, ref.root)
    me = oracle_mod.Model(ex.nodes, ex.root)
    cols = mr.generate(theta, 11, 0, 0, 3000)
    a = mr.nll(theta, cols)
    b = me.nll(theta, cols)
    assert a[4] == 0 and b[4] == 0
    assert abs(a[0] - b[0]) <= 1e-13 * a[2], (a[0], b[0])
    assert np.all(np.abs(a[1] - b[1]) <= 1e-11 * a[3]), (a[1], b[1])
    I_ref, dI_ref = mr.leaf_norm(5, theta)
    I_ex, dI_ex = me.leaf_norm(5, theta)
    assert abs(I_ex - I_ref) <= 1e-14 * I_ref
    assert np.allclose(dI_ex, dI_ref, rtol=1e-12, atol=1e-14 * I_ref)


def _power_model(lo, hi):
    # x^a on [lo, hi], a free: I(a) = (hi^(a+1) - lo^(a+1)) / (a + 1)
    nodes = [Node("obs", (), 0.0, lo, hi), Node("param", (), 0.7, -0.99, 5.0, True),
             Node("expr", (0, 1), prog=expr_program("x p0 pow"))]
    return nodes, 2


@pytest.mark.parametrize("a", [-0.5, 0.0, 0.7, 2.3])
def test_expr_normalisation_closed_form(oracle_mod, a):
    nodes, root = _power_model(1.0, 2.0)
    m = oracle_mod.Model(nodes, root)
    I, dI = m.leaf_norm(2, np.array([a]))
    A = mp.mpf(a)
    want = (2 ** (A + 1) - 1) / (A + 1)
    dwant = (2 ** (A + 1) * mp.log(2) * (A + 1) - (2 ** (A + 1) - 1)) / (A + 1) ** 2
    assert abs(I - float(want)) <= 1e-14 * float(want)
    assert abs(dI[0] - float(dwant)) <= 1e-13 * abs(float(dwant)) + 1e-15


def test_expr_mix_nll_brute_force_mpmath(oracle_mod):
    """The mixed model (Cauchy line and gamma-like density as programs beside
    a Chebychev and a SUM/PROD) at 30 digits on a few events: NLL by the
    definitions, gradient by 30-digit central differences of the definition."""
    spec = W.expr_mix_model()
    m = oracle_mod.Model(spec.nodes, spec.root)
    cols = m.generate(W.EXPR_MIX_TRUE, 99, 0, 0, 6)
    theta = W.EXPR_MIX_TRUE * (1 + 0.04 * np.cos(np.arange(6)))
    nll, g, al, ag, rc = m.nll(theta, cols)
    assert rc == 0
    evs = list(zip(*[c.tolist() for c in cols]))
    th = [mp.mpf(t) for t in theta]
    want = mp_defs.nll(spec.nodes, spec.root, th, evs)
    assert abs(nll - float(want)) <= 1e-13 * al, (nll, want)
    for k in range(6):
        h = mp.mpf(10) ** -12 * max(abs(th[k]), 1)
        tp = list(th); tp[k] += h
        tm = list(th); tm[k] -= h
        d = (mp_defs.nll(spec.nodes, spec.root, tp, evs) - mp_defs.nll(spec.nodes, spec.root, tm, evs)) / (2 * h)
        assert abs(g[k] - float(d)) <= 1e-9 * ag[k] + 1e-10, (k, g[k], d)


def test_expr_mix_generation_follows_each_factor(oracle_mod):
    spec = W.expr_mix_model()
    m = oracle_mod.Model(spec.nodes, spec.root)
    th = W.EXPR_MIX_TRUE
    cols = m.generate(th, 123, 0, 0, 40000)
    root = spec.nodes[spec.root]
    for col, (f, (lo, hi)) in enumerate(zip(root.inputs, [(5.2, 5.4), (0.2, 5.0)])):
        def dens(x, f=f, col=col):
            c = [np.array([5.3]), np.array([1.0])]
            c[col] = np.array([x])
            return m.pdf(th, c, node=f)[0]
        edges = np.linspace(lo, hi, 31)
        cnt, _ = np.histogram(cols[col], edges)
        prob = np.array([integrate.quad(dens, a, b, epsrel=1e-10, limit=200)[0] for a, b in zip(edges[:-1], edges[1:])])
        assert abs(prob.sum() - 1) < 1e-9
        chi2 = ((cnt - len(cols[col]) * prob) ** 2 / (len(cols[col]) * prob)).sum()
        assert stats.chi2.sf(chi2, 29) > 1e-4, col


@pytest.mark.parametrize("text,consts,n_par", [
    ("x +", (), 0),                 # stack underflow
    ("x x", (), 0),                 # two values left
    ("p1", (), 1),                  # parameter index out of range
    ("c0", (), 0),                  # constant index out of range
    (" ".join(["x"] * 17) + " +" * 16, (), 0),  # deeper than 16
    (" ".join(["x exp"] * 33), (), 0),          # longer than 64 (and two values)
])
def test_expr_invalid_programs_are_rejected(oracle_mod, text, consts, n_par):
    nodes = [Node("obs", (), 0.0, 0.0, 1.0)] + [Node("param", (), 0.5, 0.0, 1.0, True)] * n_par
    nodes.append(Node("expr", tuple(range(n_par + 1)), prog=expr_program(text), consts=consts))
    with pytest.raises(ValueError):
        oracle_mod.Model(nodes, len(nodes) - 1)


def test_expr_domain(oracle_mod):
    # log(x - 0.5) on [0, 1] is undefined below 0.5: no normalisation
    nodes = [Node("obs", (), 0.0, 0.0, 1.0), Node("expr", (0,), prog=expr_program("x c0 - log"), consts=(0.5,))]
    m = oracle_mod.Model(nodes, 1)
    _, _, _, _, rc = m.nll(np.zeros(0), [np.array([0.7])])
    assert rc == -2
    # a positive program with an event where it is 0: that event's pdf is 0
    nodes = [Node("obs", (), 0.0, 0.0, 1.0), Node("expr", (0,), prog=expr_program("x x *"))]
    m = oracle_mod.Model(nodes, 1)
    nll, _, _, _, rc = m.nll(np.zeros(0), [np.array([0.0, 0.5])])
    assert rc == -3 and nll == np.inf
