"""RF_EXPR on the GPU (the fall-back evaluation for PDFs without
specialised code, paper Sec. 5): the FP64 interpreter's per-event program
and its forward-mode derivatives, the block-cooperative Gauss-Kronrod
normalisation, and everything around them (generation, fits) against the
oracle's own program interpreter and adaptive Gauss-Legendre quadrature, at
the NLL and gradient tolerances of the other parity tests."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import _lib as L
from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node, expr_program

from helpers import check_nll

pytestmark = pytest.mark.gpu

CASES = [("expr_gauss_poly1_model", W.GAUSS_POLY1_TRUE), ("expr_mix_model", W.EXPR_MIX_TRUE)]


@pytest.mark.parametrize("which,true", CASES)
@pytest.mark.parametrize("n", [1, 4095, 3 * 4096 + 1001])
def test_expr_nll_grad_matches_oracle(oracle_mod, which, true, n):
    spec = W.model_for(which)
    om = oracle_mod.Model(spec.nodes, spec.root)
    gen = oracle_mod.Model(W.gauss_poly1_model().nodes, W.gauss_poly1_model().root) if which.startswith("expr_g") else om
    cols = gen.generate(true, 321, 0, 0, n)
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols)
    for th in [true, true * (1 + 0.05 * np.sin(np.arange(len(true)) + 1.0))]:
        nll, g = api.nll_grad(m, d, th)
        check_nll(nll, g, om.nll(th, cols), f"{which} n={n}")


def test_expr_gaussian_matches_the_builtin_on_the_gpu():
    """The same events through the built-in Gaussian (float-float program,
    analytic normalisation) and through the program (FP64 interpreter,
    numerical normalisation)."""
    import oracle

    g = W.gauss_poly1_model()
    cols = oracle.Model(g.nodes, g.root).generate(W.GAUSS_POLY1_TRUE, 5, 0, 0, 50_000)
    a = api.Model.from_spec(g)
    b = api.Model.from_spec(W.expr_gauss_poly1_model())
    da, db = api.Data.upload(a, cols), api.Data.upload(b, cols)
    for th in [W.GAUSS_POLY1_TRUE, np.array([0.4, 0.07, 0.7, 0.01])]:
        na, ga = api.nll_grad(a, da, th)
        nb, gb = api.nll_grad(b, db, th)
        assert abs(na - nb) <= 1e-12 * abs(na), (na, nb)
        assert np.allclose(ga, gb, rtol=1e-9, atol=1e-9 * np.abs(ga).max())


def test_expr_batched_sets_and_generation(oracle_mod):
    """Ragged toys of the mixed model generated on the device, bitwise the
    oracle's draws (the same counter-based definition), then every set's NLL
    and gradient against the oracle."""
    spec = W.expr_mix_model()
    om = oracle_mod.Model(spec.nodes, spec.root)
    m = api.Model.from_spec(spec)
    S = 24
    mean = W.toy_mean_sizes(S, 17, 50.0, 3e4)
    d = api.generate_toys(m, W.EXPR_MIX_TRUE, 777, mean, poisson=True)
    off = d.offsets()
    th = np.tile(W.EXPR_MIX_TRUE * (1 + 0.02 * np.cos(np.arange(6))), (S, 1))
    nll, g = api.nll_grad(m, d, th)
    bounds = om.gen_bounds(W.EXPR_MIX_TRUE)
    for s in range(S):
        n = int(off[s + 1] - off[s])
        assert n == oracle_mod.poisson(777, s, mean[s])
        cols = om.generate(W.EXPR_MIX_TRUE, 777, s, 0, n, bounds=bounds)
        for c in range(2):
            assert np.array_equal(d.read(c, off[s], off[s + 1]), cols[c]), (s, c)
        check_nll(nll[s], g[s], om.nll(th[s], cols), f"set {s}")


def test_expr_fit_matches_oracle_fit(oracle_mod):
    spec = W.expr_mix_model()
    om = oracle_mod.Model(spec.nodes, spec.root)
    cols = om.generate(W.EXPR_MIX_TRUE, 4242, 0, 0, 60_000)
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols)
    start = W.EXPR_MIX_TRUE * np.array([1.001, 1.3, 0.8, 1.2, 0.8, 1.25])
    r = api.fit(m, d, theta0=start, tol_edm=1e-10)
    o = om.fit(cols, theta0=start, tol_edm=1e-10)
    assert r["status"][0] == L.RF_OK and o["status"] == 0
    sig = np.sqrt(np.diag(o["cov"]))
    assert np.all(np.abs(r["theta"][0] - o["theta"]) <= 1e-3 * sig), (r["theta"][0], o["theta"], sig)
    assert abs(r["nll"][0] - o["nll"]) <= 1e-7 * abs(o["nll"])


def test_expr_domain_on_the_device():
    # log(x - p0) on [0, 1] with p0 = 0.5 is undefined below 0.5: the
    # normalisation leaves the program's domain, so the point is outside
    # the model's domain and the NLL is +inf (RF_E_DOMAIN)
    nodes = [Node("obs", (), 0.0, 0.0, 1.0), Node("param", (), 0.5, -1.0, 1.0, True),
             Node("expr", (0, 1), prog=expr_program("x p0 - log"))]
    m = api.Model(nodes, 2)
    d = api.Data.upload(m, [np.array([0.7, 0.9])])
    nll, _ = api.nll_grad(m, d, np.array([0.5]), allow_domain=True)
    assert nll == np.inf
    # with p0 = -1 the program is positive on the range: a finite NLL
    nll, _ = api.nll_grad(m, d, np.array([-1.0]))
    assert np.isfinite(nll)
