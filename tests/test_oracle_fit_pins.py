"""Pins of the oracle's fitter on the 6-parameter decay model, where no closed
form exists: at the reported minimum the analytic gradient vanishes to its
rounding scale and the estimated distance to the minimum is below the stopping
rule; the reported covariance inverts to the Hessian taken independently, by
Richardson-extrapolated second differences of NLL values alone (no gradient
code).  As a statistical sanity check rather than parity, the pulls
(theta_hat - theta_true)/sigma of the Gauss + Poly1 model over seeded toys
have mean ~0 and width ~1."""
import math

import numpy as np

from paper_2003_12861_gb300 import workloads as W


def _decay(oracle_mod):
    s = W.decay_model()
    return oracle_mod.Model(s.nodes, s.root)


def _value_hessian(f, th, step):
    P = len(th)
    H = np.zeros((P, P))
    for i in range(P):
        for j in range(i, P):
            ei = np.zeros(P)
            ej = np.zeros(P)
            ei[i] = step[i]
            ej[j] = step[j]
            v = (f(th + ei + ej) - f(th + ei - ej) - f(th - ei + ej) + f(th - ei - ej)) / (4 * step[i] * step[j])
            H[i, j] = H[j, i] = v
    return H


def test_decay_fit_minimum_and_covariance(oracle_mod):
    m = _decay(oracle_mod)
    cols = m.generate(W.DECAY_TRUE, 99, 0, 0, 20000)
    r = m.fit(cols, tol_edm=1e-12)
    assert r["status"] == 0
    th, C = r["theta"], r["cov"]
    nll, g, al, ag, rc = m.nll(th, cols)
    assert rc == 0 and abs(nll - r["nll"]) <= 1e-12 * al
    assert np.all(np.abs(g) <= 1e-8 * ag)
    assert 0.5 * g @ C @ g < 1e-10
    sig = np.sqrt(np.diag(C))
    f = lambda x: m.nll(x, cols)[0]
    H1 = _value_hessian(f, th, 0.2 * sig)
    H2 = _value_hessian(f, th, 0.1 * sig)
    H = (4 * H2 - H1) / 3
    scale = np.sqrt(np.outer(np.diag(H), np.diag(H)))
    assert np.abs((H - np.linalg.inv(C)) / scale).max() < 2e-3
    assert np.linalg.eigvalsh(H).min() > 0


def test_gauss_poly1_fit_pulls_are_standard(oracle_mod):
    # f Gauss + (1 - f) Poly1 at 1e4 events: every parameter is many sigma
    # inside its bounds, so the pulls are close to standard normal.  (The
    # decay model's small toys are not: with a few thousand events its
    # resolution and signal fraction often end on their bounds.)
    s = W.gauss_poly1_model()
    m = oracle_mod.Model(s.nodes, s.root)
    pulls = []
    for k in range(60):
        cols = m.generate(W.GAUSS_POLY1_TRUE, 4242, k, 0, 10000)
        r = m.fit(cols, tol_edm=1e-9)
        assert r["status"] == 0
        pulls.append((r["theta"] - W.GAUSS_POLY1_TRUE) / np.sqrt(np.diag(r["cov"])))
    pulls = np.array(pulls)
    n = len(pulls)
    # mean within ~3.5 standard errors of 0; width within a wide band around 1
    assert np.all(np.abs(pulls.mean(axis=0)) < 3.5 / math.sqrt(n)), pulls.mean(axis=0)
    assert np.all((pulls.std(axis=0) > 0.7) & (pulls.std(axis=0) < 1.35)), pulls.std(axis=0)
