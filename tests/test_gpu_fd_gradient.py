"""The adjoint gradient against central finite differences of the GPU's own
NLL, with steps h = 1e-6 |theta_k| (1e-6 where theta_k = 0), on the
12-parameter product model with FP32 observables and on the decay model.

Tolerance per component: 1e-6 of sum_i |dlog p_i/dtheta_k| (the oracle's
scale).  The central difference's truncation error is O(h^2) (~1e-12
relative) and its rounding error ~1e-14 |NLL| / h, which for these sizes is
below 1e-7 of that scale."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import api

from helpers import TRUE, oracle_data

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which,n", [("prod3_model", 20000), ("decay_model", 30000)])
def test_gradient_matches_central_differences(oracle_mod, which, n):
    spec, om, cols = oracle_data(oracle_mod, which, n, seed=71)
    f32 = which == "prod3_model"
    if f32:
        cols = [c.astype(np.float32).astype(np.float64) for c in cols]
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols, f32=[f32] * len(cols))
    th = np.array(TRUE[which], dtype=np.float64) * 1.01
    nll, g = api.nll_grad(m, d, th)
    _, _, _, ag, _ = om.nll(th, cols)
    for k in range(len(th)):
        h = 1e-6 * abs(th[k]) if th[k] != 0.0 else 1e-6
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (api.nll(m, d, tp) - api.nll(m, d, tm)) / (tp[k] - tm[k])
        assert abs(fd - g[k]) <= 1e-6 * ag[k], (which, k, fd, g[k], ag[k])
