"""CUDA path against the oracle's stored values (tests/golden/oracle_nll.json):
the CUDA generator draws the same events (SHA-256 of the columns), and
rf_nll_grad on them matches the stored NLL to 1e-12 of sum |log p_i| and each
gradient component to 1e-9 of sum_i |dlog p_i/dtheta_k|.  No oracle code runs
here."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

import golden_data as G
from helpers import GRAD_RTOL, NLL_RTOL

pytestmark = pytest.mark.gpu

CASES = G.cases()


@pytest.mark.parametrize("case", CASES, ids=[c["model"] for c in CASES])
def test_cuda_matches_stored_oracle_values(case):
    spec = W.model_for(case["model"])
    m = api.Model.from_spec(spec)
    d = api.generate_toys(m, np.array(case["generate_theta"]), case["seed"], [float(case["events"])],
                          poisson=False)
    assert d.n_events == case["events"]
    cols = [d.read(c) for c in range(m.n_obs)]
    assert G.columns_sha256(cols) == case["columns_sha256"]
    for ev in case["evaluations"]:
        nll, g = api.nll_grad(m, d, np.array(ev["theta"]))
        assert abs(nll - ev["nll"]) <= NLL_RTOL * ev["sum_abs_logp"], (nll, ev["nll"])
        for k in range(len(g)):
            assert abs(g[k] - ev["grad"][k]) <= GRAD_RTOL * ev["sum_abs_grad"][k], (k, g[k], ev["grad"][k])
    d.close()


def test_cuda_binned_matches_stored_oracle_values():
    _, cases = G.binned()
    m = api.BinnedModel(W.binned_model())
    for counts, evals in cases:
        th = np.array([theta for theta, _ in evals])
        nll, g = m.nll_grad(np.tile(counts, (len(evals), 1)), th)
        for i, (_, ev) in enumerate(evals):
            assert abs(nll[i] - ev["nll"]) <= NLL_RTOL * ev["nll_scale"], (nll[i], ev["nll"])
            for k, v in ev["grad"].items():
                assert abs(g[i, int(k)] - v) <= GRAD_RTOL * ev["grad_scale"], (k, g[i, int(k)], v)
