"""The oracle still reproduces its stored values (tests/golden/oracle_nll.json,
written by tests/golden/make_oracle_golden.py): the same events from the
counter-based generator, and the same NLL and gradient to a few ulp of their
scales (the host's libm may round exp/log/erfc differently in the last bit).
A change to the oracle's arithmetic shows up here and must be justified by
the definition it follows before the file is rewritten."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import workloads as W

import golden_data as G

CASES = G.cases()


@pytest.mark.parametrize("case", CASES, ids=[c["model"] for c in CASES])
def test_oracle_reproduces_stored_values(oracle_mod, case):
    spec = W.model_for(case["model"])
    om = oracle_mod.Model(spec.nodes, spec.root)
    cols = om.generate(np.array(case["generate_theta"]), case["seed"], case["set"], 0, case["events"])
    assert G.columns_sha256(cols) == case["columns_sha256"]
    for ev in case["evaluations"]:
        nll, g, al, ag, rc = om.nll(np.array(ev["theta"]), cols)
        assert rc == 0
        assert abs(nll - ev["nll"]) <= 1e-14 * ev["sum_abs_logp"]
        for k in range(len(g)):
            assert abs(g[k] - ev["grad"][k]) <= 1e-14 * ev["sum_abs_grad"][k], k


def test_binned_oracle_reproduces_stored_values():
    from oracle import binned as OB

    _, cases = G.binned()
    om = OB.from_spec(W.binned_model())
    for counts, evals in cases:
        for theta, ev in evals:
            nll, g, scale = om.nll(theta, counts)
            assert abs(nll - ev["nll"]) <= 1e-14 * ev["nll_scale"]
            for k, v in ev["grad"].items():
                assert abs(g[int(k)] - v) <= 1e-14 * ev["grad_scale"], k
