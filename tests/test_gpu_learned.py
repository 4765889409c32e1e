"""What the trained network gains over the method without it: on fresh toys,
fits started from the network's prediction converge in fewer evaluations
than fits from the plain default start and reach the same (or a lower)
minimum.  A small training set (toys of 1e3-5e3 events) keeps it quick."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import api, learned
from paper_2003_12861_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_learned_start_beats_plain_start():
    model = api.Model.from_spec(W.decay_model())
    X, Y, info = learned.build_training_set(model, 16384, seed=123, n_lo=1e3, n_hi=5e3)
    assert info["converged"] > 0.9 * info["toys"]
    net, tinfo = learned.train(X, Y, epochs=30, batch=512, lr=2e-3, seed=7)
    r = learned.compare(net, model, 2048, seed=98765, n_lo=1e3, n_hi=5e3)
    assert r["learned"]["mean_evals"] < 0.85 * r["plain"]["mean_evals"], r
    assert r["learned"]["wall_s"] < r["plain"]["wall_s"], r
    # Small toys of this model often have several local minima, so neither
    # start always finds the deepest one; the learned start must reach the
    # plain fit's minimum for most toys and must not be worse on balance.
    assert r["same_minimum_frac"] >= 0.6, r
    assert r["learned_higher_nll_frac"] <= r["learned_lower_nll_frac"] + 0.05, r
    assert r["learned"]["converged"] >= r["plain"]["converged"] - 0.01, r
