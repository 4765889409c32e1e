"""What the trained network gains over the method without it: on fresh toys,
fits started from the network's prediction converge in fewer evaluations
than fits from the plain default start and reach the same minimum for most
toys; the rest are characterised (distinct minima, mostly on a bound).  A
small training set (toys of 1e3-5e3 events) keeps it quick."""
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
    r = learned.compare(net, model, 2048, seed=98765, n_lo=1e3, n_hi=5e3, characterise=True)
    print({k: r[k] for k in ("same_minimum_frac", "learned_lower_nll_frac", "learned_higher_nll_frac",
                             "at_lowest_of_three_minima_frac")},
          r["plain"]["mean_evals"], r["learned"]["mean_evals"], r["mismatch"])
    assert r["learned"]["mean_evals"] < 0.85 * r["plain"]["mean_evals"], r
    assert r["learned"]["wall_s"] < r["plain"]["wall_s"], r
    assert r["learned"]["converged"] >= r["plain"]["converged"] - 0.01, r
    # Toys of 1e3-5e3 events of this model often have several local minima
    # (measured: 85.1 % identical, 8.0 % learned lower, 6.9 % higher, with
    # fits to EDM < 1e-9).  The learned start must reach the plain fit's
    # minimum for most toys and must not be worse on balance; the toys where
    # the two differ are distinct minima (a tight refit from both end points
    # rarely joins them), most with a parameter on a bound.
    assert r["same_minimum_frac"] >= 0.80, r
    assert r["learned_higher_nll_frac"] <= r["learned_lower_nll_frac"], r
    # against the lowest of three minima (plain, learned, generating values;
    # measured 88.3 %, 89.3 %, 87.7 %): the learned start finds it at least
    # as often as the plain one
    ab = r["at_lowest_of_three_minima_frac"]
    assert ab["learned"] >= ab["plain"], ab
    for side in ("learned_higher", "learned_lower"):
        mm = r["mismatch"][side]
        if mm["count"] >= 20:
            assert mm["resolved_by_tight_refit"] <= 0.25, mm
            assert mm["near_a_bound"] >= 0.5, mm


def test_learned_starts_stay_inside_the_bounds():
    """rf_mlp_predict keeps every bounded parameter's start 5 % of its range
    inside the bounds: an untrained network's outputs (near 0) fall below
    the band of tau and f_sig, and are moved onto its edge."""
    model = api.Model.from_spec(W.decay_model())
    data = api.generate_toys(model, W.toy_thetas(256, 5), 5, W.toy_mean_sizes(256, 5, 1e3, 5e3), poisson=True)
    net = api.MLP(seed=3)
    lo, hi = (np.array(v) for v in learned.model_bounds(model))
    a, b = lo + 0.05 * (hi - lo), hi - 0.05 * (hi - lo)
    t = learned.predict_starts(net, model, data)
    assert np.all(t >= a - 1e-12) and np.all(t <= b + 1e-12), (t.min(axis=0), t.max(axis=0))
    assert np.any(np.isclose(t, a) | np.isclose(t, b)), t[:4]
