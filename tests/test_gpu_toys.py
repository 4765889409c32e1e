"""GPU toy generation and histograms against the oracle's own implementation of
the same counter-based definition (Philox4x32-10 streams, PTRS Poisson sizes,
accept-reject per factor).  Integer work (sizes, histogram bins) must match
bitwise; the events match bitwise too, because both sides take every
accept/reject decision in FP64 on the same draws (a flip would need a draw
within a few ulp of the density)."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

from helpers import TRUE

pytestmark = pytest.mark.gpu


def test_single_set_matches_oracle(oracle_mod):
    spec = W.gauss_poly1_model()
    m = api.Model.from_spec(spec)
    om = oracle_mod.Model(spec.nodes, spec.root)
    d = api.generate_toys(m, TRUE["gauss_poly1_model"], 20031286, [10000.0], poisson=False)
    assert d.n_events == 10000
    got = d.read(0)
    want = om.generate(TRUE["gauss_poly1_model"], 20031286, 0, 0, 10000)[0]
    assert np.array_equal(got, want)


def test_ragged_poisson_toys_match_oracle(oracle_mod):
    spec = W.decay_model()
    m = api.Model.from_spec(spec)
    om = oracle_mod.Model(spec.nodes, spec.root)
    S = 24
    mean = W.toy_mean_sizes(S, 99, 3.0, 2e4)   # includes means below 10 (inversion branch)
    mean[0] = 0.0
    mean[1] = 4.5
    th = W.toy_thetas(S, 99)
    seed = 0x1234_5678_9ABC
    d = api.generate_toys(m, th, seed, mean, poisson=True)
    off = d.offsets()
    sizes = np.diff(off)
    want_sizes = np.array([oracle_mod.poisson(seed, s, mean[s]) for s in range(S)])
    assert np.array_equal(sizes, want_sizes)
    col = d.read(0)
    for s in range(S):
        if sizes[s] == 0:
            continue
        want = om.generate(th[s], seed, s, 0, int(sizes[s]))[0]
        assert np.array_equal(col[off[s]:off[s + 1]], want), s


def test_product_factors_f32_columns(oracle_mod):
    spec = W.prod3_model()
    m = api.Model.from_spec(spec)
    om = oracle_mod.Model(spec.nodes, spec.root)
    n = 9000
    d = api.generate_toys(m, TRUE["prod3_model"], 7, [float(n)], poisson=False, f32=[True, True, True])
    want = om.generate(TRUE["prod3_model"], 7, 0, 0, n)
    for c in range(3):
        got = d.read(c)
        assert np.array_equal(got, want[c].astype(np.float32).astype(np.float64)), c


def test_sampled_events_at_scale(oracle_mod):
    # 2e6 events generated on the device; the oracle regenerates a sample of
    # 4096-event windows by their counters alone.
    spec = W.decay_model()
    m = api.Model.from_spec(spec)
    om = oracle_mod.Model(spec.nodes, spec.root)
    n = 2_000_000
    d = api.generate_toys(m, TRUE["decay_model"], 31, [float(n)], poisson=False)
    for i0 in [0, 409600, 1234567, n - 4096]:
        got = d.read(0, i0, i0 + 4096)
        want = om.generate(TRUE["decay_model"], 31, 0, i0, i0 + 4096)[0]
        assert np.array_equal(got, want), i0


def test_hist64_matches_oracle(oracle_mod):
    import torch

    spec = W.decay_model()
    m = api.Model.from_spec(spec)
    S = 8
    mean = W.toy_mean_sizes(S, 5)
    d = api.generate_toys(m, TRUE["decay_model"], 5, mean, poisson=True)
    out = torch.zeros(S * 64, dtype=torch.float32, device="cuda")
    api.hist64(m, d, 0, out)
    torch.cuda.synchronize()
    h = out.cpu().numpy().reshape(S, 64)
    off = d.offsets()
    col = d.read(0)
    for s in range(S):
        want = oracle_mod.hist64(col[off[s]:off[s + 1]], 0.0, 10.0)
        assert np.array_equal(h[s], want), s
