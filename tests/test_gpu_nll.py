"""GPU parity of rf_nll / rf_nll_grad against the CPU oracle, element by
element, on datasets the oracle generates (several 4096-event chunks and a
ragged tail), plus edge cases and determinism."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import _lib as L
from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node

from helpers import TRUE, check_nll, oracle_data

pytestmark = pytest.mark.gpu


def thetas(which):
    t = TRUE[which]
    spec = W.model_for(which)
    lo, hi = spec.bounds().T
    out = [t, t * (1 + 0.05 * np.cos(np.arange(len(t)) * 1.7)), spec.defaults()]
    if which == "decay_model":
        # mu_r shifted right: events with t < mu_r take the erfcx branch,
        # events near mu_r the erfc branch of the slow path.
        out.append(np.array([1.2, 0.3, 0.2, -0.1, 0.02, 0.4]))
        out.append(np.array([0.4, -0.2, 0.6, 0.1, -0.05, 0.7]))
        # float-float edge regimes: a decay that underflows long before t = 10,
        # a pure signal (the total density itself underflows), no signal
        out.append(np.array([0.12, 0.0, 0.05, -0.2, 0.05, 0.2]))
        out.append(np.array([0.3, 0.0, 0.05, -0.2, 0.05, 1.0]))
        out.append(np.array([1.5, 0.0, 0.05, -0.2, 0.05, 0.0]))
    if which == "gauss_poly1_model":
        out.append(np.array([5.0, 0.05, 0.3, -0.05]))   # narrow: far tails underflow
        out.append(np.array([9.9, 0.3, 1.0, 0.0]))      # pure Gaussian at the range edge
    if which == "prod3_model":
        e = t.copy()
        e[0], e[1] = 5.205, 0.003                       # mass peak at the range edge, narrow
        out.append(e)
    return out


@pytest.mark.parametrize("which,n", [("gauss_poly1_model", 10000), ("decay_model", 30001), ("prod3_model", 20000)])
def test_nll_grad_parity(oracle_mod, which, n):
    spec, om, cols = oracle_data(oracle_mod, which, n, seed=11)
    m = api.Model.from_spec(spec)
    f32 = which == "prod3_model"
    if f32:  # observables stored in FP32: both sides see the same rounded values
        cols = [c.astype(np.float32).astype(np.float64) for c in cols]
    d = api.Data.upload(m, cols, f32=[f32] * len(cols))
    for th in thetas(which):
        nll, g = api.nll_grad(m, d, th)
        ref = om.nll(th, cols)
        check_nll(nll, g, ref, which)
        assert api.nll(m, d, th) == nll  # the NLL-only pass sums in the same tree


@pytest.mark.parametrize("n", [0, 1, 127, 128, 4095, 4096, 4097, 8192 + 33, 32 * 4096 + 5])
def test_sizes_and_ragged_tails(oracle_mod, n):
    spec, om, cols = oracle_data(oracle_mod, "decay_model", max(n, 1), seed=5)
    cols = [c[:n] for c in cols]
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols)
    th = TRUE["decay_model"]
    nll, g = api.nll_grad(m, d, th)
    if n == 0:
        assert nll == 0.0 and np.all(g == 0.0)
    else:
        check_nll(nll, g, om.nll(th, cols), f"n={n}")


def test_ragged_sets(oracle_mod):
    spec = W.decay_model()
    om = oracle_mod.Model(spec.nodes, spec.root)
    sizes = [0, 1, 4096, 5000, 130000, 17, 0, 4097]
    cols, off = [], [0]
    for s, n in enumerate(sizes):
        cols.append(om.generate(TRUE["decay_model"], 21, s, 0, n)[0] if n else np.zeros(0))
        off.append(off[-1] + n)
    allc = np.concatenate(cols)
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, [allc], offsets=off)
    rng = np.random.Generator(np.random.PCG64(3))
    th = np.array([TRUE["decay_model"] * (1 + 0.1 * rng.uniform(-1, 1, 6)) for _ in sizes])
    nll, g = api.nll_grad(m, d, th)
    for s, n in enumerate(sizes):
        if n == 0:
            assert nll[s] == 0.0
            continue
        check_nll(nll[s], g[s], om.nll(th[s], [cols[s]]), f"set {s}")


def test_deterministic_across_launch_shapes_and_reruns(oracle_mod):
    spec, om, cols = oracle_data(oracle_mod, "decay_model", 200000, seed=8)
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols)
    th = TRUE["decay_model"]
    ref = api.nll_grad(m, d, th)
    for bps in [1, 2, 3, 8, 16]:
        m.set_launch(0, bps)
        for _ in range(2):
            r = api.nll_grad(m, d, th)
            assert r[0] == ref[0] and np.array_equal(r[1], ref[1]), bps


def test_deterministic_whole_chunk_units_and_autotune_grid():
    """A dataset of >= 1024 chunks runs whole-chunk work units (three FP32
    columns: the all-FP32 kernel): its result is bitwise the same for every
    launch shape the autotuner tries, and the tuner reports its grid."""
    spec = W.prod3_model()
    m = api.Model.from_spec(spec)
    d = api.generate_toys(m, TRUE["prod3_model"], 31, [1100 * 4096 + 77.0], poisson=False, f32=[True] * 3)
    th = TRUE["prod3_model"] * (1 + 0.01 * np.cos(np.arange(12)))
    ref = api.nll_grad(m, d, th)
    grid = api.autotune_scan(m, d, passes=1)
    assert len(grid) >= 3 and all(t > 0 for _, t in grid)
    assert {b for b, _ in grid} <= {1, 2, 3, 4, 5, 6, 7, 8, 12, 16}
    for bps in [b for b, _ in grid] + [0]:
        m.set_launch(0, bps)
        r = api.nll_grad(m, d, th)
        assert r[0] == ref[0] and np.array_equal(r[1], ref[1]), bps


def test_domain_errors(oracle_mod):
    # A polynomial that goes negative inside the range: pdf < 0 for some events.
    nodes = [Node("obs", (), 0, 0, 10), Node("param", (), -0.2, -1, 1, True), Node("poly", (0, 1))]
    m = api.Model(nodes, 2)
    x = np.linspace(0.01, 9.99, 5000)
    d = api.Data.upload(m, [x])
    with pytest.raises(L.RFError) as e:
        api.nll(m, d, [-0.2])
    assert e.value.status == L.RF_E_DOMAIN
    assert api.nll(m, d, [-0.2], allow_domain=True) == np.inf
    assert np.isfinite(api.nll(m, d, [0.05]))
    # sigma <= 0 is outside the Gaussian's domain
    spec = W.gauss_poly1_model()
    mg = api.Model.from_spec(spec)
    dg = api.Data.upload(mg, [x])
    th = W.GAUSS_POLY1_TRUE.copy()
    th[1] = -0.5
    assert api.nll(mg, dg, th, allow_domain=True) == np.inf


def test_sum_and_prod_special_cases(oracle_mod):
    # SUM with f = 1 equals its first component; PROD of one factor equals the factor.
    x = np.linspace(0.05, 9.95, 9000)
    base = [Node("obs", (), 0, 0, 10), Node("param", (), 4.0, 0, 10, True), Node("param", (), 1.2, 0.1, 5, True),
            Node("gauss", (0, 1, 2)), Node("param", (), 0.1, -1, 1, True), Node("cheb", (0, 4)),
            Node("param", (), 1.0, 0, 1, False), Node("sum", (3, 5, 6)), Node("prod", (3,))]
    th = np.array([4.0, 1.2, 0.1])
    m_sum = api.Model(base, 7)
    m_leaf = api.Model(base, 3)
    m_prod = api.Model(base, 8)
    vals = [api.nll_grad(mm, api.Data.upload(mm, [x]), th) for mm in (m_sum, m_leaf, m_prod)]
    om = oracle_mod.Model(base, 3)
    check_nll(vals[1][0], vals[1][1], om.nll(th, [x]))
    assert abs(vals[0][0] - vals[1][0]) <= 1e-12 * abs(vals[1][0])
    assert vals[2][0] == vals[1][0]


def test_generic_graph_other_kinds(oracle_mod):
    # EXP and a 3-component SUM with a shared parameter and a fixed one.
    nodes = [Node("obs", (), 0, -1.0, 4.0),
             Node("param", (), -0.6, -5, 5, True),     # c
             Node("param", (), 1.0, -5, 5, True),      # mu (shared by two Gaussians)
             Node("param", (), 0.3, 0.01, 5, True),
             Node("param", (), 0.9, 0.01, 5, False),   # fixed width
             Node("exp", (0, 1)), Node("gauss", (0, 2, 3)), Node("gauss", (0, 2, 4)),
             Node("param", (), 0.5, 0, 1, True), Node("param", (), 0.2, 0, 1, True),
             Node("sum", (5, 6, 7, 8, 9))]
    om = oracle_mod.Model(nodes, 10)
    x = om.generate(np.array([-0.6, 1.0, 0.3, 0.5, 0.2]), 3, 0, 0, 12345)[0]
    m = api.Model(nodes, 10)
    d = api.Data.upload(m, [x])
    for th in [np.array([-0.6, 1.0, 0.3, 0.5, 0.2]), np.array([0.0, 0.8, 0.5, 0.3, 0.3]),
               np.array([2e-7, 1.2, 0.2, 0.6, 0.1])]:
        nll, g = api.nll_grad(m, d, th)
        check_nll(nll, g, om.nll(th, [x]))


def test_chunk_partials_match_oracle(oracle_mod):
    spec, om, cols = oracle_data(oracle_mod, "decay_model", 5 * 4096 + 100, seed=19)
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, cols)
    th = TRUE["decay_model"]
    parts = api.nll_chunks(m, d, th)
    assert parts.shape == (6, 1 + m.n_free)
    for c in range(6):
        sl = [col[c * 4096:(c + 1) * 4096] for col in cols]
        nll, g, al, ag, _ = om.nll(th, sl)
        assert abs(parts[c, 0] - (-nll)) <= 1e-12 * al
        assert np.all(np.abs(parts[c, 1:] - (-g)) <= 1e-9 * ag)


def test_device_resident_async_pass(oracle_mod):
    import torch

    spec, om, cols = oracle_data(oracle_mod, "decay_model", 50000, seed=23)
    m = api.Model.from_spec(spec)
    tcols = [torch.from_numpy(c).cuda() for c in cols]
    d = api.Data.from_torch(m, tcols)
    th = torch.tensor(TRUE["decay_model"], dtype=torch.float64, device="cuda")
    out = torch.zeros(1 + m.n_free, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        api.nll_grad_async(m, d, th, out, flags, stream=s)
    s.synchronize()
    o = out.cpu().numpy()
    check_nll(o[0], o[1:], om.nll(TRUE["decay_model"], cols))
    assert int(flags.item()) == 0


def test_launch_count(oracle_mod):
    """rf_launch_count: one pass is K1 + the event kernel; a batched fit's
    graph replays count their two kernels each."""
    spec = W.decay_model()
    m = api.Model.from_spec(spec)
    d = api.generate_toys(m, W.DECAY_TRUE, 3, [20000.0], poisson=False)
    api.nll_grad(m, d, W.DECAY_TRUE)
    n0 = api.launch_count()
    api.nll_grad(m, d, W.DECAY_TRUE)
    assert api.launch_count() - n0 == 2
    sets = api.generate_toys(m, np.tile(W.DECAY_TRUE, (8, 1)), 4, np.full(8, 3000.0))
    api.fit(m, sets, want_cov=False)  # first fit captures its graphs
    n1 = api.launch_count()
    r = api.fit(m, sets, want_cov=False)
    n = api.launch_count() - n1
    assert n % 2 == 0 and int(r["n_evals"].max()) <= n // 2 <= 2 * int(r["n_evals"].max()) + 2
