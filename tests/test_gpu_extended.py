"""GPU parity of the Poisson leaf and the extended likelihood against the
oracle: NLL and gradient (generic interpreter and, under an extended root,
the float-float decay kernel), empty sets, domain errors, batched fits (the
extended MLE nu = N), and bitwise generation."""
import math

import numpy as np
import pytest

from paper_2003_12861_gb300 import _lib as L
from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node

from helpers import TRUE, check_nll

pytestmark = pytest.mark.gpu


def poisson_model(a=0, b=40, lam=6.0):
    return [Node("obs", (), 0.0, a, b), Node("param", (), lam, 0.1, 100.0, True), Node("poisson", (0, 1))], 2


def two_poisson_sum():
    # signal + background counts: f Poisson(k; l1) + (1-f) Poisson(k; l2)
    return [Node("obs", (), 0.0, 0, 60), Node("param", (), 4.0, 0.1, 50, True), Node("param", (), 15.0, 0.1, 50, True),
            Node("poisson", (0, 1)), Node("poisson", (0, 2)), Node("param", (), 0.4, 0.0, 1.0, True),
            Node("sum", (3, 4, 5))], 6


def poisson_times_gauss():
    return [Node("obs", (), 0.0, 0, 30), Node("obs", (), 0.0, -5.0, 5.0), Node("param", (), 7.0, 0.1, 50, True),
            Node("poisson", (0, 2)), Node("param", (), 0.2, -3, 3, True), Node("param", (), 1.1, 0.1, 5, True),
            Node("gauss", (1, 4, 5)), Node("prod", (3, 6))], 7


def extended(nodes, root, nu=800.0):
    nodes = list(nodes) + [Node("param", (), nu, 1.0, 1e8, True)]
    nodes.append(Node("extend", (root, len(nodes) - 1)))
    return nodes, len(nodes) - 1


def decay_extended():
    spec = W.decay_model()
    return extended(spec.nodes, spec.root, 5000.0)


CASES = {
    "poisson": (poisson_model(), np.array([6.0])),
    "poisson_offset_range": (poisson_model(3, 17, 9.0), np.array([8.2])),
    "poisson_large_lambda": (poisson_model(100, 400, 230.0), np.array([236.5])),
    "two_poisson_sum": (two_poisson_sum(), np.array([4.2, 14.1, 0.37])),
    "poisson_times_gauss": (poisson_times_gauss(), np.array([7.3, 0.25, 1.05])),
    "extended_poisson": (extended(*poisson_model()), np.array([6.1, 950.0])),
    "extended_decay": (decay_extended(), np.concatenate([TRUE["decay_model"] * 1.01, [4321.0]])),
}


@pytest.mark.parametrize("name", list(CASES))
def test_nll_grad_parity(oracle_mod, name):
    (nodes, root), th = CASES[name]
    om = oracle_mod.Model(nodes, root)
    m = api.Model(nodes, root)
    if name == "extended_decay":
        assert "kernel=ff_" in m.describe()
    for n in (1, 4096 * 3 + 51):
        cols = om.generate(om_default(om, nodes), 11, 0, 0, n)
        d = api.Data.upload(m, cols)
        nll, g = api.nll_grad(m, d, th)
        check_nll(nll, g, om.nll(th, cols), f"{name} n={n}")


def om_default(om, nodes):
    return np.array([nd.value for nd in nodes if nd.kind == "param" and nd.free])


def test_extended_ragged_sets_and_empty(oracle_mod):
    nodes, root = extended(*poisson_model())
    om = oracle_mod.Model(nodes, root)
    m = api.Model(nodes, root)
    sizes = [0, 17, 5000, 0, 4096]
    parts = [om.generate([6.0, 100.0], 5, s, 0, n)[0] if n else np.zeros(0) for s, n in enumerate(sizes)]
    d = api.Data.upload(m, [np.concatenate(parts)], offsets=np.concatenate([[0], np.cumsum(sizes)]))
    th = np.array([[6.2, 30.0 + 10 * s] for s in range(len(sizes))])
    nll, g = api.nll_grad(m, d, th)
    for s, n in enumerate(sizes):
        if n == 0:  # the extended term alone: nu, d/dnu = 1
            assert nll[s] == th[s, 1] and g[s, 1] == 1.0 and g[s, 0] == 0.0
            continue
        check_nll(nll[s], g[s], om.nll(th[s], [parts[s]]), f"set {s}")


def test_domain_errors():
    nodes, root = extended(*poisson_model())
    m = api.Model(nodes, root)
    d = api.Data.upload(m, [np.arange(10.0)])
    for th in ([6.0, -1.0], [0.0, 10.0]):
        with pytest.raises(L.RFError):
            api.nll_grad(m, d, np.array(th))
        nll, _ = api.nll_grad(m, d, np.array(th), allow_domain=True)
        assert math.isinf(nll)
    import torch
    th = torch.tensor([6.0, 10.0], dtype=torch.float64).cuda()
    with pytest.raises(L.RFError):
        api.nll_grad_partial(m, d, th, torch.zeros((1, 3, 2), dtype=torch.float64).cuda(),
                             torch.zeros(1, dtype=torch.int32).cuda())


def test_generation_bitwise(oracle_mod):
    for nodes, root in (poisson_model(0, 40, 6.0), two_poisson_sum(), poisson_times_gauss(), extended(*poisson_model())):
        om = oracle_mod.Model(nodes, root)
        m = api.Model(nodes, root)
        th = om_default(om, nodes)
        d = api.generate_toys(m, th, 77, [6000.0], poisson=False)
        want = om.generate(th, 77, 0, 0, 6000)
        for c in range(len(want)):
            assert np.array_equal(d.read(c), want[c])


def test_batched_extended_fits_give_nu_equal_n(oracle_mod):
    nodes, root = extended(*poisson_model(0, 40, 6.0), nu=500.0)
    om = oracle_mod.Model(nodes, root)
    m = api.Model(nodes, root)
    S = 64
    mean = np.linspace(200.0, 3000.0, S)
    th = np.tile([6.0, 1000.0], (S, 1))
    d = api.generate_toys(m, th, 2024, mean, poisson=True)
    off = d.offsets()
    r = api.fit(m, d)
    x = d.read(0)
    for s in range(S):
        N = off[s + 1] - off[s]
        assert r["status"][s] == 0
        assert abs(r["theta"][s, 1] - N) < 1e-3 * math.sqrt(N), (s, r["theta"][s], N)
        k = np.floor(x[off[s]:off[s + 1]])
        assert abs(r["theta"][s, 0] - k.mean()) < 1e-3 * math.sqrt(6.0 / N)
    # one set against the oracle's own fit: within 1e-3 of the oracle's sigma
    ref = om.fit([x[off[3]:off[4]]])
    sig = np.sqrt(np.diag(ref["cov"]))
    assert np.all(np.abs(r["theta"][3] - ref["theta"]) < 1e-3 * sig), (r["theta"][3], ref["theta"], sig)
