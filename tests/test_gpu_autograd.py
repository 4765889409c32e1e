"""The torch binding RfNLL: forward is one device pass (rf_nll_grad_async),
backward the saved gradient; both equal rf_nll_grad's results exactly."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_single_set_matches_nll_grad():
    m = api.Model.from_spec(W.decay_model())
    d = api.generate_toys(m, W.DECAY_TRUE, 21, [30000.0], poisson=False)
    ref_nll, ref_g = api.nll_grad(m, d, W.DECAY_START)
    th = torch.tensor(W.DECAY_START, dtype=torch.float64, device="cuda", requires_grad=True)
    nll = api.RfNLL.apply(th, m, d)
    assert nll.dim() == 0 and nll.item() == ref_nll
    nll.backward()
    assert np.array_equal(th.grad.cpu().numpy(), ref_g)
    # the chain rule through a scaled objective
    th.grad = None
    (3.0 * api.RfNLL.apply(th, m, d)).backward()
    assert np.array_equal(th.grad.cpu().numpy(), 3.0 * ref_g)


def test_batched_and_shared_theta():
    m = api.Model.from_spec(W.decay_model())
    S = 5
    th_sets = np.tile(W.DECAY_TRUE, (S, 1)) * (1 + 0.02 * np.arange(S))[:, None]
    d = api.generate_toys(m, th_sets, 22, np.full(S, 8000.0))
    ref_nll, ref_g = api.nll_grad(m, d, th_sets)
    th = torch.tensor(th_sets, dtype=torch.float64, device="cuda", requires_grad=True)
    nll = api.RfNLL.apply(th, m, d)
    assert nll.shape == (S,) and np.array_equal(nll.detach().cpu().numpy(), ref_nll)
    w = torch.arange(1, S + 1, dtype=torch.float64, device="cuda")
    (w * nll).sum().backward()
    assert np.array_equal(th.grad.cpu().numpy(), np.arange(1, S + 1)[:, None] * ref_g)
    # one theta shared by every set: the gradient sums over the sets
    sh = torch.tensor(W.DECAY_TRUE, dtype=torch.float64, device="cuda", requires_grad=True)
    nll_s = api.RfNLL.apply(sh, m, d)
    r_nll, r_g = api.nll_grad(m, d, np.tile(W.DECAY_TRUE, S))
    assert np.array_equal(nll_s.detach().cpu().numpy(), r_nll)
    nll_s.sum().backward()
    np.testing.assert_allclose(sh.grad.cpu().numpy(), r_g.sum(0), rtol=1e-15, atol=0)


def test_gradient_descent_lowers_the_nll():
    m = api.Model.from_spec(W.gauss_poly1_model())
    d = api.generate_toys(m, W.GAUSS_POLY1_TRUE, 23, [20000.0], poisson=False)
    th = torch.tensor(W.GAUSS_POLY1_TRUE * np.array([1.02, 1.1, 0.9, 1.0]), dtype=torch.float64,
                      device="cuda", requires_grad=True)
    opt = torch.optim.SGD([th], lr=1e-7)
    first = None
    for _ in range(5):
        opt.zero_grad()
        nll = api.RfNLL.apply(th, m, d)
        first = nll.item() if first is None else first
        nll.backward()
        opt.step()
    assert api.RfNLL.apply(th, m, d).item() < first
