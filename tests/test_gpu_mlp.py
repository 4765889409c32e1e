"""The learned-start network on the GPU (tensor-core BF16 GEMMs, FP32
accumulation) against the float64 oracle with the same BF16 operand
rounding.  Tolerance: the only differences are FP32 accumulation (~1e-6
relative) and the rare BF16 rounding of an activation that lands on the other
side of a rounding boundary (one BF16 ulp, 2^-8, in a few elements), so
outputs and gradients agree to 1e-2 of their largest magnitude and mostly to
1e-4."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2003_12861_gb300 import api

pytestmark = pytest.mark.gpu

SHAPES = M.layer_shapes(64, 128, 3, 6)


def net_and_data(B, seed=0):
    net = api.MLP(seed=seed)
    p = net.get_params()
    rng = np.random.default_rng(seed + 1)
    x = rng.dirichlet(np.ones(64), size=B).astype(np.float32) * 3.0  # histogram-like inputs
    t = rng.standard_normal((B, 6)).astype(np.float32)
    return net, p, x, t


def close(a, b, scale_rtol=1e-2, med_rtol=1e-4):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    scale = np.max(np.abs(b))
    err = np.abs(a - b)
    assert err.max() <= scale_rtol * scale, (err.max(), scale)
    assert np.median(err) <= med_rtol * scale, (np.median(err), scale)


@pytest.mark.parametrize("B", [1, 37, 300, 1024])
def test_forward_matches_oracle(B):
    net, p, x, _ = net_and_data(B)
    dx = torch.from_numpy(x).cuda()
    dy = torch.zeros(B, 6, device="cuda")
    net.forward(dx, dy)
    torch.cuda.synchronize()
    want, _ = M.forward(p, x, SHAPES)
    close(dy.cpu().numpy(), want)


@pytest.mark.parametrize("B", [64, 333])
def test_gradient_matches_oracle(B):
    net, p, x, t = net_and_data(B, seed=7)
    # train a little first so that the activations are not all near initial values
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    g = torch.zeros(net.n_params, device="cuda")
    loss = net.grad(dx, dt, g)
    torch.cuda.synchronize()
    want_loss, want_g = M.loss_and_grad(p, x, t, SHAPES)
    assert abs(loss - want_loss) <= 1e-4 * want_loss
    gg = g.cpu().numpy()
    o = 0
    for (i, j) in SHAPES:  # per layer: weights then biases
        for n in (i * j, j):
            close(gg[o:o + n], want_g[o:o + n], scale_rtol=2e-2, med_rtol=2e-3)
            o += n


def test_adam_step_matches_oracle():
    net, p, x, t = net_and_data(128, seed=3)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    g = torch.zeros(net.n_params, device="cuda")
    net.grad(dx, dt, g)
    net.adam(1e-3)
    torch.cuda.synchronize()
    got = net.get_params()
    want, _, _ = M.adam(p, g.cpu().numpy().astype(np.float64), np.zeros(p.size), np.zeros(p.size), 1, 1e-3)
    assert np.allclose(got, want, rtol=0, atol=2e-7)


def test_training_learns_and_checkpoints(tmp_path):
    # a smooth target the network can fit: a fixed random linear map of x
    rng = np.random.default_rng(11)
    x = rng.dirichlet(np.ones(64), size=8192).astype(np.float32) * 3.0
    A = rng.standard_normal((64, 6)).astype(np.float32)
    t = (x @ A * 5.0 + 2.0).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    net = api.MLP(seed=5)
    l1 = net.train(dx, dt, batch=512, epochs=1, lr=1e-3, seed=1)
    l20 = net.train(dx, dt, batch=512, epochs=20, lr=1e-3, seed=2)
    assert l20 < 0.05 * l1, (l1, l20)
    dy = torch.zeros(8192, 6, device="cuda")
    net.forward(dx, dy)
    torch.cuda.synchronize()
    rel = np.sqrt(np.mean((dy.cpu().numpy() - t) ** 2)) / t.std()
    assert rel < 0.1, rel
    path = str(tmp_path / "net.bin")
    net.save(path)
    net2 = api.MLP.load(path)
    dy2 = torch.zeros(8192, 6, device="cuda")
    net2.forward(dx, dy2)
    torch.cuda.synchronize()
    assert torch.equal(dy, dy2)
    # training is bitwise reproducible
    n1, n2 = api.MLP(seed=9), api.MLP(seed=9)
    n1.train(dx, dt, batch=256, epochs=2, seed=4)
    n2.train(dx, dt, batch=256, epochs=2, seed=4)
    assert np.array_equal(n1.get_params(), n2.get_params())


def test_predict_is_histogram_then_forward():
    """rf_mlp_predict: per set the 64-bin histogram, the forward pass and the
    prediction on the host -- the same values as the two calls by hand."""
    from paper_2003_12861_gb300 import workloads as W

    m = api.Model.from_spec(W.decay_model())
    S = 7
    d = api.generate_toys(m, np.tile(W.DECAY_TRUE, (S, 1)), 31, np.full(S, 2500.0))
    net = api.MLP(seed=5)
    got = net.predict(m, d)
    assert got.shape == (S, m.n_free)
    h = torch.zeros(S * 64, dtype=torch.float32, device="cuda")
    api.hist64(m, d, 0, h)
    y = torch.zeros(S, 6, dtype=torch.float32, device="cuda")
    net.forward(h.view(S, 64), y)
    torch.cuda.synchronize()
    assert np.array_equal(got, y.cpu().numpy().astype(np.float64))
    bad = api.MLP(n_in=64, n_hidden=16, n_hidden_layers=1, n_out=4, seed=1)
    with pytest.raises(RuntimeError):
        bad.predict(m, d)
