"""Pins of the MLP oracle: BF16 rounding against torch's bfloat16 cast, GELU
against torch's exact GELU, the backward formulas against central finite
differences (roundings off), Adam against torch.optim.Adam."""
import numpy as np
import torch

from oracle import mlp as M

SHAPES = M.layer_shapes(8, 16, 2, 3)


def params(seed=0, scale=0.3):
    n = sum(i * j + j for i, j in SHAPES)
    return (np.random.default_rng(seed).standard_normal(n) * scale).astype(np.float32)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(1).standard_normal(100000).astype(np.float32) * 10
    x[:4] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -(1.0 + 2 ** -9), 0.0]  # ties and the like
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), want)


def test_gelu_matches_torch():
    z = np.linspace(-8, 8, 4001)
    want = torch.nn.functional.gelu(torch.from_numpy(z), approximate="none").numpy()
    assert np.allclose(M.gelu(z), want, rtol=0, atol=1e-15)
    h = 1e-6
    assert np.allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), rtol=0, atol=1e-8)


def test_backward_matches_finite_differences():
    p = params().astype(np.float64)
    rng = np.random.default_rng(2)
    x = rng.random((7, 8))
    y = rng.standard_normal((7, 3))
    loss, g = M.loss_and_grad(p, x, y, SHAPES, rounding=False)
    idx = rng.choice(len(p), 40, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, x, y, SHAPES, rounding=False)[0] - M.loss_and_grad(pm, x, y, SHAPES, rounding=False)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, g[i], fd)


def test_forward_matches_torch_reference_without_rounding():
    p = params(3).astype(np.float64)
    x = np.random.default_rng(4).random((5, 8))
    out, _ = M.forward(p, x, SHAPES, rounding=False)
    layers = M.unpack(p, SHAPES)
    a = torch.from_numpy(x)
    for li, (W, b) in enumerate(layers):
        a = a @ torch.from_numpy(W) + torch.from_numpy(b)
        if li < len(layers) - 1:
            a = torch.nn.functional.gelu(a)
    assert np.allclose(out, a.numpy(), rtol=1e-13, atol=1e-13)


def test_adam_matches_torch():
    p = params(5)
    g = np.random.default_rng(6).standard_normal(p.size)
    tp = torch.nn.Parameter(torch.from_numpy(p.astype(np.float64)))
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    cur = p.copy()
    for t in range(1, 4):
        tp.grad = torch.from_numpy(g * t)
        opt.step()
        cur, m, v = M.adam(cur, g * t, m, v, t, 1e-3)
    assert np.allclose(cur, tp.detach().numpy(), rtol=0, atol=1e-6)
