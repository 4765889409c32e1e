"""The library's float-float elementary functions (Tang's table-driven exp and
log, Newton reciprocal, piecewise-Chebyshev erfcx) against CUDA's FP64
functions on the GPU and against 50-digit mpmath on a sample.

Bounds, from the error analysis: a float pair holds ~48 bits, so a double
input is rounded by up to 2^-48 relative on conversion; exp amplifies that by
|x| (error <= 3e-14 + 2^-47 |x|); one Newton step from the hardware
reciprocal leaves ~2^-46; log and erfcx stay below 3e-14 relative (log:
relative to max(1, |log x|)).  All are far inside what the likelihood
tolerances (1e-12 on the NLL, 1e-9 on the gradient) need."""
import mpmath as mp
import numpy as np
import pytest
import torch

from paper_2003_12861_gb300 import api

pytestmark = pytest.mark.gpu


def run(fn, x):
    dx = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    dy = torch.empty_like(dx)
    api.math_eval(fn, dx, dy)
    torch.cuda.synchronize()
    return dy.cpu().numpy()


def inputs(kind):
    rng = np.random.default_rng(42)
    if kind == "exp":
        return np.concatenate([rng.uniform(-69, 69, 400000), rng.uniform(-1e-3, 1e-3, 10000),
                               [0.0, 1e-30, -1e-30, 1.0, -1.0, 0.5, -68.9, 68.9, np.log(2)]])
    if kind == "log":
        return np.concatenate([np.exp(rng.uniform(np.log(1e-29), np.log(1e29), 400000)),
                               1 + rng.uniform(-1e-3, 1e-3, 10000), 1 + rng.uniform(-1e-12, 1e-12, 1000),
                               [1.0, 2.0, 0.5, 1 - 2 ** -24, 1 + 2 ** -23, 3.0, 1e-29]])
    if kind == "rcp":
        return np.concatenate([np.exp(rng.uniform(-60, 60, 400000)) * rng.choice([-1, 1], 400000), [1.0, 3.0, -7.0]])
    if kind == "erfcx":
        return np.concatenate([rng.uniform(0, 10, 300000), np.exp(rng.uniform(np.log(1e-8), np.log(1e8), 100000)),
                               [0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 1e-30, 1e20]])


@pytest.mark.parametrize("kind,fn,ref", [("exp", 0, 10), ("log", 1, 11), ("rcp", 2, 12), ("erfcx", 3, 13)])
def test_ff_function_against_cuda_fp64(kind, fn, ref):
    x = inputs(kind)
    got = run(fn, x)
    want = run(ref, x)
    assert np.all(np.isfinite(got)), x[~np.isfinite(got)][:5]
    if kind == "log":
        # the double input is rounded to ~48 bits on conversion: 2^-47 absolute near 1
        err = np.abs(got - want) - 3e-14 * np.abs(want) - 2.0 ** -47
        assert err.max() <= 0, (err.max(), x[np.argmax(err)])
        # inputs a float pair holds exactly (<= 46 significant bits): full
        # relative precision of log(x) near 1
        near = np.round((1 + np.random.default_rng(3).uniform(-1e-3, 1e-3, 20000)) * 2.0 ** 45) / 2.0 ** 45
        near = near[near != 1.0]
        g2, w2 = run(fn, near), run(ref, near)
        rel = np.abs(g2 - w2) / np.abs(w2)
        assert rel.max() < 3e-13, (rel.max(), near[np.argmax(rel)])
    else:
        rel = np.abs(got - want) / np.abs(want)
        bound = 3e-14 + (2.0 ** -47) * np.abs(x) if kind == "exp" else 3e-14
        assert np.all(rel < bound), (rel.max(), x[np.argmax(rel / bound)])


def test_ff_erfcx_and_exp_against_mpmath():
    mp.mp.dps = 40
    y = np.array([0.0, 0.1, 0.49, 0.51, 0.99, 1.01, 1.7, 1.99, 2.01, 3.3, 3.99, 4.01, 6.0, 7.99, 8.01, 30.0, 1e4])
    got = run(3, y)
    for yi, gi in zip(y, got):
        want = mp.exp(mp.mpf(yi) ** 2) * mp.erfc(mp.mpf(yi))
        assert abs(gi - float(want)) <= 3e-14 * float(want), (yi, gi, want)
    x = np.array([-68.0, -6.7, -0.3, 0.0, 1e-8, 2.5, 40.0])
    got = run(0, x)
    for xi, gi in zip(x, got):
        want = mp.exp(mp.mpf(xi))
        assert abs(gi - float(want)) <= 3e-14 * float(want) + 2.0 ** -47 * abs(xi) * float(want), (xi, gi, want)


def test_ff_out_of_range_is_flagged():
    assert np.isnan(run(0, np.array([-80.0, 90.0]))).all()
    assert np.isnan(run(1, np.array([0.0, -1.0, 1e-35]))).all()
