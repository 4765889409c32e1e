"""Learned fit start: build the training set with the method itself, train the
network, and compare learned-start fits with plain-start fits.

Orchestration only: toys are generated (rf_generate_toys), histogrammed
(rf_hist64) and fitted (rf_fit) by the library, the network is trained and
evaluated by its kernels (rf_mlp_*); PyTorch holds the device buffers.

Training labels are the plain fits' minima (theta-hat) of each training toy,
whose generating parameters are drawn uniformly within +-30 % of the decay
model's values; the plain fit from the default start is also the fallback
and the yardstick: a learned start that fails (outside the domain, or no
convergence) is refitted from the default start, and a learned fit that ends
in a different minimum (|delta NLL| >= 1e-6) is counted and reported.
"""
from __future__ import annotations

import time

import numpy as np

from . import api
from . import workloads as W


def _hist(model, data, torch):
    h = torch.zeros(data.n_sets * 64, dtype=torch.float32, device="cuda")
    api.hist64(model, data, 0, h)
    return h.view(data.n_sets, 64)


def build_training_set(model, n_toys: int, seed: int, chunk: int = 4096, n_lo: float = 1e3, n_hi: float = 1e5,
                       tol_edm: float = 1e-7):
    """Generate and plain-fit `n_toys` toys; returns (hist, labels) CUDA
    tensors of the converged fits and a summary dict."""
    import torch

    xs, ys = [], []
    fitted = conv = 0
    t0 = time.perf_counter()
    for k, start in enumerate(range(0, n_toys, chunk)):
        S = min(chunk, n_toys - start)
        th = W.toy_thetas(S, seed + k)
        mean = W.toy_mean_sizes(S, seed + k, n_lo, n_hi)
        data = api.generate_toys(model, th, seed + k, mean, poisson=True)
        h = _hist(model, data, torch)
        r = api.fit(model, data, tol_edm=tol_edm, want_cov=False)
        ok = r["status"] == 0
        fitted += S
        conv += int(ok.sum())
        idx = torch.from_numpy(np.nonzero(ok)[0]).cuda()
        xs.append(h.index_select(0, idx))
        ys.append(torch.from_numpy(r["theta"][ok].astype(np.float32)).cuda())
        data.close()
    X = torch.cat(xs).contiguous()
    Y = torch.cat(ys).contiguous()
    return X, Y, {"toys": fitted, "converged": conv, "seconds": time.perf_counter() - t0}


def train(X, Y, epochs: int = 30, batch: int = 1024, lr: float = 1e-3, seed: int = 0):
    net = api.MLP(seed=seed)
    t0 = time.perf_counter()
    loss = net.train(X, Y, batch=batch, epochs=epochs, lr=lr, seed=seed + 1, standardise=True)
    return net, {"final_loss": loss, "epochs": epochs, "seconds": time.perf_counter() - t0}


def predict_starts(net, model, data):
    return net.predict(model, data, 0)


def compare(net, model, n_toys: int, seed: int, tol_edm: float = 1e-7, n_lo: float = 1e3, n_hi: float = 1e5):
    """Fit fresh toys from the plain default start and from the learned start."""
    import torch

    th = W.toy_thetas(n_toys, seed)
    mean = W.toy_mean_sizes(n_toys, seed, n_lo, n_hi)
    data = api.generate_toys(model, th, seed, mean, poisson=True)
    torch.cuda.synchronize()
    n0 = api.launch_count()
    t0 = time.perf_counter()
    plain = api.fit(model, data, tol_edm=tol_edm, want_cov=False)
    t_plain = time.perf_counter() - t0
    n1 = api.launch_count()
    t0 = time.perf_counter()
    start = predict_starts(net, model, data)
    learned = api.fit(model, data, theta0=start, tol_edm=tol_edm, want_cov=False)
    bad = np.nonzero(learned["status"] != 0)[0]
    if len(bad):
        # fallback: refit the toys whose learned start failed from the default
        # start (their own dataset), charging its time and evaluations
        off = data.offsets()
        col = data.read(0)
        parts = [col[off[s]:off[s + 1]] for s in bad]
        sub_off = np.concatenate([[0], np.cumsum([len(p) for p in parts])])
        sub = api.Data.upload(model, [np.concatenate(parts)], offsets=sub_off)
        rb = api.fit(model, sub, tol_edm=tol_edm, want_cov=False)
        for j, s in enumerate(bad):
            learned["theta"][s] = rb["theta"][j]
            learned["nll"][s] = rb["nll"][j]
            learned["status"][s] = rb["status"][j]
            learned["n_evals"][s] += rb["n_evals"][j]
    t_learned = time.perf_counter() - t0
    n2 = api.launch_count()
    both = (plain["status"] == 0) & (learned["status"] == 0)
    d = learned["nll"][both] - plain["nll"][both]
    return {
        "toys": n_toys, "events": int(data.n_events),
        "plain": {"wall_s": t_plain, "toy_fits_per_s": n_toys / t_plain,
                  "mean_evals": float(plain["n_evals"].mean()), "max_evals": int(plain["n_evals"].max()),
                  "converged": float((plain["status"] == 0).mean()), "gpu_launches": n1 - n0},
        "learned": {"wall_s": t_learned, "toy_fits_per_s": n_toys / t_learned,
                    "mean_evals": float(learned["n_evals"].mean()), "max_evals": int(learned["n_evals"].max()),
                    "converged": float((learned["status"] == 0).mean()), "fallbacks": int(len(bad)),
                    "gpu_launches": n2 - n1},
        "same_minimum_frac": float(np.mean(np.abs(d) < 1e-6)) if d.size else 0.0,
        "learned_lower_nll_frac": float(np.mean(d <= -1e-6)) if d.size else 0.0,
        "learned_higher_nll_frac": float(np.mean(d >= 1e-6)) if d.size else 0.0,
        "median_abs_dnll": float(np.median(np.abs(d))) if d.size else None,
    }
