"""Learned fit start: build the training set with the method itself, train the
network, and compare learned-start fits with plain-start fits.

Orchestration only: toys are generated (rf_generate_toys), histogrammed
(rf_hist64) and fitted (rf_fit) by the library, the network is trained and
evaluated by its kernels (rf_mlp_*); PyTorch holds the device buffers.

Training toys have generating parameters drawn uniformly within +-30 % of
the decay model's values.  Each is fitted twice, from the plain default start
and from its generating parameters, and its label is the fitted point
(theta-hat) of the lower of the two minima: small toys of this model have
several local minima (a resolution parameter or the signal fraction on a
bound against an interior minimum), and the network should point at the
deeper one.  Its predictions start the fits at least 5 % of each bounded
parameter's range inside the bounds (rf_mlp_predict: at a bound the fit's
bound transform is stationary).  The plain fit from the default start is also the fallback and
the yardstick: a learned start that fails (outside the domain, or no
convergence) is refitted from the default start, and a learned fit that ends
in a different minimum (|delta NLL| >= 1e-6) is counted and reported, higher
and lower separately.  As a reference for how often each start finds the
deepest minimum known, the toys are also fitted from their generating
values (untimed): the fraction of toys where each start reaches the lowest
of the three minima is reported beside.
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
    """Generate `n_toys` toys and fit each from the default start and from
    its generating parameters; returns (hist, labels) CUDA tensors of the
    toys with a converged fit (labels: the deeper minimum) and a summary."""
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
        rt = api.fit(model, data, theta0=th, tol_edm=tol_edm, want_cov=False)
        # the deeper of the two minima (a fit that did not converge loses)
        nll_p = np.where(r["status"] == 0, r["nll"], np.inf)
        nll_t = np.where(rt["status"] == 0, rt["nll"], np.inf)
        use_t = nll_t < nll_p
        r["theta"][use_t] = rt["theta"][use_t]
        r["status"][use_t] = 0
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


def compare(net, model, n_toys: int, seed: int, tol_edm: float = 1e-9, n_lo: float = 1e3, n_hi: float = 1e5,
            characterise: bool = False):
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
        # start, charging its time and evaluations
        rb = api.fit_sets(model, data, bad, tol_edm=tol_edm)
        for j, s in enumerate(bad):
            learned["theta"][s] = rb["theta"][j]
            learned["nll"][s] = rb["nll"][j]
            learned["status"][s] = rb["status"][j]
            learned["n_evals"][s] += rb["n_evals"][j]
    t_learned = time.perf_counter() - t0
    n2 = api.launch_count()
    both = (plain["status"] == 0) & (learned["status"] == 0)
    d = learned["nll"][both] - plain["nll"][both]
    mismatch = _characterise(model, data, plain, learned, both) if characterise else None
    # reference, untimed: the fit from each toy's generating values
    truth = api.fit(model, data, theta0=th, tol_edm=tol_edm, want_cov=False)
    inf = np.inf
    best = np.minimum(np.minimum(np.where(plain["status"] == 0, plain["nll"], inf),
                                 np.where(learned["status"] == 0, learned["nll"], inf)),
                      np.where(truth["status"] == 0, truth["nll"], inf))
    at_best = {name: float(np.mean((r["status"] == 0) & (r["nll"] - best < 1e-6)))
               for name, r in (("plain", plain), ("learned", learned), ("generating_values", truth))}
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
        "tol_edm": tol_edm,
        "at_lowest_of_three_minima_frac": at_best,
        "mismatch": mismatch,
    }


def _characterise(model, data, plain, learned, both):
    """The toys whose two fits end in different minima: refitted from each
    end point with a tight tolerance (EDM < 1e-11), a pair that then agrees
    was a stop short of one minimum; the others are distinct minima.  Also
    how many have a parameter within 1e-3 of its range at either end point."""
    spec_lo = np.array(model_bounds(model)[0])
    spec_hi = np.array(model_bounds(model)[1])
    off = data.offsets()
    col = data.read(0)
    d = learned["nll"] - plain["nll"]
    out = {}
    for name, sel in (("learned_higher", both & (d >= 1e-6)), ("learned_lower", both & (d <= -1e-6))):
        idx = np.nonzero(sel)[0]
        if len(idx) == 0:
            out[name] = {"count": 0}
            continue
        parts = [col[off[s]:off[s + 1]] for s in idx]
        sub = api.Data.upload(model, [np.concatenate(parts)], offsets=np.concatenate([[0], np.cumsum([len(p) for p in parts])]))
        rl = api.fit(model, sub, theta0=learned["theta"][idx], tol_edm=1e-11, want_cov=False)
        rp = api.fit(model, sub, theta0=plain["theta"][idx], tol_edm=1e-11, want_cov=False)
        span = spec_hi - spec_lo
        near = [np.any(np.minimum(t - spec_lo, spec_hi - t) < 1e-3 * span) or
                np.any(np.minimum(u - spec_lo, spec_hi - u) < 1e-3 * span)
                for t, u in zip(learned["theta"][idx], plain["theta"][idx])]
        out[name] = {"count": int(len(idx)), "resolved_by_tight_refit": float(np.mean(np.abs(rl["nll"] - rp["nll"]) < 1e-6)),
                     "near_a_bound": float(np.mean(near)), "median_abs_dnll": float(np.median(np.abs(d[idx]))),
                     "median_events": float(np.median(np.diff(off)[idx]))}
    return out


def model_bounds(model):
    nodes = [n for n in model.nodes if n.kind == "param" and n.free]
    return [n.lo for n in nodes], [n.hi for n in nodes]
