"""Oracle for the binned (HistFactory-style) likelihood.

TEST INFRASTRUCTURE ONLY: a plain, slow restatement of what the library's
binned kernels compute, for the tests, the package's smoke check and the
benchmark's CPU baseline.  It shares no code with the CUDA library.

The paper builds binned models from histograms (Sec. 3: HistFactory,
channels of samples with +-1 sigma systematic histograms).  Definitions:

* samples s with nominal rates h_s[i] on the contiguous bins b0_s + i;
* modifiers of a sample, each tied to one parameter theta_k:
    normfactor  nu *= theta_k
    normsys     nu *= eta(alpha) = exp(a alpha + b g(alpha)),
                a = (log k_hi - log k_lo)/2, b = (log k_hi + log k_lo)/2
    histosys    nu += delta(alpha) = a_i alpha + b_i g(alpha) bin by bin,
                a_i = (h_hi - h_lo)/2, b_i = (h_hi + h_lo)/2 - h; the
                factors multiply the sum
  with g(alpha) = alpha^2 for |alpha| <= 1 and 2|alpha| - 1 beyond: the
  variation is quadratic inside +-1 sigma and linear outside (in log for
  normsys), continuous with a continuous first derivative, and reaches
  k_hi, k_lo and h_hi, h_lo at alpha = +1, -1
  so nu_s[i] = prod(normfactors) prod(eta) (h_s[i] + sum delta_m[i]);
* expected count of bin b: nu_b = sum of nu_s over the samples on b;
* NLL(theta) = sum_b (nu_b - n_b log nu_b) + sum over constrained
  parameters of theta_k^2 / 2 (the Poisson terms without log n_b!, the
  unit-Gaussian constraints without their normalisation).

Everything below is a direct loop over bins, samples and modifiers in float64;
the gradient is the analytic derivative of the same expressions.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

NORMFACTOR, NORMSYS, HISTOSYS = 0, 1, 2


def interp_g(alpha: float):
    """g(alpha) = alpha^2 inside +-1, 2|alpha| - 1 outside, and g'(alpha)."""
    if abs(alpha) <= 1.0:
        return alpha * alpha, 2.0 * alpha
    return 2.0 * abs(alpha) - 1.0, 2.0 if alpha > 0 else -2.0


@dataclass
class Modifier:
    sample: int
    kind: int
    param: int
    k_lo: float = 1.0
    k_hi: float = 1.0
    h_lo: np.ndarray | None = None
    h_hi: np.ndarray | None = None


@dataclass
class BinnedModel:
    n_bins: int
    bin0: List[int]                  # per sample
    nominal: List[np.ndarray]        # per sample
    constrained: List[bool]          # per parameter
    modifiers: List[Modifier] = field(default_factory=list)

    @property
    def n_params(self) -> int:
        return len(self.constrained)

    def sample_rates(self, theta):
        """nu_s[i] per sample and its derivatives d nu_s[i] / d theta_k
        (list of (n_i, P) arrays)."""
        P = self.n_params
        out, dout = [], []
        for s, h in enumerate(self.nominal):
            h = np.asarray(h, dtype=np.float64)
            shape = h.copy()                      # h + sum delta
            dshape = np.zeros((len(h), P))
            factor = 1.0
            dlogf = np.zeros(P)
            for m in self.modifiers:
                if m.sample != s:
                    continue
                al = float(theta[m.param])
                g, dg = interp_g(al)
                if m.kind == NORMFACTOR:
                    factor *= al
                    dlogf[m.param] += 1.0 / al
                elif m.kind == NORMSYS:
                    a = 0.5 * (np.log(m.k_hi) - np.log(m.k_lo))
                    b = 0.5 * (np.log(m.k_hi) + np.log(m.k_lo))
                    factor *= np.exp(a * al + b * g)
                    dlogf[m.param] += a + b * dg
                else:  # HISTOSYS
                    a = 0.5 * (np.asarray(m.h_hi) - np.asarray(m.h_lo))
                    b = 0.5 * (np.asarray(m.h_hi) + np.asarray(m.h_lo)) - h
                    shape += a * al + b * g
                    dshape[:, m.param] += a + b * dg
            nu = factor * shape
            dnu = factor * dshape + nu[:, None] * dlogf[None, :]
            out.append(nu)
            dout.append(dnu)
        return out, dout

    def expected(self, theta):
        nus, dnus = self.sample_rates(theta)
        nu = np.zeros(self.n_bins)
        dnu = np.zeros((self.n_bins, self.n_params))
        for s, (v, dv) in enumerate(zip(nus, dnus)):
            b0 = self.bin0[s]
            for i in range(len(v)):           # bin by bin, samples in order
                nu[b0 + i] += v[i]
                dnu[b0 + i] += dv[i]
        return nu, dnu

    def nll(self, theta, counts):
        """(nll, grad, sum |terms|) for one dataset of bin counts; +inf if
        some expected count is not positive."""
        theta = np.asarray(theta, dtype=np.float64)
        n = np.asarray(counts, dtype=np.float64)
        nu, dnu = self.expected(theta)
        if np.any(~(nu > 0)):
            return np.inf, np.full(self.n_params, np.nan), np.inf
        terms = nu - n * np.log(nu)
        w = 1.0 - n / nu
        grad = w @ dnu
        cons = np.asarray(self.constrained, dtype=bool)
        nll = terms.sum() + 0.5 * np.sum(theta[cons] ** 2)
        grad = grad + np.where(cons, theta, 0.0)
        scale = np.abs(terms).sum() + 0.5 * np.sum(theta[cons] ** 2)
        return nll, grad, scale


def from_spec(spec) -> BinnedModel:
    """The oracle's model from workloads.binned_model's plain data."""
    mods = [Modifier(s, k, p, klo, khi, None if lo is None else np.asarray(lo), None if hi is None else np.asarray(hi))
            for (s, k, p, klo, khi, lo, hi) in spec["modifiers"]]
    return BinnedModel(spec["n_bins"], list(spec["bin0"]), [np.asarray(h) for h in spec["nominal"]],
                       list(spec["constrained"]), mods)
