"""Seeded synthetic workloads: model node lists and the random inputs drawn
outside the method.

This module holds data only -- node lists, constants and numpy draws of the
quantities the method takes as inputs (per-toy mean sizes, per-toy generating
parameters, seeds).  It holds none of the method's arithmetic (no pdf, no
normalisation, no likelihood), so both the CUDA path and the CPU oracle may
consume it.

A model is a list of ``Node`` plus the index of its top pdf.  This mirrors the
paper's computation graph (Sec. 1, Fig. 1): observables and parameters are
leaves; functions/PDFs take them as inputs.  Input conventions per kind:

=========  ==========================================================
obs        no inputs; ``lo``/``hi`` = observable range; column = order of obs nodes
param      no inputs; ``value`` = default start, ``lo``/``hi`` = fit bounds
gauss      [obs, mu, sigma]
exp        [obs, c]                       (exp(c x))
gaussexp   [obs, tau, mu, sigma]          (decay (x) Gaussian resolution)
cheb       [obs, c1, ..., cn]             (1 + sum c_k T_k, implicit c0 = 1)
poly       [obs, a1, ..., an]             (1 + sum a_k x^k, implicit a0 = 1)
sum        [pdf_1..pdf_n, f_1..f_{n-1}]   (last fraction = 1 - sum f)
prod       [pdf_1..pdf_n]                 (disjoint observables)
poisson    [obs, lambda]                  (count k = floor(x); integer range)
extend     [pdf, nu]                      (root only: extended likelihood)
expr       [obs, p_1, ..., p_n]           (a density given as a postfix program,
                                           ``prog`` / ``consts``; see expr_program)
=========  ==========================================================

The five workloads (sizes, true values and ranges) are the ones the
benchmark configurations name; constants the configurations leave open
(fit bounds, default starts, the product model's mass and angle shapes) are
fixed here once.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

KINDS = ("obs", "param", "gauss", "exp", "gaussexp", "cheb", "poly", "sum", "prod", "poisson", "extend", "expr")


@dataclass(frozen=True)
class Node:
    kind: str
    inputs: Sequence[int] = ()
    value: float = 0.0
    lo: float = 0.0
    hi: float = 0.0
    free: bool = False
    prog: Tuple[int, ...] = ()       # expr: the program's operations
    consts: Tuple[float, ...] = ()   # expr: its constants


# The program format of an expr node: one int per operation, code | (arg <<
# 8), evaluated on a stack.  x pushes the observable, p<j> the node's j-th
# parameter (input 1 + j), c<j> constant j; + - * / and pow pop two values
# (a then b, pushing a op b, pow = a^b with a > 0), neg, exp and log pop one.
EXPR_CODES = {"x": 0, "p": 1, "c": 2, "+": 3, "-": 4, "*": 5, "/": 6, "neg": 7, "exp": 8, "log": 9, "pow": 10}


def expr_program(text: str) -> Tuple[int, ...]:
    """Encode a whitespace-separated postfix program, e.g. "x p0 - p1 /"."""
    ops = []
    for tok in text.split():
        if tok[0] in "pc" and tok[1:].isdigit():
            ops.append(EXPR_CODES[tok[0]] | (int(tok[1:]) << 8))
        else:
            ops.append(EXPR_CODES[tok])
    return tuple(ops)


@dataclass
class ModelSpec:
    nodes: List[Node]
    root: int
    names: List[str] = field(default_factory=list)  # free-parameter names, theta order

    @property
    def n_free(self) -> int:
        return sum(1 for n in self.nodes if n.kind == "param" and n.free)

    @property
    def n_obs(self) -> int:
        return sum(1 for n in self.nodes if n.kind == "obs")

    def defaults(self) -> np.ndarray:
        return np.array([n.value for n in self.nodes if n.kind == "param" and n.free], dtype=np.float64)

    def bounds(self) -> np.ndarray:
        return np.array([[n.lo, n.hi] for n in self.nodes if n.kind == "param" and n.free], dtype=np.float64)


class _Builder:
    def __init__(self):
        self.nodes: List[Node] = []
        self.names: List[str] = []

    def add(self, node: Node, name: str | None = None) -> int:
        self.nodes.append(node)
        if node.kind == "param" and node.free:
            self.names.append(name or f"p{len(self.names)}")
        return len(self.nodes) - 1

    def obs(self, lo, hi):
        return self.add(Node("obs", (), 0.0, lo, hi))

    def param(self, name, value, lo, hi, free=True):
        return self.add(Node("param", (), value, lo, hi, free), name)

    def pdf(self, kind, *inputs):
        return self.add(Node(kind, tuple(inputs)))

    def expr(self, text, consts, *inputs):
        return self.add(Node("expr", tuple(inputs), prog=expr_program(text), consts=tuple(consts)))

    def spec(self, root):
        return ModelSpec(self.nodes, root, self.names)


# ------------------------------------------------------------------ models

def gauss_poly1_model() -> ModelSpec:
    """1-D f*Gauss(x; mu, sigma) + (1-f)*Poly1(x; a1) on x in [0, 10].
    Parameter defaults are the fit start (mu=4.5, sigma=1, f=0.5, a1=0)."""
    b = _Builder()
    x = b.obs(0.0, 10.0)
    mu = b.param("mu", 4.5, 0.0, 10.0)
    sg = b.param("sigma", 1.0, 0.01, 10.0)
    f = b.param("f", 0.5, 0.0, 1.0)
    a1 = b.param("a1", 0.0, -0.1, 1.0)
    g = b.pdf("gauss", x, mu, sg)
    p = b.pdf("poly", x, a1)
    return b.spec(b.pdf("sum", g, p, f))


GAUSS_POLY1_TRUE = np.array([5.0, 0.5, 0.3, -0.05])


def _decay_part(b: _Builder, t: int, start: Sequence[float]):
    tau = b.param("tau", start[0], 0.1, 10.0)
    mur = b.param("mu_r", start[1], -0.5, 0.5)
    sgr = b.param("sigma_r", start[2], 0.005, 1.0)
    c1 = b.param("c1", start[3], -1.0, 1.0)
    c2 = b.param("c2", start[4], -1.0, 1.0)
    fs = b.param("f_sig", start[5], 0.0, 1.0)
    sig = b.pdf("gaussexp", t, tau, mur, sgr)
    bkg = b.pdf("cheb", t, c1, c2)
    return b.pdf("sum", sig, bkg, fs)


DECAY_TRUE = np.array([1.5, 0.0, 0.05, -0.2, 0.05, 0.2])
DECAY_START = np.array([1.0, 0.0, 0.1, 0.0, 0.0, 0.5])


def decay_model() -> ModelSpec:
    """Decay-time model on t in [0, 10]: f_sig * [exp(-t/tau) (x) Gauss(mu_r, sigma_r)]
    + (1 - f_sig) * Chebychev2(c1, c2).  Defaults are the plain fit start."""
    b = _Builder()
    t = b.obs(0.0, 10.0)
    return b.spec(_decay_part(b, t, DECAY_START))


def decay_generic_model() -> ModelSpec:
    """The decay model with the SUM operands in the other order (background
    first, f_bkg = 1 - f_sig): the same density, matched by no float-float
    program, so it runs on the generic FP64 interpreter.  Defaults are the
    generating values of DECAY_GENERIC_TRUE."""
    b = _Builder()
    t = b.obs(0.0, 10.0)
    tau = b.param("tau", DECAY_TRUE[0], 0.1, 10.0)
    mur = b.param("mu_r", DECAY_TRUE[1], -0.5, 0.5)
    sgr = b.param("sigma_r", DECAY_TRUE[2], 0.005, 1.0)
    c1 = b.param("c1", DECAY_TRUE[3], -1.0, 1.0)
    c2 = b.param("c2", DECAY_TRUE[4], -1.0, 1.0)
    fb = b.param("f_bkg", 1.0 - DECAY_TRUE[5], 0.0, 1.0)
    sig = b.pdf("gaussexp", t, tau, mur, sgr)
    bkg = b.pdf("cheb", t, c1, c2)
    return b.spec(b.pdf("sum", bkg, sig, fb))


DECAY_GENERIC_TRUE = np.array([*DECAY_TRUE[:5], 1.0 - DECAY_TRUE[5]])

PROD3_TRUE = np.array([5.28, 0.015, 0.4, -0.3, *DECAY_TRUE, 0.1, 0.3])


def prod3_model() -> ModelSpec:
    """3-observable product: [mass m in [5.2,5.4]: f_m Gauss + (1-f_m) Chebychev1]
    x [decay time t in [0,10]: the decay model] x [cos(theta) in [-1,1]: Poly2].
    12 free parameters; defaults are the generating values."""
    b = _Builder()
    m = b.obs(5.2, 5.4)
    t = b.obs(0.0, 10.0)
    c = b.obs(-1.0, 1.0)
    mum = b.param("mu_m", 5.28, 5.2, 5.4)
    sgm = b.param("sigma_m", 0.015, 0.001, 0.1)
    fm = b.param("f_m", 0.4, 0.0, 1.0)
    cm = b.param("c_m", -0.3, -1.0, 1.0)
    gm = b.pdf("gauss", m, mum, sgm)
    bm = b.pdf("cheb", m, cm)
    mass = b.pdf("sum", gm, bm, fm)
    decay = _decay_part(b, t, DECAY_TRUE)
    a1 = b.param("a1", 0.1, -1.0, 1.0)
    a2 = b.param("a2", 0.3, -1.0, 1.0)
    ang = b.pdf("poly", c, a1, a2)
    return b.spec(b.pdf("prod", mass, decay, ang))


def decay_extended_model() -> ModelSpec:
    """The decay model under an extended root: + nu - N log nu with a free
    yield nu (start 5000), the decay parameters first, nu last."""
    spec = decay_model()
    nodes = list(spec.nodes) + [Node("param", (), 5000.0, 1.0, 1e8, True)]
    nodes.append(Node("extend", (spec.root, len(nodes) - 1)))
    return ModelSpec(nodes, len(nodes) - 1, list(spec.names) + ["nu"])


DECAY_EXTENDED_TRUE = np.array([*DECAY_TRUE, 5000.0])


def poisson_gauss_model() -> ModelSpec:
    """Poisson(k; lambda) on k in [0, 30) times Gauss(y; mu, sigma) on
    [-5, 5]: the batched Poisson leaf beside a continuous factor."""
    b = _Builder()
    k = b.obs(0.0, 30.0)
    y = b.obs(-5.0, 5.0)
    lam = b.param("lambda", 7.0, 0.1, 50.0)
    mu = b.param("mu", 0.2, -3.0, 3.0)
    sg = b.param("sigma", 1.1, 0.1, 5.0)
    return b.spec(b.pdf("prod", b.pdf("poisson", k, lam), b.pdf("gauss", y, mu, sg)))


POISSON_GAUSS_TRUE = np.array([7.0, 0.2, 1.1])


def expr_gauss_poly1_model() -> ModelSpec:
    """gauss_poly1_model with its Gaussian written as an expr node,
    exp(-((x - mu)/sigma)^2 / 2): the same density through the generic
    program path and a numerical normalisation."""
    b = _Builder()
    x = b.obs(0.0, 10.0)
    mu = b.param("mu", 4.5, 0.0, 10.0)
    sg = b.param("sigma", 1.0, 0.01, 10.0)
    f = b.param("f", 0.5, 0.0, 1.0)
    a1 = b.param("a1", 0.0, -0.1, 1.0)
    g = b.expr("x p0 - p1 / x p0 - p1 / * c0 * exp", (-0.5,), x, mu, sg)
    p = b.pdf("poly", x, a1)
    return b.spec(b.pdf("sum", g, p, f))


def expr_mix_model() -> ModelSpec:
    """Programs beside built-in nodes: [mass m in [5.2, 5.4]: f * Cauchy(m;
    m0, gamma) + (1 - f) * Chebychev1] x [t in [0.2, 5]: t^a exp(-b t)], the
    Cauchy line shape 1/((m - m0)^2 + gamma^2) and the gamma-like t density
    as expr nodes.  6 free parameters; defaults are the generating values."""
    b = _Builder()
    m = b.obs(5.2, 5.4)
    t = b.obs(0.2, 5.0)
    m0 = b.param("m0", 5.28, 5.2, 5.4)
    gam = b.param("gamma", 0.012, 0.001, 0.1)
    fm = b.param("f_m", 0.45, 0.0, 1.0)
    cm = b.param("c_m", -0.2, -1.0, 1.0)
    a = b.param("a", 1.5, 0.0, 5.0)
    bb = b.param("b", 1.2, 0.1, 5.0)
    line = b.expr("c0 x p0 - x p0 - * p1 p1 * + /", (1.0,), m, m0, gam)
    bkg = b.pdf("cheb", m, cm)
    mass = b.pdf("sum", line, bkg, fm)
    tt = b.expr("x p0 pow x p1 * neg exp *", (), t, a, bb)
    return b.spec(b.pdf("prod", mass, tt))


EXPR_MIX_TRUE = np.array([5.28, 0.012, 0.45, -0.2, 1.5, 1.2])


# ------------------------------------------------------------------ configs

SEED_BASE = 20031286


@dataclass(frozen=True)
class Workload:
    name: str
    model: str            # constructor name above
    n_events: int         # per set (single-set workloads) or 0 for toy batches
    n_sets: int
    seed: int
    f32_columns: bool = False


WORKLOADS = {
    "gauss_poly1_1e4": Workload("gauss_poly1_1e4", "gauss_poly1_model", 10_000, 1, SEED_BASE + 0),
    "decay_1e7": Workload("decay_1e7", "decay_model", 10_000_000, 1, SEED_BASE + 1),
    "decay_toys_4096": Workload("decay_toys_4096", "decay_model", 0, 4096, SEED_BASE + 2),
    "prod3_1e8_f32": Workload("prod3_1e8_f32", "prod3_model", 100_000_000, 1, SEED_BASE + 3, True),
    "learned_start": Workload("learned_start", "decay_model", 0, 10_000, SEED_BASE + 4),
}


def model_for(name: str) -> ModelSpec:
    return globals()[name]()


def toy_mean_sizes(n_sets: int, seed: int, lo: float = 1e3, hi: float = 1e5) -> np.ndarray:
    """Per-toy mean event counts, log-uniform in [lo, hi] (numpy PCG64 stream)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(n_sets)
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))


def toy_thetas(n_sets: int, seed: int, center: np.ndarray = DECAY_TRUE, rel: float = 0.3,
               abs_width: np.ndarray | None = None) -> np.ndarray:
    """Per-toy generating parameters drawn uniformly within +-rel of `center`.
    Where a centre is 0 the half-width is taken from `abs_width` instead
    (for the decay model mu_r = 0 uses +-0.3 sigma_r = +-0.015)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    center = np.asarray(center, dtype=np.float64)
    half = np.abs(center) * rel
    if abs_width is None:
        abs_width = np.where(center == 0.0, 0.015, 0.0)
    half = np.where(center == 0.0, abs_width, half)
    u = rng.random((n_sets, center.size))
    return center + (2.0 * u - 1.0) * half


# ---------------------------------------------------- binned (HistFactory)

def binned_model(seed: int = 20031290, channels: int = 28, bins: int = 50, samples: int = 8,
                 nuisances: int = 253, histosys_per_sample: int = 20, normsys_per_sample: int = 10):
    """A synthetic HistFactory-style model of the size the paper's ATLAS
    example has (28 channels, 253 systematics, ~1e4 histograms): per channel
    `samples` nominal histograms of `bins` bins (smooth random shapes),
    each sample with normsys (kappa_lo, kappa_hi) and histosys (h_lo, h_hi)
    modifiers on nuisances drawn from a shared pool, and 3 free normalisation
    factors (a signal strength on sample 0 of every channel, two background
    scales on samples 1 and 2).  Returned as plain data:
    dict(n_bins, bin0[S], nominal[S][bins], constrained[P], modifiers=list of
    (sample, kind, param, k_lo, k_hi, h_lo, h_hi)), kind 0/1/2 =
    normfactor/normsys/histosys; parameters 0..2 are the normfactors, 3.. the
    constrained nuisances."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_bins = channels * bins
    bin0, nominal, mods = [], [], []
    x = (np.arange(bins) + 0.5) / bins
    P = 3 + nuisances
    for c in range(channels):
        for j in range(samples):
            s = len(nominal)
            amp = 10 ** rng.uniform(0.5, 3.0)
            if j == 0:  # a signal bump
                mu0, w = rng.uniform(0.3, 0.7), rng.uniform(0.05, 0.15)
                h = amp * np.exp(-0.5 * ((x - mu0) / w) ** 2) + 1e-3 * amp
            else:       # falling backgrounds
                h = amp * np.exp(-x * rng.uniform(0.5, 4.0)) * (1 + 0.2 * np.sin(6.28 * x * rng.uniform(0.5, 2)))
            bin0.append(c * bins)
            nominal.append(h)
            if j < 3:
                mods.append((s, 0, j, 1.0, 1.0, None, None))
            for k in rng.choice(nuisances, normsys_per_sample, replace=False):
                mods.append((s, 1, 3 + int(k), float(rng.uniform(0.85, 0.99)), float(rng.uniform(1.01, 1.15)),
                             None, None))
            for k in rng.choice(nuisances, histosys_per_sample, replace=False):
                tilt = rng.uniform(-0.05, 0.05) * (x - 0.5) + rng.uniform(-0.02, 0.02)
                mods.append((s, 2, 3 + int(k), 1.0, 1.0, h * (1 - tilt - rng.uniform(0, 0.01)),
                             h * (1 + tilt + rng.uniform(0, 0.01))))
    constrained = [False] * 3 + [True] * nuisances
    return {"n_bins": n_bins, "bin0": bin0, "nominal": nominal, "constrained": constrained, "modifiers": mods,
            "n_params": P}


def binned_toy_thetas(n_toys: int, seed: int, n_params: int) -> np.ndarray:
    """Per-toy parameter points: normfactors uniform in [0.8, 1.2], nuisances
    standard normal x 0.5."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = rng.normal(0.0, 0.5, (n_toys, n_params))
    th[:, :3] = rng.uniform(0.8, 1.2, (n_toys, 3))
    return th
