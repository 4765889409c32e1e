"""Write oracle_nll.json: the CPU oracle's NLL and gradient on seeded datasets
drawn by the oracle's own counter-based generator; and oracle_binned.json:
the binned oracle's NLL and sampled gradient on datasets of the binned
workload's model.

Only the oracle and the input recipe (model node lists, parameter values,
seeds) are used; nothing here touches the CUDA library.  Each case stores the
generating recipe, a SHA-256 of the event columns (float64, little-endian,
column after column) so that a reader can confirm it holds the same events,
and the oracle's NLL = -sum log p_i, gradient, sum |log p_i| and
sum |dlog p_i/dtheta_k| (the scales of the parity tolerances).

    python tests/golden/make_oracle_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2003_12861_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_nll.json")


def cases():
    """(model constructor, generating theta, seed, events, evaluation points)."""
    gp_true = W.GAUSS_POLY1_TRUE
    gp_start = np.array([4.5, 1.0, 0.5, 0.0])
    d_true = W.DECAY_TRUE
    d_start = W.DECAY_START
    d_off = d_true + np.array([0.1, 0.01, -0.01, 0.05, -0.02, 0.03])
    g_true = W.DECAY_GENERIC_TRUE
    g_off = g_true + np.array([-0.1, -0.01, 0.02, -0.05, 0.02, -0.03])
    p_true = W.PROD3_TRUE
    p_off = p_true + np.array([0.002, 0.001, -0.05, 0.1, 0.1, 0.01, -0.01, 0.05, -0.02, 0.03, -0.05, 0.05])
    e_true = W.DECAY_EXTENDED_TRUE
    e_off = e_true + np.array([0.05, 0.005, 0.01, -0.03, 0.01, 0.02, -150.0])
    q_true = W.POISSON_GAUSS_TRUE
    q_off = q_true + np.array([0.4, -0.05, 0.1])
    return [
        ("gauss_poly1_model", gp_true, W.SEED_BASE + 0, 10_000, [gp_true, gp_start]),
        ("decay_extended_model", e_true, W.SEED_BASE + 1, 5_000, [e_true, e_off]),
        ("poisson_gauss_model", q_true, W.SEED_BASE + 8, 9_000, [q_true, q_off]),
        ("decay_model", d_true, W.SEED_BASE + 1, 20_000, [d_true, d_start, d_off]),
        ("decay_generic_model", g_true, W.SEED_BASE + 1, 20_000, [g_true, g_off]),
        ("prod3_model", p_true, W.SEED_BASE + 3, 12_345, [p_true, p_off]),
    ]


def columns_sha256(cols):
    h = hashlib.sha256()
    for c in cols:
        h.update(np.ascontiguousarray(c, dtype="<f8").tobytes())
    return h.hexdigest()


BINNED_OUT = os.path.join(HERE, "oracle_binned.json")
BINNED_GRAD_K = [0, 1, 2] + list(range(3, 256, 23))


def binned_cases():
    """The binned workload's model (28 channels x 50 bins, 256 parameters):
    two datasets with counts Poisson-drawn at their parameter points
    (numpy PCG64 draws of the oracle's expected counts, stored as such),
    each evaluated at its point and at the point shifted by +0.1; the NLL,
    a sample of gradient components and the tolerance scales."""
    from oracle import binned as OB

    spec = W.binned_model()
    om = OB.from_spec(spec)
    P = spec["n_params"]
    seed = W.SEED_BASE + 7
    th = W.binned_toy_thetas(2, seed, P)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    out = []
    for t in range(2):
        counts = rng.poisson(om.expected(th[t])[0]).astype(np.int64)
        evals = []
        for shift in (0.0, 0.1):
            x = th[t] + shift
            nll, g, scale = om.nll(x, counts)
            evals.append({"shift": shift, "nll": float(nll), "nll_scale": float(scale),
                          "grad": {str(k): float(g[k]) for k in BINNED_GRAD_K},
                          "grad_scale": float(np.abs(g).sum() + np.abs(counts).sum() + 1.0)})
        out.append({"theta_recipe": f"workloads.binned_toy_thetas(2, {seed}, {P})[{t}] + shift",
                    "counts": " ".join(str(int(c)) for c in counts), "evaluations": evals})
    return {"source": "written by tests/golden/make_oracle_golden.py from the CPU oracle alone",
            "model": "workloads.binned_model()", "theta_seed": seed, "cases": out}


def main():
    oracle.build()
    with open(BINNED_OUT, "w") as f:
        json.dump(binned_cases(), f)
        f.write("\n")
    out = []
    for which, gen_theta, seed, n, points in cases():
        spec = W.model_for(which)
        om = oracle.Model(spec.nodes, spec.root)
        cols = om.generate(gen_theta, seed, 0, 0, n)
        evals = []
        for th in points:
            nll, g, al, ag, rc = om.nll(th, cols)
            if rc != 0:
                raise RuntimeError(f"{which}: oracle status {rc}")
            evals.append({"theta": [float(v) for v in th], "nll": nll, "grad": [float(v) for v in g],
                          "sum_abs_logp": al, "sum_abs_grad": [float(v) for v in ag]})
        out.append({"model": which, "generate_theta": [float(v) for v in gen_theta], "seed": seed, "set": 0,
                    "events": n, "columns_sha256": columns_sha256(cols), "evaluations": evals})
    doc = {"source": "written by tests/golden/make_oracle_golden.py from the CPU oracle alone",
           "cases": out}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(f"wrote {OUT}: {len(out)} datasets")


if __name__ == "__main__":
    main()
