"""Shared test helpers: datasets from the oracle's generator, tolerance checks."""
from paper_2003_12861_gb300 import workloads as W

TRUE = {"gauss_poly1_model": W.GAUSS_POLY1_TRUE, "decay_model": W.DECAY_TRUE, "prod3_model": W.PROD3_TRUE}

# Tolerances: NLL within 1e-12 of sum|log p|; gradient component k within
# 1e-9 of sum_i |dlog p_i/dtheta_k| (a minimum makes the gradient itself ~0).
NLL_RTOL = 1e-12
GRAD_RTOL = 1e-9


def oracle_data(oracle_mod, which, n, seed=1234, set_index=0, theta=None):
    spec = W.model_for(which)
    om = oracle_mod.Model(spec.nodes, spec.root)
    th = TRUE[which] if theta is None else theta
    cols = om.generate(th, seed, set_index, 0, n)
    return spec, om, cols


def check_nll(gpu_nll, gpu_grad, ref, what=""):
    nll, g, al, ag, rc = ref
    assert abs(gpu_nll - nll) <= NLL_RTOL * max(al, 1e-300), (what, gpu_nll, nll, al)
    if gpu_grad is not None:
        for k in range(len(g)):
            assert abs(gpu_grad[k] - g[k]) <= GRAD_RTOL * max(ag[k], 1e-300), (what, k, gpu_grad[k], g[k], ag[k])
