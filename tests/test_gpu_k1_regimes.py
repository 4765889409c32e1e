"""K1's parameter point for the decay model in every regime of its
normalisation: the range's Gaussian mass from erf (range around the
resolution mean), from erfc on either side (mean below or above the range),
vanishing (range far from the mean), and ranges narrow against the
resolution or the lifetime.  Each takes the float-float path or, where its
guards decline, the FP64 path; NLL and gradient agree with the oracle.

Where the range lies far from the resolution mean, the derivatives with
respect to mu_r and sigma_r cancel to almost nothing between the density's
and the normalisation's terms (1/tau against dlogI/dmu).  The oracle's own
per-event values then carry that cancellation's error, so those components
are compared with an absolute floor of 1e-12 of the largest component's
scale (sum_i |dlog p_i/dtheta_j|) on top of the usual 1e-9 of their own."""
import numpy as np
import pytest

from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

from helpers import GRAD_RTOL, NLL_RTOL

pytestmark = pytest.mark.gpu


def decay_spec(lo, hi):
    b = W._Builder()
    t = b.obs(lo, hi)
    tau = b.param("tau", 1.5, 0.1, 10.0)
    mur = b.param("mu_r", 0.0, -20.0, 20.0)
    sgr = b.param("sigma_r", 0.05, 0.005, 5.0)
    c1 = b.param("c1", -0.2, -1.0, 1.0)
    c2 = b.param("c2", 0.05, -1.0, 1.0)
    fs = b.param("f_sig", 0.2, 0.0, 1.0)
    sig = b.pdf("gaussexp", t, tau, mur, sgr)
    bkg = b.pdf("cheb", t, c1, c2)
    return b.spec(b.pdf("sum", sig, bkg, fs))


CASES = [
    # (lo, hi, generating theta, evaluation theta)
    (0.0, 10.0, [1.5, 0.3, 0.05, -0.2, 0.05, 0.3], [1.4, 0.3, 0.06, -0.1, 0.0, 0.25]),    # erf: mean inside
    (0.0, 10.0, [1.5, -0.3, 0.05, -0.2, 0.05, 0.3], [1.6, -0.25, 0.05, -0.2, 0.1, 0.3]),  # erfc, mean below
    (0.0, 10.0, [1.5, 10.2, 0.05, -0.2, 0.05, 0.3], [1.5, 10.1, 0.08, -0.2, 0.05, 0.3]),  # erfc, mean above
    (4.0, 4.5, [1.5, 0.0, 0.05, -0.2, 0.05, 0.5], [1.3, 0.0, 0.05, -0.1, 0.05, 0.4]),     # no Gaussian mass
    (0.0, 0.2, [1.5, 0.1, 0.3, -0.2, 0.05, 0.5], [2.0, 0.08, 0.35, -0.1, 0.05, 0.45]),    # range << sigma
    (0.0, 10.0, [0.12, 0.0, 0.8, -0.2, 0.05, 0.5], [0.15, 0.1, 0.7, -0.1, 0.05, 0.5]),    # sigma >> tau
    (0.0, 3.0, [8.0, 0.5, 0.2, -0.2, 0.05, 0.5], [7.0, 0.4, 0.25, -0.1, 0.05, 0.5]),      # tau >> range
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_k1_regimes_match_oracle(oracle_mod, case):
    lo, hi, th_gen, th_eval = CASES[case]
    spec = decay_spec(lo, hi)
    om = oracle_mod.Model(spec.nodes, spec.root)
    cols = om.generate(np.array(th_gen), 40 + case, 0, 0, 12000)
    m = api.Model.from_spec(spec)
    assert "kernel=ff_" in m.describe()
    d = api.Data.upload(m, cols)
    for th in (np.array(th_gen), np.array(th_eval)):
        nll, g = api.nll_grad(m, d, th)
        ref_nll, ref_g, al, ag, _ = om.nll(th, cols)
        assert abs(nll - ref_nll) <= NLL_RTOL * al, (case, nll, ref_nll)
        floor = 1e-12 * max(ag)
        for k in range(len(g)):
            assert abs(g[k] - ref_g[k]) <= GRAD_RTOL * ag[k] + floor, (case, k, g[k], ref_g[k], ag[k])
