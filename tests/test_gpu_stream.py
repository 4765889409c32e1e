"""rf_nll_grad_stream: events from host memory, copies overlapping the pass.
Same results as the device-resident pass and the oracle, for one large set
(many segments), ragged multi-set data, FP32 columns, and consecutive calls
with different host contents."""
import numpy as np
import pytest
import torch

from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W

from helpers import TRUE, check_nll

pytestmark = pytest.mark.gpu


def _pinned(a, dtype):
    t = torch.empty(len(a), dtype=dtype, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


@pytest.mark.parametrize("which,n", [("decay_model", 40 * 4096 * 16 + 999), ("prod3_model", 3 * 4096 + 5)])
def test_stream_matches_device_pass_and_oracle(oracle_mod, which, n):
    spec = W.model_for(which)
    om = oracle_mod.Model(spec.nodes, spec.root)
    th = np.array(TRUE[which]) * 1.01
    cols = om.generate(TRUE[which], 17, 0, 0, n)
    m = api.Model.from_spec(spec)
    d_ref = api.Data.upload(m, cols)
    ref = api.nll_grad(m, d_ref, th)
    host = [_pinned(c, torch.float64) for c in cols]
    d = api.Data.upload(m, [np.zeros(n)] * spec.n_obs)  # same layout, other contents
    got = api.nll_grad_stream(m, d, host, th)
    assert got[0] == ref[0] and np.array_equal(got[1], ref[1])  # same tree, same bits
    if n < 100_000:
        check_nll(got[0], got[1], om.nll(th, cols), which)
    # numpy (pageable) host memory works too
    got2 = api.nll_grad_stream(m, d, [np.ascontiguousarray(c) for c in cols], th)
    assert got2[0] == ref[0]


def test_stream_ragged_sets_f32_and_refills(oracle_mod):
    spec = W.decay_model()
    om = oracle_mod.Model(spec.nodes, spec.root)
    sizes = [0, 700_000, 1, 0, 600_000, 4097, 333_333]  # 4 segments
    off = np.concatenate([[0], np.cumsum(sizes)])
    m = api.Model.from_spec(spec)
    d = api.Data.upload(m, [np.zeros(off[-1], dtype=np.float32)], offsets=off, f32=[True])
    th = np.tile(TRUE["decay_model"], (len(sizes), 1))
    for seed in (3, 4):  # two batches through the same dataset
        parts = [om.generate(TRUE["decay_model"], seed, s, 0, n)[0] if n else np.zeros(0)
                 for s, n in enumerate(sizes)]
        col32 = np.concatenate(parts).astype(np.float32)
        nll, g = api.nll_grad_stream(m, d, [_pinned(col32, torch.float32)], th)
        for s, n in enumerate(sizes):
            if n == 0:
                assert nll[s] == 0.0
                continue
            check_nll(nll[s], g[s], om.nll(th[s], [col32[off[s]:off[s + 1]].astype(np.float64)]), f"set {s}")
