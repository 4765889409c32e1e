"""Sharded evaluation on one GPU: each shard is uploaded and evaluated on
its own (as each rank would on its GPU), the shards' compensated partial
sums are merged by the exchange step, and the result is compared with the
oracle on the whole dataset and with the unsharded pass.  The shards run one
after another; no kernel waits on another."""
import numpy as np
import pytest
import torch

from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node

from helpers import TRUE, check_nll

pytestmark = pytest.mark.gpu


def _partials(model, shards, theta):
    """Per shard: (pairs, flags) from rf_nll_grad_partial."""
    P = model.n_free
    out_p, out_f = [], []
    for cols, off in shards:
        d = api.Data.upload(model, cols, offsets=off)
        S = d.n_sets
        th = torch.as_tensor(np.tile(theta, (S, 1)).reshape(-1), dtype=torch.float64).cuda()
        pairs = torch.full((S, 1 + P, 2), np.nan, dtype=torch.float64, device="cuda")
        flags = torch.full((S,), -1, dtype=torch.int32, device="cuda")
        api.nll_grad_partial(model, d, th, pairs, flags)
        torch.cuda.synchronize()
        out_p.append(pairs.cpu().numpy())
        out_f.append(flags.cpu().numpy())
    return np.stack(out_p), np.stack(out_f)


def _split_sets(cols_per_set, world):
    """Every set's events split by rf_shard (4096-aligned); shard r holds its
    slice of every set."""
    shards = []
    for r in range(world):
        parts, off = [], [0]
        for c in cols_per_set:
            lo, hi = api.shard(len(c[0]), 4096, r, world)
            parts.append([x[lo:hi] for x in c])
            off.append(off[-1] + hi - lo)
        n_obs = len(cols_per_set[0])
        cols = [np.concatenate([p[j] for p in parts]) for j in range(n_obs)]
        shards.append((cols, off))
    return shards


@pytest.mark.parametrize("which", ["decay_model", "prod3_model"])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_sharded_matches_oracle_and_unsharded(oracle_mod, which, world):
    spec = W.model_for(which)
    om = oracle_mod.Model(spec.nodes, spec.root)
    sizes = [5 * 4096 + 300, 0, 4096, 77]
    th = np.array(TRUE[which]) * 1.02
    cols = [om.generate(TRUE[which], 41, s, 0, n) if n else [np.zeros(0)] * spec.n_obs
            for s, n in enumerate(sizes)]
    m = api.Model.from_spec(spec)
    allp, allf = _partials(m, _split_sets(cols, world), th)
    assert not np.isnan(allp).any() and (allf == 0).all()
    out, fo = api.combine_partials(allp, allf)
    whole = [np.concatenate([c[j] for c in cols]) for j in range(spec.n_obs)]
    d = api.Data.upload(m, whole, offsets=np.concatenate([[0], np.cumsum(sizes)]))
    nll, g = api.nll_grad(m, d, np.tile(th, (len(sizes), 1)))
    for s, n in enumerate(sizes):
        if n == 0:
            assert out[s, 0] == 0.0 and np.all(out[s, 1:] == 0.0)
            continue
        ref = om.nll(th, cols[s])
        check_nll(out[s, 0], out[s, 1:], ref, f"{which} world {world} set {s}")
        check_nll(nll[s], g[s], ref, f"unsharded set {s}")
    # a fixed shard layout gives fixed bits
    again, _ = api.combine_partials(*_partials(m, _split_sets(cols, world), th))
    assert np.array_equal(out, again)


def test_sharded_generic_kernel_and_domain_flag(oracle_mod):
    nodes = [Node("obs", (), 0, -1.0, 4.0), Node("param", (), -0.6, -5, 5, True),
             Node("param", (), 1.0, -5, 5, True), Node("param", (), 0.3, 0.01, 5, True),
             Node("exp", (0, 1)), Node("gauss", (0, 2, 3)), Node("param", (), 0.5, 0, 1, True),
             Node("sum", (4, 5, 6))]
    om = oracle_mod.Model(nodes, 7)
    th = np.array([-0.6, 1.0, 0.3, 0.5])
    x = om.generate(th, 5, 0, 0, 20000)
    m = api.Model(nodes, 7)
    assert "kernel=generic" in m.describe()
    allp, allf = _partials(m, _split_sets([x], 3), th)
    out, fo = api.combine_partials(allp, allf)
    check_nll(out[0, 0], out[0, 1:], om.nll(th, x), "generic sharded")
    bad = th.copy()
    bad[2] = -1.0  # sigma < 0: outside the Gaussian's domain on every shard
    allp, allf = _partials(m, _split_sets([x], 3), bad)
    out, fo = api.combine_partials(allp, allf)
    assert fo[0] & (1 << 30) and np.isinf(out[0, 0])
