"""Sharded evaluation (one dataset over several ranks) and its exchange step,
on the host: the shard ranges, the rank-ordered combine of compensated
partial sums, and a 2-rank gloo run against the oracle.  The shards' partial
sums come from the oracle here (no GPU on the CPU runner); the GPU's own
partial pass is compared in test_gpu_sharding.py."""
import os
import socket

import numpy as np
import pytest

from paper_2003_12861_gb300 import api

from helpers import GRAD_RTOL, NLL_RTOL, oracle_data


def test_shard_ranges_cover_disjoint_and_aligned():
    for n in (0, 1, 4095, 4096, 4097, 10_000_000, 123_456_789):
        for world in (1, 2, 3, 4, 7, 8):
            ranges = [api.shard(n, 4096, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            for a, b in ranges[:-1]:
                assert b % 4096 == 0 or b == n
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 4096 + (n % 4096 if n % 4096 else 0)
    # sets (align 1): sizes differ by at most one
    for S in (0, 1, 5, 4096, 10_000):
        for world in (1, 2, 3, 8):
            sizes = [np.subtract(*api.shard(S, 1, r, world)[::-1]) for r in range(world)]
            assert sum(sizes) == S and max(sizes) - min(sizes) <= 1
    assert api.shard(1 << 60, 4096, 7, 8)[1] == 1 << 60  # no overflow


def test_shard_rejects_bad_arguments():
    from paper_2003_12861_gb300 import _lib as L
    for args in ((-1, 1, 0, 1), (10, 0, 0, 1), (10, 1, 1, 1), (10, 1, -1, 2), (10, 1, 0, 0)):
        with pytest.raises(L.RFError):
            api.shard(*args)


def test_combine_is_exact_and_rank_ordered():
    # Per-rank sums whose plain addition loses everything but whose exact sum is 2.
    p = np.zeros((3, 1, 2, 2))
    p[0, 0, :, 0] = [1e16, 0.0]
    p[1, 0, :, 0] = [1.0, 3.0]
    p[2, 0, :, 0] = [-1e16, 0.0]
    p[1, 0, 0, 1] = 1.0  # a compensation term travels with its pair
    out, fl = api.combine_partials(p, np.zeros((3, 1), dtype=np.int32))
    assert out[0, 0] == -2.0 and out[0, 1] == -3.0 and fl[0] == 0
    # rank order is the definition: the result depends only on the array order
    q = np.random.default_rng(5).standard_normal((4, 3, 4, 2)) * 10.0 ** np.arange(4)[None, None, :, None]
    a, _ = api.combine_partials(q, np.zeros((4, 3), dtype=np.int32))
    b, _ = api.combine_partials(q.copy(), np.zeros((4, 3), dtype=np.int32))
    assert np.array_equal(a, b)
    assert np.allclose(a, -q.sum(axis=(0, 3)), rtol=1e-14, atol=1e-12)


def test_combine_flags():
    p = np.ones((2, 2, 3, 2))
    f = np.array([[0, 3], [1 << 30, 2]], dtype=np.int32)
    out, fo = api.combine_partials(p, f)
    assert list(fo) == [1 << 30, 5]
    assert np.isinf(out[0, 0]) and np.isinf(out[1, 0]) and out[1, 1] == -4.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    """One gloo rank: its shard of a decay dataset (events) and of a toy batch
    (sets); partial sums from the oracle; the exchange; the combined result."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import oracle
    from paper_2003_12861_gb300 import api as A
    from paper_2003_12861_gb300 import workloads as W2
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        res = {}
        # one set of 3 chunks + a ragged tail, split by events
        n = 3 * 4096 + 777
        spec, om, cols = oracle_data(oracle, "decay_model", n, seed=77)
        th = np.array(W2.DECAY_TRUE) * 1.03
        lo, hi = A.shard(n, 4096, rank, world)
        nll, g, *_ = om.nll(th, [c[lo:hi] for c in cols])
        pairs = np.zeros((1, 1 + len(g), 2))
        pairs[0, 0, 0] = -nll
        pairs[0, 1:, 0] = -np.asarray(g)
        allp, allf = A.gather_partials(pairs, np.zeros(1, dtype=np.int32))
        res["events"] = A.combine_partials(allp, allf)[0]
        # a batch of 5 ragged toys, split by sets
        sizes = [100, 0, 5000, 4096, 33]
        s0, s1 = A.shard(len(sizes), 1, rank, world)
        pairs = np.zeros((s1 - s0, 1 + len(g), 2))
        for j, s in enumerate(range(s0, s1)):
            if sizes[s]:
                c = om.generate(W2.DECAY_TRUE, 9, s, 0, sizes[s])
                v, gg, *_ = om.nll(th, c)
                pairs[j, 0, 0] = -v
                pairs[j, 1:, 0] = -np.asarray(gg)
        # sets are disjoint across ranks: each rank sends a full-size block with
        # zeros outside its own sets, so the rank-ordered merge is the union
        full = np.zeros((len(sizes), 1 + len(g), 2))
        full[s0:s1] = pairs
        allp, allf = A.gather_partials(full, np.zeros(len(sizes), dtype=np.int32))
        res["sets"] = A.combine_partials(allp, allf)[0]
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_sharded_nll_matches_the_whole_dataset(oracle_mod, world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank holds the same bits
    for r in range(1, world):
        for k in got[0]:
            assert np.array_equal(got[0][k], got[r][k])
    # and they match the oracle on the whole data
    n = 3 * 4096 + 777
    spec, om, cols = oracle_data(oracle_mod, "decay_model", n, seed=77)
    from paper_2003_12861_gb300 import workloads as W2
    th = np.array(W2.DECAY_TRUE) * 1.03
    ref = om.nll(th, cols)
    nll, g, al, ag, _ = ref
    out = got[0]["events"][0]
    assert abs(out[0] - nll) <= NLL_RTOL * al
    assert np.all(np.abs(out[1:] - g) <= GRAD_RTOL * np.maximum(ag, 1e-300))
    sizes = [100, 0, 5000, 4096, 33]
    for s, N in enumerate(sizes):
        o = got[0]["sets"][s]
        if N == 0:
            assert o[0] == 0.0 and np.all(o[1:] == 0.0)
            continue
        c = om.generate(W2.DECAY_TRUE, 9, s, 0, N)
        v, gg, a2, ag2, _ = om.nll(th, c)
        assert abs(o[0] - v) <= NLL_RTOL * a2
        assert np.all(np.abs(o[1:] - gg) <= GRAD_RTOL * np.maximum(ag2, 1e-300))
