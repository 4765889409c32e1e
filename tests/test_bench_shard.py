"""bench.py --shard (strong scaling of one dataset over the ranks): its
exchange step, driven on 2 gloo ranks on the CPU.  The shards' partial sums
come from the oracle (the GPU's own partial pass is compared in
test_gpu_sharding.py); bench.exchange_partials gathers them in rank order and
merges them exactly, and every rank must hold the whole dataset's NLL and
gradient, bitwise the same on every rank."""
import os
import socket

import numpy as np

from helpers import GRAD_RTOL, NLL_RTOL, oracle_data


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, here)
    sys.path.insert(0, os.path.dirname(here))
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2003_12861_gb300 import api
    from paper_2003_12861_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n = 5 * 4096 + 321
        spec, om, cols = oracle_data(oracle, "prod3_model", n, seed=5)
        th = np.array(W.PROD3_TRUE) * (1 + 0.01 * np.cos(np.arange(12)))
        lo, hi = api.shard(n, 4096, rank, world)
        nll, g, *_ = om.nll(th, [c[lo:hi] for c in cols])
        pairs = np.zeros((1, 13, 2))
        pairs[0, 0, 0] = -nll
        pairs[0, 1:, 0] = -np.asarray(g)
        out, fo = bench.exchange_partials(api, pairs, np.zeros(1, dtype=np.int32))
        q.put((rank, out, fo))
    finally:
        dist.destroy_process_group()


def test_shard_mode_exchange_on_two_gloo_ranks(oracle_mod):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, out, fo = q.get(timeout=300)
        got[r] = (out, fo)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])
    n = 5 * 4096 + 321
    spec, om, cols = oracle_data(oracle_mod, "prod3_model", n, seed=5)
    from paper_2003_12861_gb300 import workloads as W
    th = np.array(W.PROD3_TRUE) * (1 + 0.01 * np.cos(np.arange(12)))
    nll, g, al, ag, _ = om.nll(th, cols)
    out = got[0][0][0]
    assert got[0][1][0] == 0
    assert abs(out[0] - nll) <= NLL_RTOL * al
    assert np.all(np.abs(out[1:] - g) <= GRAD_RTOL * ag)
