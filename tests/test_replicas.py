"""Multi-rank bookkeeping on the CPU (gloo, world size 2): the slowest
rank's time reaches every rank, and the longest-processing-time mesh
assignment covers every mesh once with balanced loads."""
import os

import pytest

from paper_2508_13386_gb300.replicas import lpt_shards, max_over_ranks


def test_lpt_shards_cover_and_balance():
    import numpy as np
    rng = np.random.default_rng(0)
    w = list(np.exp(rng.uniform(np.log(2e3), np.log(6e4), size=64)))
    for world in (1, 2, 3, 4, 8):
        shards = lpt_shards(w, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(64))
        loads = [sum(w[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(w) + 1e-9
    assert lpt_shards([3.0, 1.0], 4)[2:] == [[], []]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.25, 3.5][rank]
        q.put((rank, max_over_ranks(local, dist)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 3.5), (1, 3.5)]


def test_max_over_ranks_without_a_group():
    assert max_over_ranks(2.5) == 2.5
