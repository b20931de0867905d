"""Domain decomposition over CPU ranks (gloo): ranks exchanging halos give the
monolithic oracle's result bit for bit (the oracle is the local stepper)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1310_3422_gb300 import decomp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, r, bl, br, steps, depth, step0, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u0 = np.random.default_rng(42).standard_normal(n)
        part = decomp.partition(n, world, rank, depth + 1)
        own = decomp.solve_decomposed(u0, r, bl, br, steps, depth, dist, stepper=oracle.run, step0=step0)
        q.put((rank, part.a, part.b, own))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,steps,depth,step0", [
    (2, 1001, 57, 8, 0), (2, 1000, 40, 16, 1), (3, 2003, 77, 12, 0), (4, 997, 30, 5, 3)])
def test_decomposed_equals_monolithic(world, n, steps, depth, step0):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    r, bl, br = 1.7, 0.3, -0.8
    procs = [ctx.Process(target=_worker, args=(k, world, port, n, r, bl, br, steps, depth, step0, q))
             for k in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u0 = np.random.default_rng(42).standard_normal(n)
    want = oracle.run(u0, r, bl, br, steps, step0=step0)
    got = np.empty(n)
    covered = np.zeros(n, bool)
    for rank, a, b, own in parts:
        got[a:b] = own
        covered[a:b] = True
    assert covered.all()
    assert np.array_equal(got, want)


def test_partition_bounds():
    for world in (1, 2, 3, 5):
        cuts = [decomp.partition(1000, world, k, 9) for k in range(world)]
        assert cuts[0].a == 0 and cuts[-1].b == 1000
        for k in range(world):
            assert cuts[k].a % 2 == 0 and cuts[k].halo == 10
            if k:
                assert cuts[k].a == cuts[k - 1].b
    with pytest.raises(ValueError):
        decomp.partition(30, 4, 0, 9)
