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


def _halo_worker(rank, world, port, n, depth, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u = np.arange(n, dtype=np.float64) * 0.5 + 1.0
        p = decomp.partition(n, world, rank, depth + 1)
        ext = u[p.lo:p.hi].copy()
        # spoil the halos: the exchange must bring back the neighbours' values
        ext[:p.a - p.lo] = np.nan
        ext[p.b - p.lo:] = np.nan
        st = decomp.ArrayState(ext, 1.0, 0.0, 0.0, 0, stepper=None)
        decomp.exchange_halos(st, p, dist)
        q.put((rank, p.lo, p.hi, st.u.copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,depth", [(2, 1000, 16), (3, 999, 7), (4, 4000, 33)])
def test_halo_exchange_restores_neighbour_values(world, n, depth):
    """One exchange step alone: every rank's halos end up holding exactly the
    neighbours' owned values (the range plan and the send/receive pairing)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_halo_worker, args=(k, world, port, n, depth, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u = np.arange(n, dtype=np.float64) * 0.5 + 1.0
    for rank, lo, hi, ext in got:
        assert np.array_equal(ext, u[lo:hi]), rank


def test_halo_plan_pairs_up():
    """What rank q sends to q+1 is exactly what q+1 expects in its left halo."""
    for world, n, halo in ((2, 1000, 17), (5, 3001, 9), (3, 64, 10)):
        parts = [decomp.partition(n, world, k, halo) for k in range(world)]
        for k in range(world - 1):
            left, right = parts[k], parts[k + 1]
            send = [pl for pl in decomp.halo_plan(left) if pl[0] == k + 1][0][1]
            recv = [pl for pl in decomp.halo_plan(right) if pl[0] == k][0][2]
            assert send[1] == recv[1]
            assert left.lo + send[0] == right.lo + recv[0]
            send = [pl for pl in decomp.halo_plan(right) if pl[0] == k][0][1]
            recv = [pl for pl in decomp.halo_plan(left) if pl[0] == k + 1][0][2]
            assert send[1] == recv[1]
            assert right.lo + send[0] == left.lo + recv[0]


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
