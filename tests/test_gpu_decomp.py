"""Domain decomposition with a device-resident GE context of the library
(tiled FP64 kernel) per rank for the whole solve, halos read and written as
device ranges: two gloo ranks in separate processes share the one GPU (their
launches never wait on one another; under gloo the halos are staged through
the host between launches), and the assembled result matches the monolithic
oracle to the FP64 parity tolerance."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from tolerances import tol64

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, r, bl, br, steps, depth, step0, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    from paper_1310_3422_gb300 import decomp
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u0 = np.random.default_rng(43).standard_normal(n)
        part = decomp.partition(n, world, rank, depth + 1)
        own = decomp.solve_decomposed(u0, r, bl, br, steps, depth, dist, step0=step0)
        q.put((rank, part.a, part.b, own))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,steps,depth,step0", [(2, 100001, 130, 40, 0), (2, 50000, 97, 33, 1)])
def test_decomposed_gpu_stepper_matches_oracle(world, n, steps, depth, step0):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    r, bl, br = 1.7, 0.3, -0.8
    procs = [ctx.Process(target=_worker, args=(k, world, port, n, r, bl, br, steps, depth, step0, q))
             for k in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    u0 = np.random.default_rng(43).standard_normal(n)
    want = oracle.run(u0, r, bl, br, steps, step0=step0)
    got = np.empty(n)
    covered = np.zeros(n, bool)
    for rank, a, b, own in parts:
        got[a:b] = own
        covered[a:b] = True
    assert covered.all()
    assert np.max(np.abs(got - want)) <= tol64(r) * np.max(np.abs(want))
