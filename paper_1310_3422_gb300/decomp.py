"""Domain decomposition of one large GE solve over ranks (torch.distributed).

Rank q owns the contiguous range [a_q, b_q) of the grid (even bounds, so the
groups of every parity stay on one rank or straddle a boundary the same way
they do globally).  It keeps a copy of `halo` points on each side; every block
of `depth` steps it advances its extended range locally, then refreshes its
halos from its neighbours with one point-to-point exchange per side.  After S
steps a point depends only on the points within S+1 of it (the dependency cone
of the GE step, arXiv:1310.3422 Sec. 2), so with halo >= depth + 1 the owned
points come out exactly as in a monolithic solve; the garbage that a halo's
outer end collects (it is treated as a wall) stays inside the halo.

The local stepper advances a 1D array by some steps with given wall values and
global step counter; by default it is the CUDA library (``gpu_stepper``).
Collectives: none on the data path, only send/recv of halos.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable

import numpy as np

Stepper = Callable[[np.ndarray, float, float, float, int, int], np.ndarray]


@dataclass
class Part:
    rank: int
    world: int
    n: int
    a: int          # first owned point
    b: int          # one past the last owned point
    lo: int         # first point of the extended (owned + halo) range
    hi: int         # one past the last point of the extended range
    halo: int       # halo width (even)


def partition(n: int, world: int, rank: int, halo: int) -> Part:
    """Contiguous owned ranges with even bounds; extended by `halo` (rounded
    up to even) points on each side, clipped to the grid.  Every rank must own
    at least `halo` points (its neighbours' halos come from its owned values)."""
    if halo % 2:
        halo += 1
    cuts = [2 * ((n * q) // (2 * world)) for q in range(world)] + [n]
    a, b = cuts[rank], cuts[rank + 1]
    if world > 1 and min(cuts[q + 1] - cuts[q] for q in range(world)) < halo:
        raise ValueError("each rank must own at least depth + 1 points")
    return Part(rank, world, n, a, b, max(0, a - halo), min(n, b + halo), halo)


def gpu_stepper(u: np.ndarray, r: float, beta_l: float, beta_r: float, steps: int, step0: int) -> np.ndarray:
    """Advance u with the CUDA library (tiled FP64 kernel) on the current device."""
    import torch

    from . import binding as B
    x = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).cuda()
    ctx = B.ge_create(x.numel(), r, beta_l, beta_r, B.GE_F64, x)
    B.ge_write_state(ctx, x, step0)
    B.ge_step_n(ctx, steps)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    return out.cpu().numpy()


def solve_decomposed(u0: np.ndarray, r: float, beta_l: float, beta_r: float, steps: int, depth: int,
                     dist, stepper: Stepper = gpu_stepper, step0: int = 0) -> np.ndarray:
    """Advance the global state u0 (every rank passes the same array) by
    `steps` steps, split over dist.get_world_size() ranks.  Returns this
    rank's owned values u[a:b] after the steps.  `dist` is torch.distributed
    with an initialised process group."""
    import torch
    world, rank = dist.get_world_size(), dist.get_rank()
    n = u0.size
    halo = depth + 1
    p = partition(n, world, rank, halo)
    ext = np.array(u0[p.lo:p.hi], dtype=np.float64)
    done = 0
    while done < steps:
        L = min(depth, steps - done)
        # walls: the true walls at the grid's ends, anything elsewhere (the
        # halo's outer end is corrupted anyway)
        bl = beta_l if p.lo == 0 else 0.0
        br = beta_r if p.hi == n else 0.0
        ext = stepper(ext, r, bl, br, L, step0 + done)
        done += L
        if done < steps:
            ext = _exchange(ext, p, dist, torch)
    return ext[p.a - p.lo:p.b - p.lo].copy()


def _exchange(ext: np.ndarray, p: Part, dist, torch) -> np.ndarray:
    """Refresh both halos from the neighbours' owned values.  My left halo is
    [lo, a) = the left neighbour's last a - lo owned points; the left
    neighbour's right halo is my first min(halo, n - a) owned points (and
    symmetrically on the right)."""
    off = p.lo
    reqs, recv_l, recv_r = [], None, None
    if p.rank > 0:
        n_send = min(p.halo, p.n - p.a)
        send = torch.from_numpy(np.ascontiguousarray(ext[p.a - off:p.a - off + n_send]))
        recv_l = torch.empty(p.a - p.lo, dtype=torch.float64)
        reqs.append(dist.isend(send, p.rank - 1))
        reqs.append(dist.irecv(recv_l, p.rank - 1))
    if p.rank < p.world - 1:
        n_send = min(p.halo, p.b)
        send = torch.from_numpy(np.ascontiguousarray(ext[p.b - off - n_send:p.b - off]))
        recv_r = torch.empty(p.hi - p.b, dtype=torch.float64)
        reqs.append(dist.isend(send, p.rank + 1))
        reqs.append(dist.irecv(recv_r, p.rank + 1))
    for q in reqs:
        q.wait()
    if recv_l is not None:
        ext[:p.a - off] = recv_l.numpy()
    if recv_r is not None:
        ext[p.b - off:] = recv_r.numpy()
    return ext
