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

The extended range lives in a local state that advances in place and lets
ranges of it be read and written:
  * ``DeviceState``: one GE context of the CUDA library over the extended
    range for the whole solve (tiled FP64 kernel); halos move as device
    tensors (``ge_read_range`` / ``ge_write_range``), sent with NCCL
    point-to-point calls when the process group is NCCL, staged through
    host memory for gloo;
  * ``ArrayState``: a host array advanced by a given stepper function
    (a CPU reference, for tests).
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


def halo_plan(p: Part):
    """The exchange of one rank, as (peer, send range, receive range) per
    neighbour, ranges in coordinates of the extended range.  My left halo
    [lo, a) is the left neighbour's last a - lo owned points; the left
    neighbour's right halo is my first min(halo, n - a) owned points (and
    symmetrically on the right)."""
    off = p.lo
    plan = []
    if p.rank > 0:
        n_send = min(p.halo, p.n - p.a)
        plan.append((p.rank - 1, (p.a - off, n_send), (0, p.a - p.lo)))
    if p.rank < p.world - 1:
        n_send = min(p.halo, p.b)
        plan.append((p.rank + 1, (p.b - off - n_send, n_send), (p.b - off, p.hi - p.b)))
    return plan


class ArrayState:
    """Extended range held in a host array, advanced by `stepper(u, r,
    beta_l, beta_r, steps, step0)`."""

    def __init__(self, u, r, beta_l, beta_r, step0, stepper: Stepper):
        self.u = np.array(u, dtype=np.float64)
        self.r, self.bl, self.br, self.step = r, beta_l, beta_r, step0
        self.stepper = stepper
        self.device = None

    def step_n(self, k: int):
        self.u = self.stepper(self.u, self.r, self.bl, self.br, k, self.step)
        self.step += k

    def read(self, off: int, count: int):
        import torch
        return torch.from_numpy(np.ascontiguousarray(self.u[off:off + count]))

    def write(self, off: int, values):
        self.u[off:off + values.numel()] = values.numpy()

    def result(self, off: int, count: int) -> np.ndarray:
        return self.u[off:off + count].copy()

    def close(self):
        pass


class DeviceState:
    """Extended range held by one GE context of the CUDA library (tiled FP64
    kernel, `depth` steps per launch) for the whole solve, on the current
    device and stream."""

    def __init__(self, u, r, beta_l, beta_r, step0, depth: int = 0):
        import torch

        from . import binding as B
        self.B, self.torch = B, torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        x = torch.as_tensor(np.ascontiguousarray(u, dtype=np.float64)).to(self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self.ctx = B.ge_create(x.numel(), r, beta_l, beta_r, B.GE_F64, x, stream=self.stream)
        B.ge_set_kernel(self.ctx, B.GE_KERNEL_TEMPORAL, depth)
        B.ge_write_state(self.ctx, x, step0)

    def step_n(self, k: int):
        self.B.ge_step_n(self.ctx, k)

    def read(self, off: int, count: int):
        t = self.torch.empty(count, dtype=self.torch.float64, device=self.device)
        self.B.ge_read_range(self.ctx, off, count, t)
        return t

    def write(self, off: int, values):
        self.B.ge_write_range(self.ctx, off, values.numel(), values)

    def result(self, off: int, count: int) -> np.ndarray:
        t = self.read(off, count)
        self.B.ge_sync(self.ctx)
        return t.cpu().numpy()

    def close(self):
        self.B.ge_sync(self.ctx)
        self.B.ge_destroy(self.ctx)


def exchange_halos(state, p: Part, dist):
    """Refresh both halos of `state` from the neighbours' owned values: one
    send and one receive per neighbour, issued together as one batch (NCCL
    runs a batch as one group, so no pairing order can deadlock).  Device
    tensors go to NCCL as they are; under another backend (gloo) they are
    staged through host memory."""
    import torch
    plan = halo_plan(p)
    if not plan:
        return
    on_device = state.device is not None
    direct = not on_device or dist.get_backend() == "nccl"
    ops, recvs = [], []
    for peer, (s_off, s_cnt), (r_off, r_cnt) in plan:
        send = state.read(s_off, s_cnt)
        if not direct:
            send = send.cpu()
        recv = torch.empty(r_cnt, dtype=torch.float64, device=send.device)
        ops.append(dist.P2POp(dist.isend, send, peer))
        ops.append(dist.P2POp(dist.irecv, recv, peer))
        recvs.append((r_off, recv))
    for q in dist.batch_isend_irecv(ops):
        q.wait()
    for r_off, recv in recvs:
        if on_device and not direct:
            recv = recv.to(state.device)
        state.write(r_off, recv)


def solve_decomposed(u0: np.ndarray, r: float, beta_l: float, beta_r: float, steps: int, depth: int,
                     dist, stepper: Stepper | None = None, step0: int = 0) -> np.ndarray:
    """Advance the global state u0 (every rank passes the same array) by
    `steps` steps, split over dist.get_world_size() ranks.  Returns this
    rank's owned values u[a:b] after the steps.  `dist` is torch.distributed
    with an initialised process group.  With `stepper` the extended range is
    a host array advanced by it; without, a device-resident GE context on
    the current device."""
    world, rank = dist.get_world_size(), dist.get_rank()
    n = u0.size
    p = partition(n, world, rank, depth + 1)
    # walls: the true walls at the grid's ends, anything elsewhere (the halo's
    # outer end is corrupted anyway)
    bl = beta_l if p.lo == 0 else 0.0
    br = beta_r if p.hi == n else 0.0
    ext = u0[p.lo:p.hi]
    state = (ArrayState(ext, r, bl, br, step0, stepper) if stepper is not None
             else DeviceState(ext, r, bl, br, step0, depth))
    try:
        done = 0
        while done < steps:
            L = min(depth, steps - done)
            state.step_n(L)
            done += L
            if done < steps:
                exchange_halos(state, p, dist)
        return state.result(p.a - p.lo, p.b - p.a)
    finally:
        state.close()
