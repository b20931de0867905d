"""Learned surrogate of K GE steps with the GE solver as its fallback and arbiter.

The surrogate (the spectral neural operator of ``include/ge_sno.h``, run by
the library's own forward / backward / Adam kernels) maps the state of an
n-point problem to its state K GE steps later.  The GE solver

  * generates its training data (pairs (u_{jK}, u_{(j+1)K}) along GE
    trajectories, so the network sees the states a rollout meets),
  * checks it: ``solve_with_fallback`` re-solves a random sample of the
    problems (plus every flagged one) with GE and compares, and
  * takes over: flagged and sampled problems get GE's answer, and when any
    sampled problem misses the tolerance the whole batch is re-solved by GE.

The paper (arXiv:1310.3422) has no counterpart; the GE step itself is its
Sec. 2.  Everything here is orchestration: data movement and reductions in
torch on the device, all arithmetic of the network and of GE in libge.so.
Problems are equal-size rows of a [P, n] tensor with n a multiple of 32 (so
the rows are also a valid packed layout of the batched GE solver).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import binding as B
from . import inputs


@dataclass(frozen=True)
class SnoArch:
    n: int = 1024
    width: int = 64
    modes: int = 16
    layers: int = 4
    hidden: int = 128


def _torch():
    import torch
    return torch


class GEBatch:
    """Batched GE on the rows of a [P, n] tensor (per-row r and walls)."""

    def __init__(self, r, beta_l, beta_r, n: int, prec: int, stream=None):
        if n % 32:
            raise ValueError("row length must be a multiple of 32 for the packed layout")
        P = len(r)
        self.n, self.P, self.prec = n, P, prec
        self.plan = B.ge_batch_create(np.full(P, n, dtype=np.int64), np.asarray(r, dtype=np.float64),
                                      np.asarray(beta_l, dtype=np.float64), np.asarray(beta_r, dtype=np.float64),
                                      np.arange(P, dtype=np.int64) * n, P * n, prec, stream)

    def run(self, u, steps: int):
        """Advance every row of u ([P, n], the plan's dtype) by `steps` steps in place."""
        B.ge_batch_run(self.plan, u, steps)

    def close(self):
        B.ge_batch_destroy(self.plan)


@dataclass
class TrainingSet:
    """Device tensors: x, y [N, n] float32 (state and the state K steps on),
    r, beta_l, beta_r [N] float32."""
    x: object
    y: object
    r: object
    beta_l: object
    beta_r: object

    def __len__(self):
        return int(self.x.shape[0])


def make_training_set(n_traj: int, arch: SnoArch = SnoArch(), K: int = 256, jumps: int = 8,
                      seed: int = inputs.SEED_BASE + 4, prec: int = B.GE_F64) -> TrainingSet:
    """n_traj GE trajectories of `jumps` jumps of K steps (GE in precision
    `prec`, FP64 by default; stored as FP32): n_traj * jumps training pairs."""
    torch = _torch()
    probs = inputs.surrogate_problems(n_traj, arch.n, seed=seed)
    u = torch.tensor(probs.u0, dtype=torch.float64 if prec == B.GE_F64 else torch.float32, device="cuda")
    ge = GEBatch(probs.r, probs.beta_l, probs.beta_r, arch.n, prec)
    xs, ys = [], []
    for _ in range(jumps):
        # copies: with FP32 GE, u.float() would be u itself, advanced in place
        xs.append(u.to(torch.float32, copy=True))
        ge.run(u, K)
        ys.append(u.to(torch.float32, copy=True))
    B.ge_batch_sync(ge.plan)
    ge.close()

    def rep(a):
        return torch.tensor(np.tile(np.asarray(a, dtype=np.float32), jumps), device="cuda")

    return TrainingSet(torch.cat(xs), torch.cat(ys), rep(probs.r), rep(probs.beta_l), rep(probs.beta_r))


class Surrogate:
    """A ge_sno model plus its training and batched inference loops."""

    def __init__(self, arch: SnoArch = SnoArch(), K: int = 256, max_batch: int = 256, seed: int = 0,
                 split: int = 0, stream=None):
        self.arch, self.K, self.max_batch = arch, K, max_batch
        self.model = B.ge_sno_create(arch.n, arch.width, arch.modes, arch.layers, arch.hidden, max_batch, seed,
                                     stream)
        B.ge_sno_set_precision(self.model, split)
        self.num_params = B.ge_sno_num_params(self.model)

    def set_precision(self, split: int):
        B.ge_sno_set_precision(self.model, split)

    def params(self):
        torch = _torch()
        p = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        B.ge_sno_get_params(self.model, p)
        return p

    def set_params(self, p):
        B.ge_sno_set_params(self.model, p.contiguous())

    def train(self, data: TrainingSet, steps: int, batch: int = 64, lr: float = 1e-3, lr_min: float = 1e-5,
              seed: int = 0, warmup: int = 100) -> np.ndarray:
        """Adam on random mini-batches, linear warm-up then cosine decay of the
        learning rate.  Returns the mean training loss of every step."""
        torch = _torch()
        if batch > self.max_batch:
            raise ValueError("batch larger than the model's max_batch")
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        losses = torch.empty(steps, batch, dtype=torch.float32, device="cuda")
        for s in range(steps):
            idx = torch.randint(0, len(data), (batch,), device="cuda", generator=g)
            if s < warmup:
                rate = lr * (s + 1) / warmup
            else:
                rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * (s - warmup) / max(1, steps - warmup)))
            B.ge_sno_train_step(self.model, batch, data.x[idx].contiguous(), data.r[idx].contiguous(),
                                data.beta_l[idx].contiguous(), data.beta_r[idx].contiguous(),
                                data.y[idx].contiguous(), rate, losses[s])
        return losses.mean(dim=1).cpu().numpy()

    def predict(self, u, r, beta_l, beta_r, out=None):
        """One jump of K steps for every row of u ([P, n] float32)."""
        torch = _torch()
        P = u.shape[0]
        if out is None:
            out = torch.empty_like(u)
        for s in range(0, P, self.max_batch):
            e = min(P, s + self.max_batch)
            B.ge_sno_forward(self.model, e - s, u[s:e], r[s:e], beta_l[s:e], beta_r[s:e], out[s:e])
        return out

    def rollout(self, u0, r, beta_l, beta_r, jumps: int):
        """`jumps` jumps (jumps * K steps) from u0 ([P, n] float32)."""
        torch = _torch()
        bufs = (torch.empty_like(u0), torch.empty_like(u0))
        src = u0.contiguous()
        for j in range(jumps):
            self.predict(src, r, beta_l, beta_r, out=bufs[j % 2])
            src = bufs[j % 2]
        return src

    def evaluate(self, data: TrainingSet, limit: int | None = None) -> np.ndarray:
        """Per-pair relative L2 error of one jump on (part of) a data set."""
        torch = _torch()
        n = len(data) if limit is None else min(limit, len(data))
        pred = self.predict(data.x[:n], data.r[:n], data.beta_l[:n], data.beta_r[:n])
        y = data.y[:n]
        return (torch.linalg.vector_norm(pred - y, dim=1) / torch.linalg.vector_norm(y, dim=1)).cpu().numpy()

    def close(self):
        B.ge_sno_destroy(self.model)


@dataclass
class FallbackReport:
    n_problems: int
    n_sampled: int
    n_flagged: int
    sample_max_err: float
    sample_mean_err: float
    n_sample_over_tol: int
    fell_back_all: bool
    sample: np.ndarray = field(repr=False, default=None)


def solve_with_fallback(sur: Surrogate, u0, r, beta_l, beta_r, jumps: int, tol: float = 1e-3,
                        sample_frac: float = 0.01, seed: int = 0, r_range=(0.5, 4.0),
                        ge_prec: int = B.GE_F32):
    """State after jumps * K steps for every row of u0 ([P, n] float32 on the
    device; r, beta_l, beta_r float32 [P]).

    1. The surrogate jumps every problem ahead `jumps` times.
    2. Flagged problems: a non-finite result or r outside the trained range.
    3. GE (precision ge_prec) re-solves a random sample of ceil(sample_frac P)
       problems plus the flagged ones from u0, and those rows take GE's result.
    4. If any sampled problem's relative L2 error exceeds tol, the surrogate
       is not trusted on this batch and every problem is re-solved by GE.
    Returns (state, FallbackReport)."""
    torch = _torch()
    P, n = u0.shape
    steps = jumps * sur.K
    dev = u0.device
    u0 = u0.contiguous()
    u = sur.rollout(u0, r, beta_l, beta_r, jumps)
    # flag, gather, compare and scatter rows with the library's own kernels;
    # the host only draws the sample and takes the decisions
    bad = torch.empty(P, dtype=torch.int32, device=dev)
    B.ge_sno_rows_nonfinite(sur.model, u, bad)
    r_h, bl_h, br_h = (x.double().cpu().numpy() for x in (r, beta_l, beta_r))
    flagged = (bad.cpu().numpy() != 0) | (r_h < r_range[0]) | (r_h > r_range[1])
    flagged_idx = np.nonzero(flagged)[0]
    rng = np.random.default_rng(seed)
    n_sample = min(P, max(1, int(math.ceil(sample_frac * P))))
    sample = np.sort(rng.choice(P, n_sample, replace=False))
    check = np.union1d(sample, flagged_idx)
    ci = torch.tensor(check, dtype=torch.int64, device=dev)
    ref = torch.empty(check.size, n, dtype=torch.float32, device=dev)
    B.ge_sno_rows_gather(sur.model, u0, ci, ref)
    ge = GEBatch(r_h[check], bl_h[check], br_h[check], n, ge_prec)
    if ge_prec == B.GE_F64:
        ref64 = ref.double()
        ge.run(ref64, steps)
        ref = ref64.float()
    else:
        ge.run(ref, steps)
    ge.close()
    err = torch.empty(check.size, dtype=torch.float32, device=dev)
    B.ge_sno_rows_rel_err(sur.model, u, ci, ref, err)
    err_h = err.cpu().numpy()
    se = err_h[np.isin(check, sample) & ~flagged[check]]
    n_over = int((se > tol).sum())
    B.ge_sno_rows_scatter(sur.model, u, ci, ref)
    fell_back = n_over > 0
    if fell_back:
        ref_dtype = torch.float64 if ge_prec == B.GE_F64 else torch.float32
        full = u0.to(ref_dtype, copy=True)
        ge = GEBatch(r_h, bl_h, br_h, n, ge_prec)
        ge.run(full, steps)
        u = full.float() if ge_prec == B.GE_F64 else full
        ge.close()
    rep = FallbackReport(P, n_sample, int(flagged_idx.size), float(se.max()) if se.size else 0.0,
                         float(se.mean()) if se.size else 0.0, n_over, fell_back, sample)
    return u, rep
