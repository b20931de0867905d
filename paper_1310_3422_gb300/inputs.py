"""Seeded synthetic inputs for the GE solver (initial states, boundary values,
batches).  Holds none of the method's arithmetic: the same arrays feed the
CUDA library and the CPU oracle in the tests and the benchmark.

Grid convention: ``n`` interior points, ``x_i = (i + 1) / (n + 1)`` for
0-based index ``i``, walls at x = 0 and x = 1 (arXiv:1310.3422 Sec. 2,
mesh with h = 1/M, here M = n + 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 13103422


def grid(n: int) -> np.ndarray:
    """Interior node coordinates x_1..x_n of a mesh with h = 1/(n+1)."""
    return np.arange(1, n + 1, dtype=np.float64) / float(n + 1)


def sine_state(n: int) -> np.ndarray:
    """u0 = sin(pi x): the decaying first mode exp(-pi^2 t) sin(pi x)."""
    return np.sin(np.pi * grid(n))


def sine_modes_state(n: int, n_modes: int = 8, k_max: int = 64, seed: int = SEED_BASE + 1,
                     chunk: int = 1 << 22) -> np.ndarray:
    """u0 = sum_m A_m sin(k_m pi x) with distinct k_m drawn from 1..k_max and
    A_m ~ U(-1, 1) (the single large solve's initial state)."""
    rng = np.random.default_rng(seed)
    ks = rng.choice(np.arange(1, k_max + 1), size=n_modes, replace=False)
    amps = rng.uniform(-1.0, 1.0, size=n_modes)
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        x = np.arange(s + 1, min(n, s + chunk) + 1, dtype=np.float64) / float(n + 1)
        acc = np.zeros_like(x)
        for k, a in zip(ks, amps):
            acc += a * np.sin(k * np.pi * x)
        out[s:s + x.size] = acc
    return out


def random_state(n: int, seed: int) -> np.ndarray:
    """Rough state: independent N(0, 1) values (worst case for round-off)."""
    return np.random.default_rng(seed).standard_normal(n)


def fourier_state(n: int, beta_l: float, beta_r: float, rng: np.random.Generator,
                  n_modes: int = 16) -> np.ndarray:
    """Wall-compatible smooth state: the linear profile between the wall values
    plus sum_{k=1..n_modes} a_k / k^2 sin(k pi x), a_k ~ N(0, 1)."""
    x = grid(n)
    u = beta_l + (beta_r - beta_l) * x
    a = rng.standard_normal(n_modes)
    for k in range(1, n_modes + 1):
        u += a[k - 1] / float(k * k) * np.sin(k * np.pi * x)
    return u


@dataclass
class Batch:
    """Independent 1D problems packed back to back.

    ``offsets[b]`` is the element offset of problem b in ``u0`` (a multiple
    of ``align`` elements; 32 keeps every problem on its own 128-byte rows for
    both FP32 and FP64), ``n[b]`` its number of interior points."""
    n: np.ndarray
    r: np.ndarray
    beta_l: np.ndarray
    beta_r: np.ndarray
    offsets: np.ndarray
    u0: np.ndarray
    total: int


def uneven_batch(n_problems: int = 4096, n_min: int = 256, n_max: int = 65536,
                 r_min: float = 0.25, r_max: float = 4.0, seed: int = SEED_BASE + 2,
                 align: int = 32) -> Batch:
    """Batch of problems with N log-uniform in [n_min, n_max] rounded to even,
    r ~ U[r_min, r_max], wall values ~ U(-1, 1), u0 from ``fourier_state``."""
    rng = np.random.default_rng(seed)
    logn = rng.uniform(np.log(n_min), np.log(n_max), size=n_problems)
    n = (np.round(np.exp(logn) / 2.0) * 2).astype(np.int64)
    n = np.clip(n, n_min, n_max)
    r = rng.uniform(r_min, r_max, size=n_problems)
    bl = rng.uniform(-1.0, 1.0, size=n_problems)
    br = rng.uniform(-1.0, 1.0, size=n_problems)
    padded = ((n + align - 1) // align) * align
    offsets = np.zeros(n_problems, dtype=np.int64)
    offsets[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum())
    u0 = np.zeros(total, dtype=np.float64)
    for b in range(n_problems):
        u0[offsets[b]:offsets[b] + n[b]] = fourier_state(int(n[b]), bl[b], br[b], rng)
    return Batch(n=n, r=r, beta_l=bl, beta_r=br, offsets=offsets, u0=u0, total=total)


@dataclass
class SurrogateProblems:
    """Equal-size problems for the learned surrogate: ``u0`` is [P, n]."""
    u0: np.ndarray
    r: np.ndarray
    beta_l: np.ndarray
    beta_r: np.ndarray


def surrogate_problems(n_problems: int, n: int = 1024, seed: int = SEED_BASE + 4, r_min: float = 0.5,
                       r_max: float = 4.0, n_modes: int = 16, n_tents: int = 2) -> SurrogateProblems:
    """P problems on n points: r ~ U[r_min, r_max], walls ~ U(-1, 1), u0 = the
    linear profile between the walls + sum_{k<=n_modes} a_k / k^2 sin(k pi x)
    (a_k ~ N(0, 1)) + `n_tents` piecewise-linear tents c (1 - |x - x_c| / w)_+
    with x_c ~ U(0.1, 0.9), w ~ U(0.02, 0.2), c ~ N(0, 0.5^2)."""
    rng = np.random.default_rng(seed)
    x = grid(n)
    r = rng.uniform(r_min, r_max, n_problems)
    bl = rng.uniform(-1.0, 1.0, n_problems)
    br = rng.uniform(-1.0, 1.0, n_problems)
    k = np.arange(1, n_modes + 1, dtype=np.float64)
    basis = np.sin(np.pi * k[:, None] * x[None, :]) / (k * k)[:, None]
    u0 = rng.standard_normal((n_problems, n_modes)) @ basis
    u0 += bl[:, None] + (br - bl)[:, None] * x[None, :]
    for _ in range(n_tents):
        xc = rng.uniform(0.1, 0.9, n_problems)[:, None]
        w = rng.uniform(0.02, 0.2, n_problems)[:, None]
        c = rng.normal(0.0, 0.5, n_problems)[:, None]
        u0 += c * np.maximum(0.0, 1.0 - np.abs(x[None, :] - xc) / w)
    return SurrogateProblems(u0=u0, r=r, beta_l=bl, beta_r=br)
