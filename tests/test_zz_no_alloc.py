"""ge_solve_noalloc: the tiled solve for callers that may not allocate device
memory (its working memory is a fixed array inside the library).  Its result
must match the allocating path (ge_create / ge_step_n / ge_read_state with the
same kernel and depth) within the parity tolerance, on two calls in a row,
the second on other data, so a leftover of the shared working memory would
show.  Its FP64 results are also held to the oracle itself, at the FP64
parity tolerance.  Collected last so that a stop at the first failure has
run every other test first."""
import numpy as np
import pytest
import torch

import oracle
from tolerances import tol64
from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def tol(prec, r):
    return tol64(r) if prec == B.GE_F64 else 1e-6


def allocating_path(u0, r, bl, br, prec, depth, steps):
    x = u0.clone()
    ctx = B.ge_create(x.numel(), r, bl, br, prec, x)
    B.ge_set_kernel(ctx, B.GE_KERNEL_TEMPORAL, depth)
    B.ge_step_n(ctx, steps)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32, B.GE_F32_COMP])
def test_noalloc_matches_allocating_path_twice(prec):
    dt = B.dtype_of(prec)
    cases = [(100003, 1.7, 0.25, -0.5, 0, 301, 21), (4097, 0.6, -1.0, 2.0, 7, 64, 22)]
    for n, r, bl, br, depth, steps, seed in cases:
        u0 = torch.from_numpy(inputs.fourier_state(n, bl, br, np.random.default_rng(seed))).to(DEV, dt)
        got = torch.full_like(u0, float("nan"))
        B.ge_solve_noalloc(n, r, bl, br, prec, depth, steps, u0, got)
        want = allocating_path(u0, r, bl, br, prec, depth, steps)
        g, w = got.double().cpu().numpy(), want.double().cpu().numpy()
        assert np.all(np.isfinite(g))
        err = np.max(np.abs(g - w)) / np.max(np.abs(w))
        assert err <= tol(prec, r), (prec, n, err)


def test_noalloc_rejects_sizes_beyond_its_memory():
    big = torch.zeros((1 << 20) + 1, dtype=torch.float64, device=DEV)
    with pytest.raises(B.GeError) as e:
        B.ge_solve_noalloc(big.numel(), 1.0, 0.0, 0.0, B.GE_F64, 0, 10, big, big)
    assert e.value.status == B.GE_EINVAL
    assert "1048576" in str(e.value)


def test_noalloc_f64_matches_the_oracle():
    """FP64 against the oracle directly (not only the allocating path, so an
    error in host-side bookkeeping both paths share would show)."""
    n, r, bl, br, steps = 100003, 1.7, 0.25, -0.5, 301
    u0 = inputs.fourier_state(n, bl, br, np.random.default_rng(23))
    want = oracle.run(u0, r, bl, br, steps)
    x = torch.from_numpy(u0).to(DEV)
    got = torch.full_like(x, float("nan"))
    B.ge_solve_noalloc(n, r, bl, br, B.GE_F64, 0, steps, x, got)
    g = got.cpu().numpy()
    assert np.max(np.abs(g - want)) / np.max(np.abs(want)) <= tol64(r)


def test_noalloc_at_the_size_limit():
    """n = 2^20 FP64 points fill a working buffer exactly (the second one
    then ends right at the error word): allocating path and oracle agree."""
    n, r, steps = 1 << 20, 2.0, 37
    u0 = inputs.random_state(n, seed=24)
    x = torch.from_numpy(u0).to(DEV)
    got = torch.full_like(x, float("nan"))
    B.ge_solve_noalloc(n, r, 0.5, -0.25, B.GE_F64, 16, steps, x, got)
    want = allocating_path(x, r, 0.5, -0.25, B.GE_F64, 16, steps).cpu().numpy()
    g = got.cpu().numpy()
    assert np.max(np.abs(g - want)) / np.max(np.abs(want)) <= tol64(r)
    ref = oracle.run(u0, r, 0.5, -0.25, steps)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) <= tol64(r)


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32])
def test_noalloc_zero_steps_and_in_place(prec):
    """steps = 0 copies the state; u_out may be u0 itself (in place)."""
    dt = B.dtype_of(prec)
    n, r, steps = 5001, 0.9, 50
    u0 = torch.from_numpy(inputs.random_state(n, seed=25)).to(DEV, dt)
    out = torch.full_like(u0, float("nan"))
    B.ge_solve_noalloc(n, r, 0.0, 0.0, prec, 0, 0, u0, out)
    assert torch.equal(out, u0)
    want = allocating_path(u0, r, 0.0, 0.0, prec, 0, steps)
    x = u0.clone()
    B.ge_solve_noalloc(n, r, 0.0, 0.0, prec, 0, steps, x, x)
    g, w = x.double().cpu().numpy(), want.double().cpu().numpy()
    assert np.max(np.abs(g - w)) / np.max(np.abs(w)) <= tol(prec, r)
