"""ge_solve_noalloc: the tiled solve for callers that may not allocate device
memory (its working memory is a fixed array inside the library).  Its result
must match the allocating path (ge_create / ge_step_n / ge_read_state with the
same kernel and depth) within the parity tolerance, on two calls in a row,
the second on other data, so a leftover of the shared working memory would
show.  Collected last so that a stop at the first failure has run every
other test first."""
import numpy as np
import pytest
import torch

from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def tol(prec, r):
    return 1e-12 * max(1.0, 2.0 * r - 1.0) if prec == B.GE_F64 else 1e-6


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
