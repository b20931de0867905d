"""General sub-domain width k on the GPU against the oracle: FP64 bit for
bit (the sweep kernel evaluates the oracle's operations in its order), FP32
within 1e-5 relative max-norm."""
import numpy as np
import pytest
import torch

import oracle
from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def run_k(u0, r, bl, br, k, steps, prec=B.GE_F64, chunks=None, step0=0):
    x = torch.as_tensor(np.asarray(u0), dtype=B.dtype_of(prec), device=DEV).contiguous()
    ctx = B.ge_create(len(u0), r, bl, br, prec, x)
    B.ge_set_subdomain_width(ctx, k)
    if k == 1:  # width 1 runs the chosen k = 1 kernel; the canonical one is bit-exact
        B.ge_set_kernel(ctx, B.GE_KERNEL_CANONICAL, 0)
    if step0:
        B.ge_write_state(ctx, x, step0)
    for s in (chunks or [steps]):
        B.ge_step_n(ctx, s)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 16, 33])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 17, 31, 32, 33, 64, 100, 1001])
@pytest.mark.parametrize("step0", [0, 1])
def test_subdomain_f64_bitwise(k, n, step0):
    u0 = np.random.default_rng(n * 100 + k).standard_normal(n)
    want = oracle.run_k(u0, 1.6, 0.4, -0.3, k, 9, step0=step0)
    got = run_k(u0, 1.6, 0.4, -0.3, k, 9, step0=step0)
    assert np.array_equal(got, want)


def test_paper_setup_sdc32():
    """The paper's experiments: sub-domain couples of 32 nodes (k = 16),
    M = 8208 (n = 8207 interior points), a few hundred time steps."""
    n, k = 8207, 16
    u0 = inputs.sine_state(n)
    want = oracle.run_k(u0, 1.0, 0.0, 0.0, k, 300)
    assert np.array_equal(run_k(u0, 1.0, 0.0, 0.0, k, 300), want)
    got32 = run_k(u0.astype(np.float32), 1.0, 0.0, 0.0, k, 300, prec=B.GE_F32)
    assert np.max(np.abs(got32 - want)) / np.max(np.abs(want)) <= 1e-5


@pytest.mark.parametrize("k", [2, 7, 16])
def test_subdomain_f32_and_split_calls(k):
    n = 50001
    u0 = inputs.fourier_state(n, 0.2, -0.4, np.random.default_rng(k))
    want = oracle.run_k(u0, 2.5, 0.2, -0.4, k, 101)
    got = run_k(u0, 2.5, 0.2, -0.4, k, 101, chunks=[3, 50, 48])
    assert np.array_equal(got, want)
    got32 = run_k(u0.astype(np.float32), 2.5, 0.2, -0.4, k, 101, prec=B.GE_F32)
    assert np.max(np.abs(got32 - want)) / np.max(np.abs(want)) <= 1e-5


def test_subdomain_width_checks():
    ctx = B.ge_create(16, 1.0, 0.0, 0.0, B.GE_F32_COMP)
    with pytest.raises(B.GeError):
        B.ge_set_subdomain_width(ctx, 4)
    B.ge_destroy(ctx)
    ctx = B.ge_create(16, 1.0, 0.0, 0.0, B.GE_F64)
    with pytest.raises(B.GeError):
        B.ge_set_subdomain_width(ctx, 0)
    B.ge_destroy(ctx)


@pytest.mark.parametrize("k,n", [(200, 6001), (500, 6001), (2000, 9000), (33, 70001)])
def test_subdomain_wide_and_many_units(k, n):
    """Wide sub-domains (fewer units per CTA in shared memory, or the
    unstaged kernel once 32 units no longer fit) and many CTAs."""
    u0 = np.random.default_rng(k + n).standard_normal(n)
    for step0 in (0, 1):
        want = oracle.run_k(u0, 0.7, -0.2, 0.9, k, 5, step0=step0)
        assert np.array_equal(run_k(u0, 0.7, -0.2, 0.9, k, 5, step0=step0), want)
