"""Element-wise parity of the single-problem tiled kernels with the CPU oracle
at a size where the persistent grid's CTAs each take several tiles from the
launch's tile queue: n = 2^22 points make over 1000 tiles for the 304 CTAs
of a GB300 (152 SMs x 2), so every CTA runs the "take the next position and
prefetch it" path at least three times.  Each solve runs long enough to span
an entry launch, middle launches and an exit launch, and every point of the
grid is compared with a full oracle run (Sec. 2, Eqs. (cc)/(dd)).

Tolerances: FP64 storage (FP64 and double-float arithmetic) 1e-12 relative
max-norm (tests/tolerances.py; r = 2 here); FP32 and compensated FP32 1e-5
against the FP64 oracle started from the same FP32-rounded state."""
import numpy as np
import pytest
import torch

import oracle
from tolerances import tol64
from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
N = 1 << 22
R, BL, BR = 2.0, 0.3, -0.2
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def initial_state():
    rng = np.random.default_rng(2022)
    return inputs.fourier_state(N, BL, BR, rng) + 1e-3 * rng.standard_normal(N)


_want = {}


def oracle_run(u0, steps, key):
    if key not in _want:
        _want[key] = oracle.run(u0, R, BL, BR, steps)
    return _want[key]


def gpu_solve(u0, prec, kernel, depth, steps):
    x = torch.as_tensor(u0, dtype=B.dtype_of(prec), device=DEV).contiguous()
    ctx = B.ge_create(N, R, BL, BR, prec, x)
    B.ge_set_kernel(ctx, kernel, depth)
    B.ge_step_n(ctx, steps)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    return out.double().cpu().numpy()


def rel_max(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


@pytest.mark.parametrize("kernel,depth,steps", [
    (B.GE_KERNEL_TEMPORAL, 48, 200),      # the benchmark's kernel and depth: 5 launches
    (B.GE_KERNEL_TEMPORAL_DF, 96, 200),   # double-float arithmetic: 3 launches
    (B.GE_KERNEL_ONESTEP, 0, 6),          # one launch per step
])
def test_fullsize_f64_every_point(kernel, depth, steps):
    u0 = initial_state()
    want = oracle_run(u0, steps, ("f64", steps))
    got = gpu_solve(u0, B.GE_F64, kernel, depth, steps)
    assert np.all(np.isfinite(got))
    assert rel_max(got, want) <= tol64(R), rel_max(got, want)


@pytest.mark.parametrize("prec", [B.GE_F32, B.GE_F32_COMP])
def test_fullsize_f32_every_point(prec):
    steps = 300  # depth 128: entry, middle and exit launches
    u32 = initial_state().astype(np.float32)
    want = oracle_run(u32.astype(np.float64), steps, ("f32", steps))
    got = gpu_solve(u32, prec, B.GE_KERNEL_TEMPORAL, 128, steps)
    assert np.all(np.isfinite(got))
    assert rel_max(got, want) <= TOL32, rel_max(got, want)
