"""Failure detection on the GPU without a GPU fault.  The diagnostic stall
makes every tile-load wait of the tiled kernels poll a barrier that nothing
arrives on: the wait runs out after a few microseconds, the kernel records
GE_ETIMEOUT, lets its own TMA copies land and returns.  The host reads the
status; the context (or plan) stays usable, and a normal run afterwards is
correct."""
import numpy as np
import pytest
import torch

import oracle
from tolerances import tol64
from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
STALL_CYCLES = 20000  # about 10 us of SM clock


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


@pytest.mark.parametrize("prec,kernel", [(B.GE_F64, B.GE_KERNEL_TEMPORAL), (B.GE_F32, B.GE_KERNEL_TEMPORAL),
                                          (B.GE_F32_COMP, B.GE_KERNEL_TEMPORAL),
                                          (B.GE_F64, B.GE_KERNEL_TEMPORAL_DF)])
def test_tiled_timeout_is_reported_and_the_context_recovers(prec, kernel):
    n, steps, r = (1 << 20) + 13, 100, 1.5
    u0 = inputs.random_state(n, seed=21)
    x = torch.tensor(u0, dtype=B.dtype_of(prec), device=DEV)
    ctx = B.ge_create(n, r, 0.2, -0.1, prec, x)
    B.ge_set_kernel(ctx, kernel, 0)
    B.ge_debug_stall(ctx, STALL_CYCLES)
    B.ge_step_n(ctx, steps)
    with pytest.raises(B.GeError) as err:
        B.ge_sync(ctx)
    assert err.value.status == B.GE_ETIMEOUT
    with pytest.raises(B.GeError):  # stays reported: the state is not valid
        B.ge_sync(ctx)
    B.ge_debug_stall(ctx, 0)
    B.ge_write_state(ctx, x, 0)  # a new state clears the failure
    B.ge_step_n(ctx, steps)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    idx = np.linspace(0, n - 1, 9).astype(np.int64)
    want = oracle.sample(u0 if prec == B.GE_F64 else u0.astype(np.float32).astype(np.float64), r, 0.2, -0.1,
                         steps, idx)
    got = out.double().cpu().numpy()[idx]
    tol = tol64(r) if prec == B.GE_F64 else 1e-5
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("kind", ["f64", "f32", "f32c", "f64_df"])
def test_batch_timeout_is_reported_and_cleared(kind):
    """Every batched kernel: FP64, the warp-specialised FP32 kernel (its
    producer and consumer waits), compensated FP32 and double-float."""
    prec = {"f64": B.GE_F64, "f32": B.GE_F32, "f32c": B.GE_F32_COMP, "f64_df": B.GE_F64}[kind]
    ns = np.array([3000, 100000, 77], dtype=np.int64)
    offs = np.array([0, 3008, 103008], dtype=np.int64)  # 128-byte rows in both precisions
    total = 103008 + 96
    rng = np.random.default_rng(22)
    r, bl, br = rng.uniform(0.5, 3.0, 3), rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    u = np.zeros(total)
    for i in range(3):
        u[offs[i]:offs[i] + ns[i]] = inputs.fourier_state(int(ns[i]), bl[i], br[i], rng)
    if prec != B.GE_F64:
        u = u.astype(np.float32).astype(np.float64)
    plan = B.ge_batch_create(ns, r, bl, br, offs, total, prec)
    if kind == "f64_df":
        B.ge_batch_set_kernel(plan, B.GE_KERNEL_TEMPORAL_DF)
    x = torch.tensor(u, dtype=B.dtype_of(prec), device=DEV)
    B.ge_batch_debug_stall(plan, STALL_CYCLES)
    B.ge_batch_run(plan, x, 60)
    with pytest.raises(B.GeError) as err:
        B.ge_batch_sync(plan)
    assert err.value.status == B.GE_ETIMEOUT
    B.ge_batch_debug_stall(plan, 0)
    x = torch.tensor(u, dtype=B.dtype_of(prec), device=DEV)
    B.ge_batch_run(plan, x, 60)
    B.ge_batch_sync(plan)  # cleared after being reported once
    got = x.double().cpu().numpy()
    for i in range(3):
        want = oracle.run(u[offs[i]:offs[i] + ns[i]], r[i], bl[i], br[i], 60)
        e = np.max(np.abs(got[offs[i]:offs[i] + ns[i]] - want)) / np.max(np.abs(want))
        assert e <= (1e-12 * max(1.0, 2 * r[i] - 1) if prec == B.GE_F64 else 1e-5), (kind, i, e)
    B.ge_batch_destroy(plan)


def test_debug_stall_rejects_bad_arguments():
    ctx = B.ge_create(64, 1.0, 0.0, 0.0, B.GE_F64)
    with pytest.raises(B.GeError):
        B.ge_debug_stall(ctx, -1)
    B.ge_destroy(ctx)
