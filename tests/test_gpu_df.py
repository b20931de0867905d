"""Parity of the double-float tiled kernel (GE_KERNEL_TEMPORAL_DF: FP64
storage, steps evaluated as unevaluated sums of two floats on the FP32 pipes)
with the CPU oracle, through the C ABI.

Tolerance: the FP64 one (tests/tolerances.py: 1e-12 relative max-norm for
r <= 4), at the moderate r the kernel is meant for.  Its rounding unit is about 2^-48
instead of 2^-53.  Over s steps the rounding errors of a non-expansive map
add up like a random walk, about sqrt(s) * 2^-48 ~ 3.6e-13 at s = 10000.  At
very large r the conditioning of the scheme amplifies every evaluation's
rounding (the oracle's too); there the kernel is held to 64x the oracle's
own distance from an extended-precision evaluation (32x from the rounding
unit, 2x margin).
"""
import numpy as np
import pytest
import torch

import oracle
from ext_reference import ext_precision_run
from tolerances import tol64
from paper_1310_3422_gb300 import binding as B
from paper_1310_3422_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
DF = B.GE_KERNEL_TEMPORAL_DF




def rel_max(got, want):
    return float(np.max(np.abs(np.asarray(got, dtype=np.float64) - want)) / max(1e-300, np.max(np.abs(want))))


def df_run(u0, r, bl, br, steps, depth=0, chunks=None, step0=0):
    x = torch.as_tensor(np.asarray(u0, dtype=np.float64), device=DEV).contiguous()
    ctx = B.ge_create(len(u0), r, bl, br, B.GE_F64, x)
    B.ge_set_kernel(ctx, DF, depth)
    if step0:
        B.ge_write_state(ctx, x, step0)
    for s in (chunks or [steps]):
        B.ge_step_n(ctx, s)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    assert B.ge_get_step(ctx) == step0 + sum(chunks or [steps])
    B.ge_destroy(ctx)
    return out.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


SMALL_N = [1, 2, 3, 4, 5, 6, 7, 8, 15, 16, 17, 31, 32, 33, 63, 64, 65]
TILE_N = [3999, 4000, 4001, 4095, 4096, 4097, 8191, 12345]  # 4096-point tiles


@pytest.mark.parametrize("n", SMALL_N + TILE_N)
@pytest.mark.parametrize("depth", [0, 7])
def test_df_matches_oracle(n, depth):
    rng = np.random.default_rng(3000 + n)
    u0 = rng.standard_normal(n)
    want = oracle.run(u0, 1.7, -0.4, 0.9, 77)
    got = df_run(u0, 1.7, -0.4, 0.9, 77, depth=depth)
    assert rel_max(got, want) <= tol64(1.7)


@pytest.mark.parametrize("depth", [1, 2, 3, 15, 16, 17, 63, 64, 100, 255])
@pytest.mark.parametrize("step0", [0, 1])
def test_df_depths_and_parity(depth, step0):
    n = 9001
    u0 = np.random.default_rng(depth).standard_normal(n)
    want = oracle.run(u0, 0.8, 0.2, 0.5, 300, step0=step0)
    got = df_run(u0, 0.8, 0.2, 0.5, 300, depth=depth, step0=step0)
    assert rel_max(got, want) <= tol64(0.8)


@pytest.mark.parametrize("r", [0.01, 0.25, 0.5, 1.0, 2.0, 4.0])
def test_df_range_of_r(r):
    n = 5000
    u0 = inputs.random_state(n, seed=7)
    want = oracle.run(u0, r, 1.0, -1.0, 200)
    got = df_run(u0, r, 1.0, -1.0, 200)
    assert rel_max(got, want) <= tol64(r)


@pytest.mark.parametrize("r", [50.0, 1.0e4])
def test_df_large_r_error_is_conditioning(r):
    n, steps = 2000, 100
    u0 = inputs.random_state(n, seed=8)
    ref = ext_precision_run(u0, r, 1.0, -1.0, steps).astype(np.float64)
    e_orc = rel_max(oracle.run(u0, r, 1.0, -1.0, steps), ref)
    e_df = rel_max(df_run(u0, r, 1.0, -1.0, steps), ref)
    assert e_df <= 64.0 * e_orc + 1e-13, (e_df, e_orc)


@pytest.mark.parametrize("shift", [-700, -300, 300, 700])
def test_df_prescale_covers_the_double_range(shift):
    """Data and walls far outside the FP32 exponent range: the per-call
    prescale brings them in, the result scales back exactly."""
    n, r = 3001, 1.3
    u0 = np.ldexp(inputs.random_state(n, seed=17), shift)
    bl, br = np.ldexp(0.3, shift), np.ldexp(-0.6, shift)
    want = oracle.run(u0, r, bl, br, 150)
    got = df_run(u0, r, bl, br, 150)
    assert np.all(np.isfinite(got))
    assert rel_max(got, want) <= tol64(r)


def test_df_walls_only_and_zero_state():
    n = 2500
    want = oracle.run(np.zeros(n), 2.0, 1e5, -3e-3, 400)
    got = df_run(np.zeros(n), 2.0, 1e5, -3e-3, 400)
    assert rel_max(got, want) <= tol64(2.0)
    assert np.array_equal(df_run(np.zeros(n), 2.0, 0.0, 0.0, 50), np.zeros(n))


def test_df_split_calls_continue_parity():
    n = 7000
    u0 = inputs.random_state(n, seed=19)
    want = oracle.run(u0, 0.9, 0.25, -0.5, 1 + 5 + 64 + 200 + 3)
    got = df_run(u0, 0.9, 0.25, -0.5, 0, depth=48, chunks=[1, 5, 64, 200, 3])
    assert rel_max(got, want) <= tol64(0.9)


@pytest.mark.parametrize("r", [0.3, 0.7, 1.7])
def test_df_long_run_against_extended_precision(r):
    """20000 steps of a smooth state against an extended-precision
    evaluation, with g = 2r not exact in FP32 (its pair has a low part).  The
    scale bookkeeping (growth 1 + g of the pair the kernel holds) does not
    drift, and the exact summation of the low-order product terms keeps the
    rounding unbiased: the 1e-12 FP64 target holds.  (Rounding that sum in
    FP32 gave 1.7e-12 at r = 0.3, growing linearly with the steps.)"""
    n, steps = 512, 20000
    u0 = inputs.sine_state(n)
    ref = ext_precision_run(u0, r, 0.0, 0.0, steps).astype(np.float64)
    e_df = rel_max(df_run(u0, r, 0.0, 0.0, steps), ref)
    x = torch.tensor(u0, device=DEV)
    ctx = B.ge_create(n, r, 0.0, 0.0, B.GE_F64, x)
    B.ge_step_n(ctx, steps)
    B.ge_read_state(ctx, x)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    e_64 = rel_max(x.cpu().numpy(), ref)
    print(f"r={r}: double-float {e_df:.3e}, FP64 tiled {e_64:.3e}")
    assert e_df <= tol64(r), (e_df, e_64)


@pytest.mark.parametrize("r", [0.3, 0.7])
def test_df_long_run_fast_path(r):
    """As above with n = 4096: here the interior warps run the fast path
    (renormalised every second step, exact low-order product sum) and only
    the two wall warps the checked one."""
    n, steps = 4096, 20000
    u0 = inputs.sine_state(n)
    ref = ext_precision_run(u0, r, 0.0, 0.0, steps).astype(np.float64)
    e_df = rel_max(df_run(u0, r, 0.0, 0.0, steps), ref)
    print(f"fast path r={r}: double-float {e_df:.3e}")
    assert e_df <= tol64(r), e_df


def test_df_full_size_sampled():
    """N = 2^24, r = 2, 10000 steps, eight seeded sine modes: the single large
    solve the benchmark times, sampled points against the oracle on their
    dependency-cone windows."""
    n, r, steps = 1 << 24, 2.0, 10000
    u0 = inputs.sine_modes_state(n)
    got = df_run(u0, r, 0.0, 0.0, steps)
    rng = np.random.default_rng(99)
    idx = sorted(set([0, 1, 2, n // 2, n - 3, n - 2, n - 1] + list(rng.integers(0, n, 9))))
    want = oracle.sample(u0, r, 0.0, 0.0, steps, idx)
    err = np.max(np.abs(got[idx] - want)) / np.max(np.abs(u0))
    print(f"full size: double-float {err:.3e}")
    assert err <= tol64(r)
    assert np.all(np.isfinite(got))


def test_df_graph_capture_replays_the_steps():
    n = 10000
    u0 = inputs.random_state(n, seed=13)
    x = torch.from_numpy(u0).to(DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = B.ge_create(n, 1.0, 0.0, 0.0, B.GE_F64, x, stream=s)
        B.ge_set_kernel(ctx, DF, 16)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            B.ge_step_n(ctx, 64)  # prescale + 4 launches
        g.replay()
        g.replay()
        out = torch.empty_like(x)
        B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    want = oracle.run(u0, 1.0, 0.0, 0.0, 128)
    assert rel_max(out.cpu().numpy(), want) <= tol64(1.0)


def test_df_tune_picks_a_candidate_and_keeps_the_state():
    n, r = 300001, 1.3
    u0 = inputs.random_state(n, seed=31)
    x = torch.tensor(u0, device=DEV)
    ctx = B.ge_create(n, r, 0.1, 0.2, B.GE_F64, x)
    B.ge_set_kernel(ctx, DF, 0)
    best = B.ge_tune(ctx, 200)
    assert best in (32, 48, 64, 96, 128)
    assert B.ge_get_kernel(ctx) == (DF, best)
    B.ge_step_n(ctx, 57)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    idx = np.linspace(0, n - 1, 7).astype(np.int64)
    assert rel_max(out.cpu().numpy()[idx], oracle.sample(u0, r, 0.1, 0.2, 57, idx)) <= tol64(r)


def test_df_settings_rejected():
    x32 = torch.zeros(64, dtype=torch.float32, device=DEV)
    for prec in (B.GE_F32, B.GE_F32_COMP):
        ctx = B.ge_create(64, 1.0, 0.0, 0.0, prec, x32)
        with pytest.raises(B.GeError):
            B.ge_set_kernel(ctx, DF, 0)
        B.ge_destroy(ctx)
    ctx = B.ge_create(64, 2.0e6, 0.0, 0.0, B.GE_F64)
    with pytest.raises(B.GeError):
        B.ge_set_kernel(ctx, DF, 0)
    B.ge_destroy(ctx)


def test_df_timeout_is_reported_and_the_context_recovers():
    n, steps, r = (1 << 20) + 13, 100, 1.5
    u0 = inputs.random_state(n, seed=21)
    x = torch.tensor(u0, device=DEV)
    ctx = B.ge_create(n, r, 0.2, -0.1, B.GE_F64, x)
    B.ge_set_kernel(ctx, DF, 0)
    B.ge_debug_stall(ctx, 20000)
    B.ge_step_n(ctx, steps)
    with pytest.raises(B.GeError) as err:
        B.ge_sync(ctx)
    assert err.value.status == B.GE_ETIMEOUT
    B.ge_debug_stall(ctx, 0)
    B.ge_write_state(ctx, x, 0)
    B.ge_step_n(ctx, steps)
    out = torch.empty_like(x)
    B.ge_read_state(ctx, out)
    B.ge_sync(ctx)
    B.ge_destroy(ctx)
    idx = np.linspace(0, n - 1, 9).astype(np.int64)
    assert rel_max(out.cpu().numpy()[idx], oracle.sample(u0, r, 0.2, -0.1, steps, idx)) <= tol64(r)
