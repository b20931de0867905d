"""The batched solve of FP64 plans in double-float arithmetic
(ge_batch_set_kernel with GE_KERNEL_TEMPORAL_DF) against the CPU oracle,
problem by problem, at the FP64 tolerance 1e-12 * max(1, 2r - 1) relative
max-norm (as the single-problem double-float kernel, tests/test_gpu_df.py)."""
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




def rel(got, want):
    return float(np.max(np.abs(got - want)) / max(1e-300, np.max(np.abs(want))))


def layout(ns, align=16, gap=0):
    offs, pos = [], 0
    for n in ns:
        offs.append(pos)
        pos += ((n + align - 1) // align) * align + gap
    return np.array(offs, dtype=np.int64), pos


def make_batch(ns, seed, r_lo=0.2, r_hi=5.0, gap=0, scale=1.0):
    rng = np.random.default_rng(seed)
    offs, total = layout(ns, gap=gap)
    r = rng.uniform(r_lo, r_hi, len(ns))
    bl, br = rng.uniform(-1, 1, len(ns)) * scale, rng.uniform(-1, 1, len(ns)) * scale
    u = np.full(total, 7.25 + 1e-13)  # marks the gaps between problems (not a float pair)
    for i, n in enumerate(ns):
        u[offs[i]:offs[i] + n] = (inputs.fourier_state(n, bl[i] / scale, br[i] / scale, rng)
                                  + 0.01 * rng.standard_normal(n)) * scale
    return np.array(ns, dtype=np.int64), r, bl, br, offs, total, u


def run_df(n, r, bl, br, offs, total, u, steps, depth=0):
    x = torch.from_numpy(u).to(DEV)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64)
    B.ge_batch_set_kernel(plan, DF)
    if depth:
        B.ge_batch_set_depth(plan, depth)
    B.ge_batch_run(plan, x, steps)
    B.ge_batch_sync(plan)
    B.ge_batch_destroy(plan)
    return x.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


MIXED = [1, 2, 3, 5, 15, 16, 17, 31, 32, 33, 64, 100, 1000, 4095, 8191, 9000, 20000, 2, 40001]


@pytest.mark.parametrize("depth", [1, 7, 64, 200])
def test_batch_df_matches_oracle(depth):
    n, r, bl, br, offs, total, u = make_batch(MIXED, seed=depth, gap=16)
    got = run_df(n, r, bl, br, offs, total, u, 77, depth)
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 77)
        e = rel(got[offs[i]:offs[i] + n[i]], want)
        assert e <= tol64(r[i]), (i, n[i], r[i], e)
    # the values between problems come back bit for bit
    mask = np.ones(total, bool)
    for i in range(len(n)):
        mask[offs[i]:offs[i] + n[i]] = False
    assert np.all(got[mask] == u[mask])


@pytest.mark.parametrize("scale", [2.0 ** -700, 2.0 ** -300, 2.0 ** 300, 2.0 ** 700])
def test_batch_df_prescale_per_problem(scale):
    """Problems far outside the FP32 exponent range, each with its own
    magnitude: the per-problem prescale brings them in."""
    ns = [100, 5000, 33, 2048]
    n, r, bl, br, offs, total, u = make_batch(ns, seed=5, scale=scale)
    # a second magnitude in the same batch
    u[offs[1]:offs[1] + ns[1]] *= 2.0 ** 40
    bl[1] *= 2.0 ** 40
    br[1] *= 2.0 ** 40
    got = run_df(n, r, bl, br, offs, total, u, 150)
    assert np.all(np.isfinite(got))
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 150)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol64(r[i]), i


def test_batch_df_long_run_and_split_calls():
    """2000 steps in calls of several lengths (each call prescales afresh,
    parity carries through the step counter of the calls' sum) against an
    extended-precision evaluation of each problem."""
    ns = [512, 4096, 1000]
    n, r, bl, br, offs, total, u = make_batch(ns, seed=9, r_lo=0.3, r_hi=1.7)
    x = torch.from_numpy(u).to(DEV)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64)
    B.ge_batch_set_kernel(plan, DF)
    for s in (1000, 1000):
        B.ge_batch_run(plan, x, s)
    B.ge_batch_sync(plan)
    B.ge_batch_destroy(plan)
    got = x.cpu().numpy()
    for i in range(len(n)):
        ref = ext_precision_run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 2000).astype(np.float64)
        e = rel(got[offs[i]:offs[i] + n[i]], ref)
        assert e <= tol64(r[i]), (i, e)


def test_batch_df_switch_back_and_forth():
    """The plan's scaled form is re-planned when the kernel changes; FP64 and
    double-float runs of the same plan both match the oracle."""
    n, r, bl, br, offs, total, u = make_batch([3000, 77, 10001], seed=11)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64)
    for kern in (DF, B.GE_KERNEL_TEMPORAL, DF):
        B.ge_batch_set_kernel(plan, kern)
        x = torch.from_numpy(u).to(DEV)
        B.ge_batch_run(plan, x, 90)
        B.ge_batch_sync(plan)
        got = x.cpu().numpy()
        for i in range(len(n)):
            want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 90)
            assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol64(r[i]), (kern, i)
    B.ge_batch_destroy(plan)


def test_batch_df_graph_capture():
    n, r, bl, br, offs, total, u = make_batch([2000, 500, 7000], seed=13)
    x = torch.from_numpy(u).to(DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64, stream=s)
        B.ge_batch_set_kernel(plan, DF)
        B.ge_batch_set_depth(plan, 32)
        B.ge_batch_run(plan, x, 64)  # fills the end-factor slots outside the capture
        x.copy_(torch.from_numpy(u).to(DEV))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            B.ge_batch_run(plan, x, 64)
        x.copy_(torch.from_numpy(u).to(DEV))
        g.replay()
    B.ge_batch_sync(plan)
    got = x.cpu().numpy()
    B.ge_batch_destroy(plan)
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 64)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol64(r[i])


def test_batch_df_settings_rejected():
    n, r, bl, br, offs, total, u = make_batch([100, 200], seed=1)
    offs32, total32 = layout([100, 200], align=32)  # FP32 rows hold 32 values
    plan = B.ge_batch_create(n, r, bl, br, offs32, total32, B.GE_F32)
    with pytest.raises(B.GeError):
        B.ge_batch_set_kernel(plan, DF)
    B.ge_batch_destroy(plan)
    plan = B.ge_batch_create(n, np.array([1.0, 3.0e6]), bl, br, offs, total, B.GE_F64)
    with pytest.raises(B.GeError):
        B.ge_batch_set_kernel(plan, DF)
    with pytest.raises(B.GeError):
        B.ge_batch_set_kernel(plan, B.GE_KERNEL_CANONICAL)
    B.ge_batch_destroy(plan)


def test_batch_df_full_size_sampled():
    """The batched workload (4096 problems, N log-uniform in [256, 65536],
    r in [0.25, 4], 2000 steps) on the double-float kernel; eight problems
    checked against the oracle at the FP64 tolerance."""
    bt = inputs.uneven_batch()
    x = torch.from_numpy(bt.u0).to(DEV)
    plan = B.ge_batch_create(bt.n, bt.r, bt.beta_l, bt.beta_r, bt.offsets, bt.total, B.GE_F64)
    B.ge_batch_set_kernel(plan, DF)
    B.ge_batch_run(plan, x, 2000)
    B.ge_batch_sync(plan)
    B.ge_batch_destroy(plan)
    got = x.cpu().numpy()
    rng = np.random.default_rng(7)
    picks = list(rng.choice(len(bt.n), 6, replace=False)) + [int(np.argmin(bt.n)), int(np.argmax(bt.n))]
    for i in picks:
        o, n = bt.offsets[i], bt.n[i]
        want = oracle.run(bt.u0[o:o + n], bt.r[i], bt.beta_l[i], bt.beta_r[i], 2000)
        assert rel(got[o:o + n], want) <= tol64(bt.r[i]), (i, n, bt.r[i])


def test_batch_df_end_factor_slots_are_bounded():
    """Every distinct launch length takes one of the plan's 64 end-factor
    slots; the double-float kernel has no normalised form to fall back to, so
    a run that needs a 65th length fails with GE_EINVAL and leaves the plan
    usable for the lengths it has."""
    n, r, bl, br, offs, total, u = make_batch([37, 200, 64, 5], seed=11)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64)
    B.ge_batch_set_kernel(plan, DF)
    B.ge_batch_set_depth(plan, 128)
    x = torch.from_numpy(u).to(DEV)
    failed_at = None
    for steps in range(1, 80):
        try:
            B.ge_batch_run(plan, x, steps)
        except B.GeError as err:
            assert err.status == B.GE_EINVAL
            failed_at = steps
            break
    assert failed_at is not None and failed_at > 60
    x = torch.from_numpy(u).to(DEV)
    B.ge_batch_run(plan, x, 10)
    B.ge_batch_sync(plan)
    got = x.cpu().numpy()
    B.ge_batch_destroy(plan)
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 10)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol64(r[i])
