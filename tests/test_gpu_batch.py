"""Batched solves (many uneven problems in one packed buffer) against the
CPU oracle, problem by problem.  Tolerances as in test_gpu_parity: FP64
1e-12 relative max-norm for r <= 4 (tests/tolerances.py), FP32 1e-5 (the
batched FP32 target), per problem."""
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


def tol(prec, r):
    return tol64(r) if prec == B.GE_F64 else 1e-5


def rel(got, want):
    return float(np.max(np.abs(got - want)) / max(1e-300, np.max(np.abs(want))))


def layout(ns, align=32, gap=0):
    offs, pos = [], 0
    for n in ns:
        offs.append(pos)
        pos += ((n + align - 1) // align) * align + gap
    return np.array(offs, dtype=np.int64), pos


def make_batch(ns, seed, r_lo=0.2, r_hi=5.0, gap=0):
    rng = np.random.default_rng(seed)
    offs, total = layout(ns, gap=gap)
    r = rng.uniform(r_lo, r_hi, len(ns))
    bl, br = rng.uniform(-1, 1, len(ns)), rng.uniform(-1, 1, len(ns))
    u = np.full(total, 7.25)  # marks the gaps between problems
    for i, n in enumerate(ns):
        u[offs[i]:offs[i] + n] = inputs.fourier_state(n, bl[i], br[i], rng) + 0.01 * rng.standard_normal(n)
    return np.array(ns, dtype=np.int64), r, bl, br, offs, total, u


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


MIXED = [1, 2, 3, 5, 31, 32, 33, 64, 100, 1000, 4095, 8191, 9000, 20000, 2, 40001]


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32, B.GE_F32_COMP])
@pytest.mark.parametrize("depth", [1, 7, 64])
def test_batch_matches_oracle(prec, depth):
    n, r, bl, br, offs, total, u = make_batch(MIXED, seed=depth, gap=32)
    x = torch.from_numpy(u).to(DEV, B.dtype_of(prec))
    plan = B.ge_batch_create(n, r, bl, br, offs, total, prec)
    B.ge_batch_set_depth(plan, depth)
    B.ge_batch_run(plan, x, 77)
    B.ge_batch_sync(plan)
    got = x.double().cpu().numpy()
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 77)
        e = rel(got[offs[i]:offs[i] + n[i]], want)
        assert e <= tol(prec, r[i]), (i, n[i], r[i], e)
    # the values between problems are left as they were
    mask = np.ones(total, bool)
    for i in range(len(n)):
        mask[offs[i]:offs[i] + n[i]] = False
    assert np.all(got[mask] == np.float32(7.25))


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32])
@pytest.mark.parametrize("shape", ["one_tile", "more_tiles_than_ctas"])
def test_batch_tile_queue_extremes(prec, shape):
    """The launch's tile queue at its ends: a batch that is one tile (grid of
    one CTA), and one with more tiles than the persistent grid has CTAs
    (every CTA takes several from the queue).  97 steps at depth 96: a launch
    with the entry and 95 mid steps, then one with the last mid step and the
    exit."""
    ns = [5] if shape == "one_tile" else [8190] * 300  # 2.46e6 points: > 304 tiles of 6656 FP32 points
    n, r, bl, br, offs, total, u = make_batch(ns, seed=31)
    x = torch.from_numpy(u).to(DEV, B.dtype_of(prec))
    plan = B.ge_batch_create(n, r, bl, br, offs, total, prec)
    B.ge_batch_set_depth(plan, 96)
    B.ge_batch_run(plan, x, 97)
    B.ge_batch_sync(plan)
    B.ge_batch_destroy(plan)
    got = x.double().cpu().numpy()
    picks = sorted({0, len(ns) - 1, len(ns) // 2, len(ns) // 3, 2 * len(ns) // 3})
    for i in picks:
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 97)
        e = rel(got[offs[i]:offs[i] + n[i]], want)
        assert e <= tol(prec, r[i]), (i, e)
    # every problem moved (none was skipped by the queue), and padding is untouched
    for i in range(len(ns)):
        assert not np.array_equal(got[offs[i]:offs[i] + n[i]], u[offs[i]:offs[i] + n[i]].astype(got.dtype)), i
    mask = np.ones(total, bool)
    for i in range(len(n)):
        mask[offs[i]:offs[i] + n[i]] = False
    assert np.all(got[mask] == np.float32(7.25))


def test_one_shot_equals_plan_and_zero_steps():
    n, r, bl, br, offs, total, u = make_batch([300, 5000, 777], seed=3)
    a = torch.from_numpy(u).to(DEV)
    b = a.clone()
    status = torch.full((len(n),), -1, dtype=torch.int32, device=DEV)
    B.ge_solve_batch(n, r, bl, br, offs, total, a, 50, B.GE_F64, status=status)
    assert status.cpu().tolist() == [B.GE_OK] * len(n)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64)
    B.ge_batch_run(plan, b, 0)
    B.ge_batch_sync(plan)
    assert torch.equal(b, torch.from_numpy(u).to(DEV))
    B.ge_batch_run(plan, b, 50)
    B.ge_batch_sync(plan)
    assert torch.equal(a, b)


def test_tune_keeps_results():
    n, r, bl, br, offs, total, u = make_batch([2000, 30000, 50, 9000], seed=4)
    x = torch.from_numpy(u).to(DEV, torch.float32)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F32)
    best = B.ge_batch_tune(plan, x, 128)
    assert best in (16, 32, 48, 64, 96, 128, 192, 256)
    assert B.ge_batch_get_depth(plan) == best
    assert torch.equal(x, torch.from_numpy(u).to(DEV, torch.float32))  # tuning does not touch u
    B.ge_batch_run(plan, x, 300)
    B.ge_batch_sync(plan)
    got = x.double().cpu().numpy()
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 300)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= 1e-5


def test_graph_capture_of_a_batch_run():
    n, r, bl, br, offs, total, u = make_batch([1500, 6000, 123, 20000], seed=5)
    x = torch.from_numpy(u).to(DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64, stream=s)
        B.ge_batch_set_depth(plan, 32)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            B.ge_batch_run(plan, x, 100)
        g.replay()
        g.replay()
    B.ge_batch_sync(plan)
    got = x.cpu().numpy()
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 100)
        want = oracle.run(want, r[i], bl[i], br[i], 100)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol(B.GE_F64, r[i])


@pytest.mark.parametrize("prec", [B.GE_F32, B.GE_F32_COMP, B.GE_F64])
def test_uneven_batch_full_size_sampled(prec):
    """4096 problems, N log-uniform in [256, 65536], r in [0.25, 4], 2000
    steps (the batched workload); eight problems checked against the oracle."""
    bt = inputs.uneven_batch()
    x = torch.from_numpy(bt.u0).to(DEV, B.dtype_of(prec))
    plan = B.ge_batch_create(bt.n, bt.r, bt.beta_l, bt.beta_r, bt.offsets, bt.total, prec)
    B.ge_batch_run(plan, x, 2000)
    B.ge_batch_sync(plan)
    got = x.double().cpu().numpy()
    rng = np.random.default_rng(7)
    picks = list(rng.choice(len(bt.n), 6, replace=False)) + [int(np.argmin(bt.n)), int(np.argmax(bt.n))]
    for i in picks:
        o, n = bt.offsets[i], bt.n[i]
        want = oracle.run(bt.u0[o:o + n], bt.r[i], bt.beta_l[i], bt.beta_r[i], 2000)
        assert rel(got[o:o + n], want) <= tol(prec, bt.r[i]), (i, n, bt.r[i])


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32])
def test_end_factor_slots_exhausted_use_the_normalised_form(prec):
    """Runs of 1..70 steps: every distinct launch length takes an end-factor
    slot of the scaled form; past the 64 slots the launches fall back to the
    normalised form.  Each run starts from step counter 0."""
    n, r, bl, br, offs, total, u = make_batch([37, 200, 64, 5], seed=11)
    x = torch.from_numpy(u).to(DEV, B.dtype_of(prec))
    plan = B.ge_batch_create(n, r, bl, br, offs, total, prec)
    B.ge_batch_set_depth(plan, 128)
    want = [u[offs[i]:offs[i] + n[i]].copy() for i in range(len(n))]
    for steps in range(1, 71):
        B.ge_batch_run(plan, x, steps)
        want = [oracle.run(want[i], r[i], bl[i], br[i], steps) for i in range(len(n))]
    B.ge_batch_sync(plan)
    got = x.double().cpu().numpy()
    for i in range(len(n)):
        assert rel(got[offs[i]:offs[i] + n[i]], want[i]) <= tol(prec, r[i]), i


@pytest.mark.parametrize("prec,r_hi", [(B.GE_F64, 300.0), (B.GE_F32, 30.0)])
def test_batch_large_r_rescales_often(prec, r_hi):
    """Large mesh ratios shorten the rescaling interval of the scaled form.
    Tolerances scale with the step's max-norm 2r - 1, as for one problem
    (FP32: relative to the batched workload's r <= 4)."""
    n, r, bl, br, offs, total, u = make_batch([900, 4000, 33], seed=12, r_lo=r_hi / 2, r_hi=r_hi)
    x = torch.from_numpy(u).to(DEV, B.dtype_of(prec))
    plan = B.ge_batch_create(n, r, bl, br, offs, total, prec)
    B.ge_batch_run(plan, x, 150)
    B.ge_batch_sync(plan)
    got = x.double().cpu().numpy()
    for i in range(len(n)):
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 150)
        t = tol(prec, r[i]) if prec == B.GE_F64 else 1e-5 * max(1.0, (2 * r[i] - 1) / 7.0)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= t, (i, r[i])


def test_batch_huge_r_error_is_conditioning():
    """At r ~ 3e4 (rescaling after every block step in FP64) the scheme
    barely damps its highest mode, so every FP64 evaluation carries
    round-off of order (2r - 1) eps per step: the batched kernel stays as
    close to an extended-precision evaluation as the oracle itself."""
    n, r, bl, br, offs, total, u = make_batch([900, 33], seed=12, r_lo=2.5e4, r_hi=5.0e4)
    x = torch.from_numpy(u).to(DEV)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F64)
    B.ge_batch_run(plan, x, 100)
    B.ge_batch_sync(plan)
    got = x.cpu().numpy()
    for i in range(len(n)):
        u0 = u[offs[i]:offs[i] + n[i]]
        ref = ext_precision_run(u0, r[i], bl[i], br[i], 100).astype(np.float64)
        e_orc = rel(oracle.run(u0, r[i], bl[i], br[i], 100), ref)
        e_gpu = rel(got[offs[i]:offs[i] + n[i]], ref)
        assert e_gpu <= 4.0 * e_orc + 1e-15, (i, e_gpu, e_orc)


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32, B.GE_F32_COMP])
def test_batch_check_flags_non_finite_problems(prec):
    n, r, bl, br, offs, total, u = make_batch([100, 2000, 33, 700, 64], seed=13, gap=32)
    u = u.copy()
    u[offs[2] + 5] = np.nan
    u[offs[4] + 63] = np.inf
    x = torch.from_numpy(u).to(DEV, B.dtype_of(prec))
    plan = B.ge_batch_create(n, r, bl, br, offs, total, prec)
    B.ge_batch_run(plan, x, 20)
    status = torch.full((len(n),), -1, dtype=torch.int32, device=DEV)
    B.ge_batch_check(plan, x, status)
    B.ge_batch_sync(plan)
    assert status.cpu().tolist() == [0, 0, B.GE_ENONFINITE, 0, B.GE_ENONFINITE]
    got = x.double().cpu().numpy()
    for i in (0, 1, 3):  # the other problems are untouched by their neighbours' NaN / Inf
        want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 20)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol(prec, r[i])


@pytest.mark.parametrize("prec", [B.GE_F64, B.GE_F32, B.GE_F32_COMP])
def test_every_tile_geometry_gives_the_same_result(prec):
    """Rows per tile (256, 128) and CTAs per SM change where the tiles are
    cut and who computes them, not the arithmetic of any point: every
    geometry gives the same bits, and they match the oracle problem by
    problem."""
    n, r, bl, br, offs, total, u = make_batch(MIXED, seed=41, gap=32)
    outs = {}
    for tr in (256, 128):
        plan = B.ge_batch_create(n, r, bl, br, offs, total, prec)
        B.ge_batch_set_geometry(plan, tr, 0)
        got_tr, cmax = B.ge_batch_get_geometry(plan)
        assert got_tr == tr and cmax >= 1
        for c in sorted({1, cmax}):
            for depth in (5, 48):
                B.ge_batch_set_geometry(plan, tr, c)
                B.ge_batch_set_depth(plan, depth)
                x = torch.from_numpy(u).to(DEV, B.dtype_of(prec))
                B.ge_batch_run(plan, x, 101)
                B.ge_batch_sync(plan)
                outs[(tr, c, depth)] = x.double().cpu().numpy()
        with pytest.raises(B.GeError):
            B.ge_batch_set_geometry(plan, tr, cmax + 1)
        B.ge_batch_destroy(plan)
    ref = outs[(256, 1, 48)]
    for key, got in outs.items():
        if key[2] == 48:
            assert np.array_equal(got, ref), key
    for key in ((256, 1, 5), (128, 1, 5)):
        for i in range(len(n)):
            want = oracle.run(u[offs[i]:offs[i] + n[i]], r[i], bl[i], br[i], 101)
            assert rel(outs[key][offs[i]:offs[i] + n[i]], want) <= tol(prec, r[i]), (key, i)


def test_tune_picks_a_geometry_on_the_callers_data():
    """The autotuner searches depth and geometry on the caller's data, leaves
    the data alone, and the plan then runs at what it picked, matching the
    oracle."""
    n, r, bl, br, offs, total, u = make_batch(MIXED * 4, seed=42)
    x = torch.from_numpy(u).to(DEV, torch.float32)
    before = x.clone()
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F32)
    best = B.ge_batch_tune(plan, x, 96)
    assert torch.equal(x, before)
    tr, c = B.ge_batch_get_geometry(plan)
    assert best == B.ge_batch_get_depth(plan) and tr in (128, 256) and c >= 1
    B.ge_batch_run(plan, x, 60)
    B.ge_batch_sync(plan)
    got = x.double().cpu().numpy()
    B.ge_batch_destroy(plan)
    for i in range(len(n)):
        start = u[offs[i]:offs[i] + n[i]].astype(np.float32).astype(np.float64)
        want = oracle.run(start, r[i], bl[i], br[i], 60)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol(B.GE_F32, r[i]), i


@pytest.mark.parametrize("tile_rows", [256, 128])
@pytest.mark.parametrize("depth,steps", [(7, 301), (48, 2000), (96, 97)])
def test_persistent_launch_gives_the_per_launch_bits(tile_rows, depth, steps):
    """A plain FP32 run as one persistent launch (rounds of `depth` steps,
    tiles of a round waiting on their neighbours of the round before) gives
    the same bits as one launch per round, and matches the oracle."""
    n, r, bl, br, offs, total, u = make_batch(MIXED * 3, seed=43 + depth, gap=32)
    plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F32)
    B.ge_batch_set_geometry(plan, tile_rows, 0)
    B.ge_batch_set_depth(plan, depth)
    outs = []
    for persist in (0, 1):
        B.ge_batch_set_persistent(plan, persist)
        assert B.ge_batch_get_persistent(plan) == persist
        x = torch.from_numpy(u).to(DEV, torch.float32)
        B.ge_batch_run(plan, x, steps)
        B.ge_batch_sync(plan)
        outs.append(x.double().cpu().numpy())
    B.ge_batch_destroy(plan)
    assert np.array_equal(outs[0], outs[1])
    got = outs[1]
    for i in range(len(n)):
        start = u[offs[i]:offs[i] + n[i]].astype(np.float32).astype(np.float64)
        want = oracle.run(start, r[i], bl[i], br[i], steps)
        assert rel(got[offs[i]:offs[i] + n[i]], want) <= tol(B.GE_F32, r[i]), i


def test_persistent_launch_in_a_graph():
    """Captured into a CUDA graph, a persistent run is its counter resets and
    one launch; replays give the direct run's bits."""
    n, r, bl, br, offs, total, u = make_batch(MIXED * 2, seed=44)
    u0 = torch.from_numpy(u).to(DEV, torch.float32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = B.ge_batch_create(n, r, bl, br, offs, total, B.GE_F32, stream=s)
        B.ge_batch_set_depth(plan, 32)
        B.ge_batch_set_persistent(plan, 1)
        a = u0.clone()
        B.ge_batch_run(plan, a, 200)
        x = u0.clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            x.copy_(u0)
            B.ge_batch_run(plan, x, 200)
        g.replay()
        g.replay()
    B.ge_batch_sync(plan)
    B.ge_batch_destroy(plan)
    assert torch.equal(a, x)
