"""The FP64 tiled kernel computes a share of its interior updates (the scaled
block step x + g x_partner of Sec. 2) as exact FP64 multiply-adds on the
integer pipes (csrc/ge_dfma_emu.cuh).  Wherever that form reports its fast
path it must give the FP64 unit's fma bit for bit, and everywhere else the
kernel recomputes on the FP64 unit.  These inputs cover what decides the
rounding (ties, sticky bits, carries into the exponent) and the fast path's
limits (signs, cancellation, magnitude gaps, zeros, subnormals, infinities,
NaNs).  The kernel-level bit identity is covered by the full-size parity
tests; this checks the arithmetic itself on many more cases."""
import numpy as np
import pytest
import torch

from paper_1310_3422_gb300 import binding as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

# g = 2r for r of the benchmarks (0.25 .. 4, 1.7, 2) and awkward significands
G_VALUES = [4.0, 0.5, 8.0, 3.4, 2 * 0.3, 2 * 3.7, 1.0 / 3.0, 2.0000000000000004, 1.9999999999999998, 6.5]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def check(g, p, x):
    counts = torch.zeros(3, dtype=torch.int64, device=DEV)
    B.ge_emu_fma_check(g, torch.tensor(p, device=DEV), torch.tensor(x, device=DEV), counts)
    torch.cuda.synchronize()
    return counts.cpu().tolist()


def mixed_inputs(g, n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-1.0, 1.0, n)
    x = rng.uniform(-1.0, 1.0, n)
    mode = np.arange(n) % 8
    m = mode == 1  # magnitude gaps on both sides of the fast path's window
    x[m] = np.ldexp(x[m], rng.integers(-90, 90, m.sum()))
    m = mode == 2  # near cancellation: x = -g p (1 + tiny)
    x[m] = -g * p[m] * (1.0 + np.ldexp(rng.uniform(-1, 1, m.sum()), -rng.integers(1, 60, m.sum())))
    m = mode == 3  # same sign, similar size (the smooth-field case)
    x[m] = np.abs(x[m]) * np.sign(g * p[m])
    m = mode == 4  # short significands: exact sums and rounding ties
    p[m] = rng.integers(-2**20, 2**20, m.sum()) * 2.0**-20
    x[m] = rng.integers(-2**53, 2**53, m.sum()) * 2.0**-53
    m = mode == 5  # wide exponent range of both operands
    p[m] = np.ldexp(p[m], rng.integers(-500, 500, m.sum()))
    x[m] = np.ldexp(x[m], rng.integers(-500, 500, m.sum()))
    m = mode == 6  # x one ulp-scale away from -g p
    x[m] = -(g * p[m]) + np.ldexp(rng.uniform(-4, 4, m.sum()), -52) * np.abs(g * p[m])
    return p, x


@pytest.mark.parametrize("g", G_VALUES)
def test_integer_fma_matches_the_fp64_unit(g):
    p, x = mixed_inputs(g, 1 << 20, seed=int(g * 1000) % 9973)
    bad, fast, fast_add = check(g, p, x)
    assert bad == 0
    # the fast paths take most of the ordinary inputs
    assert fast > 0.4 * len(p)
    assert fast_add > 0.1 * len(p)


def test_special_values_leave_the_fast_path():
    tiny = np.nextafter(0.0, 1.0)  # smallest subnormal
    specials = [0.0, -0.0, tiny, -tiny, 2.2250738585072014e-308, np.inf, -np.inf, np.nan, 1.0, -1.0,
                1.7976931348623157e308, 1e-300]
    p = np.array([a for a in specials for _ in specials])
    x = np.array([b for _ in specials for b in specials])
    for g in (4.0, 0.5, 1e-300, 1e300):
        bad, fast, _ = check(g, p, x)
        assert bad == 0
        assert fast < len(p)  # zeros, subnormals, infinities and NaNs fall back


def test_results_near_the_range_limits():
    # products and sums that leave the normal range must fall back, the rest
    # must still match
    rng = np.random.default_rng(7)
    p = np.ldexp(rng.uniform(0.5, 1.0, 4096), rng.integers(-1030, -1000, 4096))
    x = np.ldexp(rng.uniform(-1.0, 1.0, 4096), rng.integers(-1030, -1000, 4096))
    for g in (0.5, 4.0):
        assert check(g, p, x)[0] == 0
    p = np.ldexp(rng.uniform(0.5, 1.0, 4096), rng.integers(1010, 1023, 4096))
    x = np.ldexp(rng.uniform(-1.0, 1.0, 4096), rng.integers(1010, 1023, 4096))
    for g in (0.5, 4.0, 7.9):
        assert check(g, p, x)[0] == 0


def test_share_is_reported():
    assert 0.0 <= B.ge_fp64_int_share() < 1.0


def _solve(u0, r, bl, br, steps, on, kernel, depth):
    n = len(u0)
    ctx = B.ge_create(n, r, bl, br, B.GE_F64, torch.tensor(u0, device=DEV))
    B.ge_set_kernel(ctx, kernel, depth)
    B.ge_set_int_pipes(ctx, on)
    B.ge_step_n(ctx, steps)
    out = torch.empty(n, dtype=torch.float64, device=DEV)
    B.ge_read_state(ctx, out)
    torch.cuda.synchronize()
    B.ge_destroy(ctx)
    return out.cpu().numpy()


def _initial(kind, n, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(1, n + 1) / (n + 1)
    if kind == "smooth":
        return np.sin(np.pi * x) + 0.3 * np.sin(7 * np.pi * x)
    if kind == "signs":  # a sign change between most neighbours
        return rng.standard_normal(n)
    if kind == "zeros":  # exact zeros in blocks, isolated spikes
        u = np.sin(np.pi * x)
        u[(np.arange(n) // 5000) % 3 == 1] = 0.0
        u[rng.integers(0, n, 50)] = 1e6
        return u
    # magnitudes over 400 decades, so the integer form's window is often left
    return rng.standard_normal(n) * 10.0 ** rng.uniform(-200, 200, n)


@pytest.mark.parametrize("kind", ["smooth", "signs", "zeros", "range"])
@pytest.mark.parametrize("r", [0.3, 2.0, 3.7])
@pytest.mark.parametrize("kernel,depth", [(B.GE_KERNEL_TEMPORAL, 48), (B.GE_KERNEL_TEMPORAL, 7),
                                          (B.GE_KERNEL_ONESTEP, 0)])
def test_kernel_bits_do_not_depend_on_the_integer_pipes(kind, r, kernel, depth):
    """The FP64 tiled kernel with part of its updates on the integer pipes
    and with every update on the FP64 unit: the same bits on every point,
    whatever the data do to the integer form's fast path (fallbacks for
    zeros, sign changes, magnitude gaps).  300,000 points span many tiles;
    301 steps span entry, middle and exit launches and rescalings."""
    u0 = _initial(kind, 300_000, seed=int(r * 10) + len(kind))
    steps = 301 if kernel == B.GE_KERNEL_TEMPORAL else 41
    on = _solve(u0, r, 0.25, -0.5, steps, 1, kernel, depth)
    off = _solve(u0, r, 0.25, -0.5, steps, 0, kernel, depth)
    assert np.array_equal(on.view(np.uint64), off.view(np.uint64))


def test_int_pipes_switch_rejects_bad_values():
    ctx = B.ge_create(64, 1.0, 0.0, 0.0, B.GE_F64)
    with pytest.raises(B.GeError):
        B.ge_set_int_pipes(ctx, 2)
    B.ge_destroy(ctx)
