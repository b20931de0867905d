"""The seeded input generators against the workload recipes they stand for
(no GPU): shapes, ranges, determinism, the batch layout the library
requires, and the structure of each initial state."""
import numpy as np

from paper_1310_3422_gb300 import inputs


def test_grid_and_sine_state():
    x = inputs.grid(7)
    assert np.allclose(x, np.arange(1, 8) / 8.0)
    # sin(pi x) vanishes at the walls and peaks at the middle node
    u = inputs.sine_state(7)
    assert np.isclose(u[3], 1.0) and np.allclose(u, u[::-1])


def test_sine_modes_state_is_seeded_and_chunk_independent():
    a = inputs.sine_modes_state(10000)
    b = inputs.sine_modes_state(10000, chunk=999)  # chunking does not change the values
    assert np.array_equal(a, b)
    assert np.array_equal(a, inputs.sine_modes_state(10000))
    # eight modes with |A| <= 1: bounded by 8, zero at the walls (extrapolated)
    assert np.max(np.abs(a)) <= 8.0
    # the state lies in the span of sin(k pi x), k = 1..64: the discrete sine
    # transform has at most 8 non-negligible coefficients, all with k <= 64
    n = 1023
    u = inputs.sine_modes_state(n)
    x = inputs.grid(n)
    k = np.arange(1, n + 1)
    coef = (2.0 / (n + 1)) * np.sin(np.pi * np.outer(k, x)) @ u
    big = np.nonzero(np.abs(coef) > 1e-9)[0] + 1
    assert 1 <= big.size <= 8 and big.max() <= 64
    assert np.all(np.abs(coef[big - 1]) <= 1.0 + 1e-9)


def test_fourier_state_meets_the_walls():
    rng = np.random.default_rng(5)
    n, bl, br = 513, 0.3, -0.7
    u = inputs.fourier_state(n, bl, br, rng)
    # the sine series vanishes at x = 0 and 1, so the state extends to the wall values
    h = 1.0 / (n + 1)
    assert abs(2 * u[0] - u[1] - bl) < 50 * h * h * 16 and abs(2 * u[-1] - u[-2] - br) < 50 * h * h * 16
    # 16 modes with 1/k^2 decay: the residual after the linear profile is smooth and bounded
    lin = bl + (br - bl) * inputs.grid(n)
    assert np.max(np.abs(u - lin)) < 6.0


def test_uneven_batch_recipe_and_layout():
    bt = inputs.uneven_batch()
    assert bt.n.size == 4096
    assert np.all(bt.n % 2 == 0) and bt.n.min() >= 256 and bt.n.max() <= 65536
    assert 4.5e7 < bt.n.sum() < 5.1e7  # log-uniform mean (65536 - 256) / ln(256) = 11.8e3 per problem
    assert np.all((bt.r >= 0.25) & (bt.r <= 4.0))
    assert np.all(np.abs(bt.beta_l) <= 1.0) and np.all(np.abs(bt.beta_r) <= 1.0)
    # every problem starts on its own 128-byte row in FP32 and FP64 and the packing has no overlap
    assert np.all(bt.offsets % 32 == 0)
    assert np.all(bt.offsets[1:] >= bt.offsets[:-1] + bt.n[:-1])
    assert bt.total >= bt.offsets[-1] + bt.n[-1] and bt.u0.size == bt.total
    # log-uniform: about half the problems below the geometric mean sqrt(256 * 65536) = 4096
    frac = np.mean(bt.n < 4096)
    assert 0.45 < frac < 0.55
    # padding between problems is zero; each problem starts near its left wall value
    mask = np.ones(bt.total, bool)
    for o, n in zip(bt.offsets, bt.n):
        mask[o:o + n] = False
    assert np.all(bt.u0[mask] == 0.0)
    b = 17
    o = bt.offsets[b]
    assert abs(bt.u0[o] - bt.beta_l[b]) < 0.05
    # determinism
    bt2 = inputs.uneven_batch()
    assert np.array_equal(bt.u0, bt2.u0) and np.array_equal(bt.r, bt2.r)


def test_surrogate_problems_recipe():
    sp = inputs.surrogate_problems(300)
    assert sp.u0.shape == (300, 1024)
    assert np.all((sp.r >= 0.5) & (sp.r <= 4.0))
    assert np.all(np.abs(sp.beta_l) <= 1.0) and np.all(np.abs(sp.beta_r) <= 1.0)
    assert np.array_equal(sp.u0, inputs.surrogate_problems(300).u0)
    # without tents the state is the wall profile plus a 16-mode series: tents add
    # kinks, so the second differences of some rows are far larger than the series allows
    d2 = np.abs(np.diff(sp.u0, 2, axis=1)).max(axis=1)
    h = 1.0 / 1025
    series_bound = (np.pi * h) ** 2 * 16 * 4.0  # sum_k |a_k| / k^2 * (k pi h)^2 with |a_k| <= 4
    assert np.mean(d2 > series_bound) > 0.5
