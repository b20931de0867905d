"""The CPU oracle pinned to the paper and the mathematics (no GPU)."""
import numpy as np
import pytest

import oracle_pins as P


@pytest.mark.parametrize("name", sorted(P.PINS))
def test_pin(orc, name):
    fn, tol = P.PINS[name]
    dev = fn(orc)
    assert dev <= tol, f"pin {name}: deviation {dev:.3e} > {tol:.1e}"


def test_composition_carries_parity(orc):
    """run(a) then run(b) from step counter a == run(a + b), bit for bit."""
    rng = np.random.default_rng(3)
    for n in (7, 10):
        u = rng.standard_normal(n)
        for a, b in ((3, 4), (1, 6), (0, 7), (4, 3)):
            one = orc.run(orc.run(u, 2.5, 0.1, -0.2, a), 2.5, 0.1, -0.2, b, step0=a)
            both = orc.run(u, 2.5, 0.1, -0.2, a + b)
            assert np.array_equal(one, both)


def test_parity_follows_global_counter(orc):
    """An odd starting counter begins with the parity-1 groups."""
    u = np.random.default_rng(4).standard_normal(9)
    assert np.array_equal(orc.run(u, 1.5, 0.0, 0.0, 1, step0=5), orc.step(u, 1.5, 0.0, 0.0, 1))
    assert np.array_equal(orc.run(u, 1.5, 0.0, 0.0, 1, step0=6), orc.step(u, 1.5, 0.0, 0.0, 0))


def test_window_sample_matches_full_grid(orc):
    """Windowed evaluation (used for full-size parity samples) equals the full
    grid: the dependency cone of S steps is S+1 points wide."""
    rng = np.random.default_rng(5)
    n, steps = 3001, 200
    u0 = rng.standard_normal(n)
    full = orc.run(u0, 3.0, 0.4, -0.6, steps, step0=1)
    idx = [0, 1, 2, 150, 999, 1500, 2998, 2999, 3000]
    got = orc.sample(u0, 3.0, 0.4, -0.6, steps, idx, step0=1)
    assert np.array_equal(got, full[idx])


def test_cone_width_is_steps_plus_one(orc):
    """A unit impulse spreads exactly S+1 points to each side in S steps."""
    n = 301
    for steps in (1, 2, 5, 16, 33):
        for j in (150, 151):
            e = np.zeros(n)
            e[j] = 1.0
            out = orc.run(e, 1.7, 0.0, 0.0, steps)
            nz = np.nonzero(out)[0]
            assert j - nz.min() <= steps + 1 and nz.max() - j <= steps + 1
            assert max(j - nz.min(), nz.max() - j) == steps + 1


def test_invalid_arguments_rejected(orc):
    with pytest.raises(ValueError):
        orc.step(np.zeros(0), 1.0, 0.0, 0.0, 0)
    with pytest.raises(ValueError):
        orc.step(np.zeros(4), -1.0, 0.0, 0.0, 0)
    with pytest.raises(ValueError):
        orc.step(np.zeros(4), float("nan"), 0.0, 0.0, 0)
    with pytest.raises(ValueError):
        orc.step(np.zeros(4), 1.0, 0.0, 0.0, 2)
    with pytest.raises(ValueError):
        orc.run(np.zeros(4), 1.0, 0.0, 0.0, -1)
    with pytest.raises(ValueError):
        orc.run_periodic(np.zeros(5), 1.0, 2)


def test_zero_steps_is_identity(orc):
    u = np.random.default_rng(6).standard_normal(11)
    assert np.array_equal(orc.run(u, 1.0, 1.0, 2.0, 0), u)
