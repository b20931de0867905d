"""The extended-precision reference used to attribute FP64 round-off
(tests/ext_reference.py) computes the same scheme as the oracle: short runs
agree to FP64 round-off for both parities of n, several r and wall values."""
import numpy as np
import pytest

import oracle
from ext_reference import ext_precision_run


@pytest.mark.parametrize("n", [1, 2, 3, 8, 17, 64])
@pytest.mark.parametrize("r", [0.3, 1.0, 7.5])
def test_ext_reference_matches_oracle(n, r):
    u0 = np.random.default_rng(n * 10 + int(r * 10)).standard_normal(n)
    want = oracle.run(u0, r, 0.7, -0.4, 25)
    got = ext_precision_run(u0, r, 0.7, -0.4, 25).astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, 2 * r - 1) * max(1.0, np.max(np.abs(want)))
