"""Pins of the surrogate's CPU reference (oracle/sno.py) against facts that do
not come from it: the DFT written out as sums, finite differences, the exact
(erf) GELU, and the definition of BF16 rounding."""
import math

import numpy as np
import pytest
import torch

from oracle import sno as S

ARCH = S.Arch(n=16, width=3, modes=4, layers=2, hidden=5)


def random_params(a: S.Arch, seed: int, scale: float = 0.5) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(S.num_params(a)) * scale


def random_inputs(a: S.Arch, batch: int, seed: int):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((batch, a.n)), rng.uniform(0.5, 4.0, batch),
            rng.uniform(-1, 1, batch), rng.uniform(-1, 1, batch))


def brute_spectral(v, Rr, Ri, modes):
    """Truncated spectral convolution with the DFT written out as sums:
    X_m[c] = sum_j v[j, c] e^{-2 pi i m j / n}, Y_m = R_m X_m,
    out_j = (1/n) (Re Y_0 + 2 sum_{m=1}^{M-1} Re(Y_m e^{2 pi i m j / n}))."""
    n, C = v.shape
    out = np.zeros((n, Rr.shape[1]))
    for m in range(modes):
        X = np.zeros(C, dtype=complex)
        for j in range(n):
            X += v[j] * complex(math.cos(2 * math.pi * m * j / n), -math.sin(2 * math.pi * m * j / n))
        Y = (Rr[m] + 1j * Ri[m]) @ X
        w = 1.0 if m == 0 else 2.0
        for j in range(n):
            out[j] += w / n * (Y * complex(math.cos(2 * math.pi * m * j / n),
                                           math.sin(2 * math.pi * m * j / n))).real
    return out


@pytest.mark.parametrize("n,C,Cout,M", [(16, 3, 3, 4), (12, 2, 2, 5), (9, 2, 2, 3)])
def test_spectral_matches_written_out_dft(n, C, Cout, M):
    rng = np.random.default_rng(n * 100 + M)
    v = rng.standard_normal((n, C))
    Rr = rng.standard_normal((M, Cout, C))
    Ri = rng.standard_normal((M, Cout, C))
    got = S.spectral(torch.tensor(v[None]), torch.tensor(Rr), torch.tensor(Ri), M)[0].numpy()
    np.testing.assert_allclose(got, brute_spectral(v, Rr, Ri, M), rtol=0, atol=1e-12)


def test_identity_modes_are_a_low_pass_projection():
    n, C, M = 32, 2, 6
    v = torch.tensor(np.random.default_rng(1).standard_normal((1, n, C)))
    eye = torch.eye(C, dtype=torch.float64).expand(M, C, C).contiguous()
    zero = torch.zeros_like(eye)
    once = S.spectral(v, eye, zero, M)
    twice = S.spectral(once, eye, zero, M)
    torch.testing.assert_close(twice, once, rtol=0, atol=1e-13)
    # a pure low mode passes unchanged, a high one is removed
    j = torch.arange(n, dtype=torch.float64)
    low = torch.cos(2 * math.pi * 3 * j / n)[None, :, None].expand(1, n, C)
    high = torch.sin(2 * math.pi * 9 * j / n)[None, :, None].expand(1, n, C)
    torch.testing.assert_close(S.spectral(low, eye, zero, M), low, rtol=0, atol=1e-13)
    assert float(S.spectral(high, eye, zero, M).abs().max()) < 1e-13


def test_gradient_matches_central_differences():
    a = ARCH
    p = random_params(a, 3)
    u0, r, bl, br = random_inputs(a, 2, 4)
    target = np.random.default_rng(5).standard_normal((2, a.n)) + 2.0
    _, g = S.loss_and_grad(p, a, u0, r, bl, br, target)

    def f(q):
        return float(S.rel_l2(torch.tensor(S.predict(q, a, u0, r, bl, br)), torch.tensor(target)).mean())

    idx = np.random.default_rng(6).choice(p.size, 40, replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        e = np.zeros_like(p)
        e[i] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_tanh_gelu_is_close_to_the_exact_gelu():
    x = torch.linspace(-8, 8, 4001, dtype=torch.float64)
    exact = 0.5 * x * (1 + torch.erf(x / math.sqrt(2.0)))
    assert float((S.gelu(x) - exact).abs().max()) < 1e-3
    assert float(S.gelu(torch.tensor(0.0, dtype=torch.float64))) == 0.0


def test_rel_l2_definition():
    rng = np.random.default_rng(7)
    y = torch.tensor(rng.standard_normal((3, 10)))
    p = torch.tensor(rng.standard_normal((3, 10)))
    assert float(S.rel_l2(y, y).abs().max()) == 0.0
    torch.testing.assert_close(S.rel_l2(3.5 * p, 3.5 * y), S.rel_l2(p, y))
    want = np.linalg.norm(p.numpy() - y.numpy(), axis=1) / np.linalg.norm(y.numpy(), axis=1)
    np.testing.assert_allclose(S.rel_l2(p, y).numpy(), want, rtol=1e-15)


def test_round_bf16_is_nearest_bf16():
    x = np.random.default_rng(8).standard_normal(10000) * np.exp(np.random.default_rng(9).uniform(-20, 20, 10000))
    x = x.astype(np.float32)
    y = S.round_bf16(torch.tensor(x)).numpy().astype(np.float32)
    assert np.all((y.view(np.uint32) & 0xFFFF) == 0)
    assert np.all(np.abs(y.astype(np.float64) - x) <= 2.0 ** -8 * np.abs(x.astype(np.float64)))
    # nearest: no other BF16 neighbour is closer
    up = (y.view(np.uint32) + 0x10000).view(np.float32).astype(np.float64)
    dn = (y.view(np.uint32) - 0x10000).view(np.float32).astype(np.float64)
    d = np.abs(y.astype(np.float64) - x)
    assert np.all(d <= np.abs(up - x)) and np.all(d <= np.abs(dn - x))


def test_param_count_and_layout():
    a = S.Arch(n=64, width=64, modes=16, layers=4, hidden=128)
    assert S.num_params(a) == 4 * 64 + 64 + 4 * (2 * 16 * 64 * 64 + 64 * 64 + 64) + 64 * 128 + 128 + 128 + 1
    w = S.unpack(torch.arange(S.num_params(ARCH), dtype=torch.float64), ARCH)
    assert float(w["lift_w"][0, 0]) == 0.0 and float(w["q2"][0]) == S.num_params(ARCH) - 1
