"""CPU FP64 reference of the spectral neural operator (the learned surrogate
of K GE steps) -- test infrastructure only, like the rest of ``oracle/``.

The surrogate has no counterpart in arXiv:1310.3422; its definition is the
model described in ``include/ge_sno.h``.  This module evaluates that
definition with plain PyTorch CPU ops in float64, along a different route
from the CUDA library: the truncated transform and its inverse are
``torch.fft.rfft`` / ``torch.fft.irfft`` (the library builds DFT matrices and
multiplies), the complex mode mixing is complex arithmetic (the library uses
the equivalent real 2x2 block form), and gradients come from autograd (the
library has its own backward kernels).  It shares no code with the library.

Parameter vector layout (same order as the library): W0 [4][C], b0 [C]; per
layer Rr [M][C out][C in], Ri [M][C][C], W [C in][C out], b [C]; Q1 [C][H],
q1 [H], Q2 [H], q2 [1].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch


@dataclass(frozen=True)
class Arch:
    n: int
    width: int
    modes: int
    layers: int
    hidden: int


def num_params(a: Arch) -> int:
    C, M, H = a.width, a.modes, a.hidden
    return 5 * C + a.layers * (2 * M * C * C + C * C + C) + C * H + 2 * H + 1


def unpack(p: torch.Tensor, a: Arch) -> dict:
    """Views of the flat parameter vector, by name."""
    C, M, H = a.width, a.modes, a.hidden
    out, off = {}, 0

    def take(name, shape):
        nonlocal off
        size = int(np.prod(shape))
        out[name] = p[off:off + size].view(*shape)
        off += size

    take("lift_w", (4, C))
    take("lift_b", (C,))
    for l in range(a.layers):
        take(f"Rr{l}", (M, C, C))
        take(f"Ri{l}", (M, C, C))
        take(f"W{l}", (C, C))
        take(f"b{l}", (C,))
    take("Q1", (C, H))
    take("q1", (H,))
    take("Q2", (H,))
    take("q2", (1,))
    assert off == p.numel()
    return out


def round_bf16(p: torch.Tensor) -> torch.Tensor:
    """Round FP32 values to the nearest BF16 value (ties to even), as float64."""
    return p.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def features(u0, r, bl, br, n: int) -> torch.Tensor:
    """[B, n, 4]: (u0, x, r, wall profile) with x_j = (j + 1) / (n + 1)."""
    x = torch.arange(1, n + 1, dtype=torch.float64) / float(n + 1)
    B = u0.shape[0]
    xb = x.expand(B, n)
    return torch.stack([u0, xb, r[:, None].expand(B, n), bl[:, None] + (br - bl)[:, None] * xb], dim=-1)


def spectral(v: torch.Tensor, Rr: torch.Tensor, Ri: torch.Tensor, modes: int) -> torch.Tensor:
    """Truncated spectral convolution along the grid axis of v [B, n, C]:
    keep the `modes` lowest rfft coefficients, multiply mode m by the complex
    matrix R_m = Rr_m + i Ri_m (out x in), transform back."""
    n = v.shape[1]
    X = torch.fft.rfft(v, dim=1)[:, :modes, :]                  # [B, M, C] complex
    R = torch.complex(Rr, Ri)                                    # [M, out, in]
    Y = torch.einsum("moi,bmi->bmo", R, X)
    full = torch.zeros(v.shape[0], n // 2 + 1, v.shape[2], dtype=Y.dtype)
    full[:, :modes, :] = Y
    return torch.fft.irfft(full, n=n, dim=1)


def gelu(x):
    return torch.nn.functional.gelu(x, approximate="tanh")


def forward(p: torch.Tensor, a: Arch, u0, r, bl, br) -> torch.Tensor:
    """Prediction [B, n] of the network with parameter vector p (float64):
    u0 plus the projected features (residual output)."""
    w = unpack(p, a)
    v = features(u0, r, bl, br, a.n) @ w["lift_w"] + w["lift_b"]
    for l in range(a.layers):
        pre = spectral(v, w[f"Rr{l}"], w[f"Ri{l}"], a.modes) + v @ w[f"W{l}"] + w[f"b{l}"]
        v = gelu(pre) if l < a.layers - 1 else pre
    h = gelu(v @ w["Q1"] + w["q1"])
    return u0 + h @ w["Q2"] + w["q2"]


def rel_l2(pred: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Per-problem relative L2 error ||pred - target|| / ||target||."""
    return torch.linalg.vector_norm(pred - target, dim=1) / torch.linalg.vector_norm(target, dim=1)


def _t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


def predict(params, a: Arch, u0, r, bl, br) -> np.ndarray:
    """Forward pass on numpy inputs (params are used as given)."""
    with torch.no_grad():
        return forward(_t(params), a, _t(u0), _t(r), _t(bl), _t(br)).numpy()


def loss_and_grad(params, a: Arch, u0, r, bl, br, target):
    """Per-problem losses and the gradient of their mean w.r.t. the parameters."""
    p = _t(params).clone().requires_grad_(True)
    losses = rel_l2(forward(p, a, _t(u0), _t(r), _t(bl), _t(br)), _t(target))
    losses.mean().backward()
    return losses.detach().numpy(), p.grad.numpy()
