"""The GE steps of arXiv:1310.3422 Sec. 2 (sub-domain width 1) in numpy
extended precision (longdouble), vectorised over the groups: a reference
for attributing FP64 round-off in long or badly conditioned runs (test
infrastructure; not a parity reference, and not used by the library)."""
import numpy as np


def ext_precision_run(u0, r, bl, br, steps):
    """The GE steps in numpy extended precision (longdouble), vectorised over
    the groups; only used to attribute round-off, not as a parity reference."""
    ld = np.longdouble
    r = ld(r)
    det = 1 + 2 * r
    c = [(r + r * r) / det, (1 - r * r) / det, (r - r * r) / det, r * r / det]
    s0, s1 = r / (1 + r), (1 - r) / (1 + r)
    u = np.asarray(u0, dtype=ld).copy()
    n = u.size
    for s in range(steps):
        p = s % 2
        ext = np.concatenate(([ld(bl)], u, [ld(br)]))
        out = u.copy()
        lo = np.arange(p, n - 1, 2)
        a, b, cc, d = ext[lo], ext[lo + 1], ext[lo + 2], ext[lo + 3]
        out[lo] = c[0] * a + c[1] * b + c[2] * cc + c[3] * d
        out[lo + 1] = c[3] * a + c[2] * b + c[1] * cc + c[0] * d
        if p == 1:
            out[0] = s0 * ld(bl) + s1 * u[0] + s0 * (u[1] if n > 1 else ld(br))
        if (n - p) % 2 == 1:
            out[n - 1] = s0 * ld(br) + s1 * u[n - 1] + s0 * (u[n - 2] if n > 1 else ld(bl))
        u = out
    return u
