"""CPU oracle of the group explicit (GE) step -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It wraps
``ge_oracle.c`` (serial FP64 C, built with ``-ffp-contract=off``) through
ctypes; it shares no code with the CUDA library.

Every function follows arXiv:1310.3422 Sec. 2 with sub-domain width k = 1:
Eqs. (cc)/(dd) for the two members of each 2-point group (prefactor
1/(1+2r)), Saul'yev A (Eq. (aa)) for a singleton at the left wall and
Saul'yev B (Eq. (bb)) for one at the right wall, and the groups of parity
``s % 2`` of the global step counter ``s``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ge_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libge_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle C file into a shared library (gcc, no contraction)."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build() -> str:
    """Build ``libge_oracle.so`` next to the source (always recompiles)."""
    return compile_oracle()


def load(path: str | None = None):
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path or _LIB_PATH)
    lib.ge_oracle_coefficients.argtypes = [_D, _PD]
    lib.ge_oracle_coefficients.restype = None
    lib.ge_oracle_step.argtypes = [_I64, _D, _D, _D, ctypes.c_int, _PD, _PD]
    lib.ge_oracle_step.restype = ctypes.c_int
    lib.ge_oracle_run.argtypes = [_I64, _D, _D, _D, _I64, _I64, _PD]
    lib.ge_oracle_run.restype = ctypes.c_int
    lib.ge_oracle_step_k.argtypes = [_I64, _D, _D, _D, ctypes.c_int, _I64, _PD, _PD]
    lib.ge_oracle_step_k.restype = ctypes.c_int
    lib.ge_oracle_run_k.argtypes = [_I64, _D, _D, _D, _I64, _I64, _I64, _PD]
    lib.ge_oracle_run_k.restype = ctypes.c_int
    lib.ge_oracle_step_periodic.argtypes = [_I64, _D, ctypes.c_int, _PD, _PD]
    lib.ge_oracle_step_periodic.restype = ctypes.c_int
    lib.ge_oracle_run_periodic.argtypes = [_I64, _D, _I64, _I64, _PD]
    lib.ge_oracle_run_periodic.restype = ctypes.c_int
    return lib


def _get():
    global _lib
    with _lock:
        if _lib is None:
            stale = (not os.path.exists(_LIB_PATH) or
                     os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
            if stale:
                build()
            _lib = load()
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_PD)


class Oracle:
    """Thin numpy front end over one oracle library (the default one, or a
    separately compiled copy, e.g. a planted-mistake build in the tests)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else _get()

    def coefficients(self, r: float) -> np.ndarray:
        out = np.zeros(6)
        self.lib.ge_oracle_coefficients(float(r), _ptr(out))
        return out

    def step(self, u, r, beta_l, beta_r, parity) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        rc = self.lib.ge_oracle_step(u.size, float(r), float(beta_l), float(beta_r),
                                     int(parity), _ptr(u), _ptr(out))
        if rc != 0:
            raise ValueError("ge_oracle_step rejected its arguments")
        return out

    def run(self, u, r, beta_l, beta_r, steps, step0=0) -> np.ndarray:
        u = np.array(u, dtype=np.float64, copy=True)
        rc = self.lib.ge_oracle_run(u.size, float(r), float(beta_l), float(beta_r),
                                    int(step0), int(steps), _ptr(u))
        if rc != 0:
            raise ValueError("ge_oracle_run rejected its arguments")
        return u

    def step_k(self, u, r, beta_l, beta_r, parity, k) -> np.ndarray:
        """One step with sub-domain width k (k = 1: the 2-point group step)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        if self.lib.ge_oracle_step_k(u.size, float(r), float(beta_l), float(beta_r), int(parity), int(k),
                                     _ptr(u), _ptr(out)):
            raise ValueError("ge_oracle_step_k rejected its arguments")
        return out

    def run_k(self, u, r, beta_l, beta_r, k, steps, step0=0) -> np.ndarray:
        u = np.array(u, dtype=np.float64, copy=True)
        if self.lib.ge_oracle_run_k(u.size, float(r), float(beta_l), float(beta_r), int(k), int(step0),
                                    int(steps), _ptr(u)):
            raise ValueError("ge_oracle_run_k rejected its arguments")
        return u

    def step_periodic(self, u, r, parity) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        if self.lib.ge_oracle_step_periodic(u.size, float(r), int(parity), _ptr(u), _ptr(out)):
            raise ValueError("ge_oracle_step_periodic rejected its arguments")
        return out

    def run_periodic(self, u, r, steps, step0=0) -> np.ndarray:
        u = np.array(u, dtype=np.float64, copy=True)
        if self.lib.ge_oracle_run_periodic(u.size, float(r), int(step0), int(steps), _ptr(u)):
            raise ValueError("ge_oracle_run_periodic rejected its arguments")
        return u

    def sample(self, u0, r, beta_l, beta_r, steps, indices, step0=0) -> np.ndarray:
        """Values u_i after `steps` steps at the given indices, each computed on
        a window of the grid only.  After S steps a point depends on the
        initial data within S+1 points on either side (the dependency cone of
        the GE step), so a window reaching S+4 points past the index, starting
        at an even index (so the window's groups are the grid's groups), gives
        the same value as the full grid.  A window edge that is not a true wall
        is treated as a wall; its error stays inside the cone margin."""
        u0 = np.asarray(u0, dtype=np.float64)
        n = u0.size
        margin = int(steps) + 4
        out = np.empty(len(indices))
        for k, i in enumerate(indices):
            lo = max(0, int(i) - margin)
            lo -= lo % 2
            hi = min(n, int(i) + margin + 1)
            bl = beta_l if lo == 0 else 0.0
            br = beta_r if hi == n else 0.0
            w = self.run(u0[lo:hi], r, bl, br, steps, step0=step0)
            out[k] = w[int(i) - lo]
        return out


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def coefficients(r):
    return default().coefficients(r)


def step(u, r, beta_l, beta_r, parity):
    return default().step(u, r, beta_l, beta_r, parity)


def run(u, r, beta_l, beta_r, steps, step0=0):
    return default().run(u, r, beta_l, beta_r, steps, step0)


def step_periodic(u, r, parity):
    return default().step_periodic(u, r, parity)


def step_k(u, r, beta_l, beta_r, parity, k):
    return default().step_k(u, r, beta_l, beta_r, parity, k)


def run_k(u, r, beta_l, beta_r, k, steps, step0=0):
    return default().run_k(u, r, beta_l, beta_r, k, steps, step0)


def run_periodic(u, r, steps, step0=0):
    return default().run_periodic(u, r, steps, step0)


def sample(u0, r, beta_l, beta_r, steps, indices, step0=0):
    return default().sample(u0, r, beta_l, beta_r, steps, indices, step0)
