"""GB300-native group explicit (GE) solver for u_t = u_xx (arXiv:1310.3422).

The compute path is the CUDA library ``libge.so`` (sm_103a) behind the C ABI in
``include/ge.h``; :mod:`paper_1310_3422_gb300.binding` is its thin ctypes
front end with the same entry-point names.  The library is loaded on first use
and a missing or unbuilt library raises immediately: there is no CPU fallback.
"""
from . import binding, inputs  # noqa: F401  (binding loads libge.so lazily)

__all__ = ["binding", "inputs"]
