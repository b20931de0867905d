"""The C-ABI library loads and exports every entry point include/*.h declares;
argument checks that fail before any device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1310_3422_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ge_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return B.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ge_create", "ge_step_n", "ge_destroy", "ge_read_state", "ge_write_state",
                     "ge_sync", "ge_solve"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names, "no declarations found"
    for name in sorted(names):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported by libge.so"
    assert set(B.EXPORTS) <= names


def test_status_strings(lib):
    assert B.ge_status_str(B.GE_OK) == "GE_OK"
    assert B.ge_status_str(B.GE_EINVAL) == "GE_EINVAL"
    assert B.ge_status_str(B.GE_ETIMEOUT) == "GE_ETIMEOUT"
    assert B.ge_status_str(99) == "GE_UNKNOWN"


@pytest.mark.parametrize("n,r,bl,br,prec", [
    (0, 1.0, 0.0, 0.0, B.GE_F64),
    (-5, 1.0, 0.0, 0.0, B.GE_F64),
    (8, 0.0, 0.0, 0.0, B.GE_F64),
    (8, -1.0, 0.0, 0.0, B.GE_F64),
    (8, float("inf"), 0.0, 0.0, B.GE_F64),
    (8, float("nan"), 0.0, 0.0, B.GE_F64),
    (8, 1.0, float("nan"), 0.0, B.GE_F64),
    (8, 1.0, 0.0, float("inf"), B.GE_F32),
    (8, 1.0, 0.0, 0.0, 7),
])
def test_create_rejects_invalid_arguments(lib, n, r, bl, br, prec):
    h = ctypes.c_void_p(123)
    st = lib.ge_create(ctypes.byref(h), n, r, bl, br, prec, None, None)
    assert st == B.GE_EINVAL
    assert h.value is None
    assert B.ge_last_error() != ""


def test_null_context_is_rejected(lib):
    assert lib.ge_step_n(None, 1) == B.GE_EINVAL
    assert lib.ge_set_kernel(None, 0, 0) == B.GE_EINVAL
    assert lib.ge_read_state(None, None) == B.GE_EINVAL
    assert lib.ge_write_state(None, None, 0) == B.GE_EINVAL
    assert lib.ge_sync(None) == B.GE_EINVAL
    assert lib.ge_create(None, 8, 1.0, 0.0, 0.0, 0, None, None) == B.GE_EINVAL
    lib.ge_destroy(None)  # no-op


def test_solve_rejects_null_host_buffers(lib):
    assert lib.ge_solve(8, 1.0, 0.0, 0.0, 0, 0, 0, 1, None, None, None) == B.GE_EINVAL


def test_batch_layout_checks(lib):
    import numpy as np
    h = ctypes.c_void_p()
    P64 = ctypes.POINTER(ctypes.c_int64)
    PD = ctypes.POINTER(ctypes.c_double)

    def create(n, offs, total, r=None):
        n = np.array(n, dtype=np.int64)
        offs = np.array(offs, dtype=np.int64)
        r = np.array(r if r is not None else [1.0] * len(n))
        z = np.zeros(len(n))
        return lib.ge_batch_create(ctypes.byref(h), len(n), n.ctypes.data_as(P64), r.ctypes.data_as(PD),
                                   z.ctypes.data_as(PD), z.ctypes.data_as(PD), offs.ctypes.data_as(P64),
                                   total, B.GE_F32, None)
    assert create([10], [3], 64) == B.GE_EINVAL             # offset not on a 128-byte row
    assert create([40, 10], [0, 32], 64) == B.GE_EINVAL     # problems share a row
    assert create([10], [0], 5) == B.GE_EINVAL              # problem outside the buffer
    assert create([0], [0], 64) == B.GE_EINVAL              # empty problem
    assert create([10], [0], 64, r=[-1.0]) == B.GE_EINVAL   # bad r
    assert lib.ge_batch_run(None, None, 1) == B.GE_EINVAL
    lib.ge_batch_destroy(None)


@pytest.mark.parametrize("n,width,modes,layers,hidden,max_batch", [
    (2, 8, 1, 1, 1, 1),      # n < 4
    (64, 8, 33, 1, 1, 1),    # modes > n / 2
    (64, 8, 0, 1, 1, 1),
    (64, 0, 4, 1, 1, 1),
    (64, 8, 4, 0, 1, 1),
    (64, 8, 4, 1, 0, 1),
    (64, 8, 4, 1, 1, 0),
])
def test_sno_create_rejects_bad_sizes(lib, n, width, modes, layers, hidden, max_batch):
    h = ctypes.c_void_p()
    st = lib.ge_sno_create(ctypes.byref(h), n, width, modes, layers, hidden, max_batch, 0, None)
    assert st == B.GE_EINVAL and h.value is None
    assert "ge_sno_create" in B.ge_last_error()


def test_sno_calls_on_null_model(lib):
    cnt = ctypes.c_int64(-1)
    assert lib.ge_sno_num_params(None, ctypes.byref(cnt)) == B.GE_EINVAL
    assert lib.ge_sno_set_precision(None, 0) == B.GE_EINVAL
    assert lib.ge_sno_forward(None, 1, 1, 1, 1, 1, 1) == B.GE_EINVAL
    assert lib.ge_sno_loss_grad(None, 1, 1, 1, 1, 1, 1, None, None) == B.GE_EINVAL
    assert lib.ge_sno_adam_step(None, 1e-3) == B.GE_EINVAL
    assert lib.ge_sno_train_step(None, 1, 1, 1, 1, 1, 1, 1e-3, None) == B.GE_EINVAL
    assert lib.ge_sno_rows_nonfinite(None, 1, 1, 1) == B.GE_EINVAL
    assert lib.ge_sno_rows_gather(None, 1, 1, 1, 1, 1) == B.GE_EINVAL
    assert lib.ge_sno_rows_scatter(None, 1, 1, 1, 1, 1) == B.GE_EINVAL
    assert lib.ge_sno_rows_rel_err(None, 1, 1, 1, 1, 1, 1) == B.GE_EINVAL
    lib.ge_sno_destroy(None)


def test_debug_stall_checks_its_arguments(lib):
    assert lib.ge_debug_stall(None, 0) == B.GE_EINVAL
    assert lib.ge_batch_debug_stall(None, 0) == B.GE_EINVAL


def test_fp64_int_share_is_a_fraction(lib):
    """The share of the FP64 tiled kernel's interior updates on the integer
    pipes: a build constant in [0, 1) (7 of a thread's 16 values by default)."""
    share = B.ge_fp64_int_share()
    assert 0.0 <= share < 1.0
    assert share * 16 == round(share * 16)
    assert lib.ge_fp64_int_share(None) == B.GE_EINVAL


def test_int_pipes_switch_checks_its_arguments(lib):
    assert lib.ge_set_int_pipes(None, 1) == B.GE_EINVAL
    assert lib.ge_emu_fma_check(1.0, None, None, 0, None, None) == B.GE_EINVAL
