"""ctypes binding of ``libge.so`` (the C ABI of ``include/ge.h`` and
``include/ge_sno.h``).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Entry points keep the C names; device buffers are torch CUDA
tensors (or raw integer device pointers), host buffers numpy arrays.  A
failing call raises :class:`GeError` with the library's status and message.
Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libge.so")

GE_OK, GE_EINVAL, GE_ENOMEM, GE_ECUDA, GE_ETIMEOUT, GE_ENONFINITE = range(6)
GE_F64, GE_F32, GE_F32_COMP = 0, 1, 2
GE_KERNEL_AUTO, GE_KERNEL_CANONICAL, GE_KERNEL_ONESTEP, GE_KERNEL_TEMPORAL, GE_KERNEL_TEMPORAL_DF = 0, 1, 2, 3, 4

# Every symbol include/ge.h and include/ge_sno.h declare.
EXPORTS = ("ge_create", "ge_set_kernel", "ge_set_subdomain_width", "ge_step_n", "ge_read_state", "ge_write_state",
           "ge_read_range", "ge_write_range",
           "ge_get_step", "ge_sync", "ge_destroy", "ge_solve", "ge_batch_create", "ge_batch_set_depth",
           "ge_batch_get_depth", "ge_batch_set_kernel", "ge_batch_tune", "ge_batch_set_geometry",
           "ge_batch_get_geometry", "ge_batch_set_persistent", "ge_batch_get_persistent", "ge_batch_run",
           "ge_batch_sync",
           "ge_batch_destroy",
           "ge_solve_batch", "ge_solve_noalloc", "ge_status_str", "ge_last_error", "ge_debug_stall",
           "ge_batch_debug_stall", "ge_batch_check", "ge_get_kernel", "ge_tune", "ge_probe_fma", "ge_fp64_int_share", "ge_set_int_pipes",
           "ge_emu_fma_check",
           "ge_sno_create", "ge_sno_num_params", "ge_sno_get_params", "ge_sno_set_params",
           "ge_sno_set_precision", "ge_sno_set_tensor_cores", "ge_sno_get_tensor_cores", "ge_sno_sync", "ge_sno_forward", "ge_sno_loss_grad", "ge_sno_adam_step",
           "ge_sno_train_step", "ge_sno_rows_nonfinite", "ge_sno_rows_gather", "ge_sno_rows_scatter",
           "ge_sno_rows_rel_err", "ge_sno_destroy")

_lock = threading.Lock()
_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_I32 = ctypes.c_int32


class GeError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {message} (status {status})")


def load(path: str | None = None):
    """Load libge.so and declare the C signatures (idempotent).  `path`
    loads another build of the library (a variant compiled with other
    tuning macros) and makes it the one every later call of this binding
    uses."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libge.so not built at {p}: run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        lib.ge_create.argtypes = [ctypes.POINTER(_VP), _I64, _D, _D, _D, ctypes.c_int, _VP, _VP]
        lib.ge_create.restype = ctypes.c_int
        lib.ge_set_kernel.argtypes = [_VP, ctypes.c_int, _I32]
        lib.ge_set_kernel.restype = ctypes.c_int
        lib.ge_set_subdomain_width.argtypes = [_VP, _I64]
        lib.ge_set_subdomain_width.restype = ctypes.c_int
        lib.ge_step_n.argtypes = [_VP, _I64]
        lib.ge_step_n.restype = ctypes.c_int
        lib.ge_read_state.argtypes = [_VP, _VP]
        lib.ge_read_state.restype = ctypes.c_int
        lib.ge_write_state.argtypes = [_VP, _VP, _I64]
        lib.ge_write_state.restype = ctypes.c_int
        lib.ge_read_range.argtypes = [_VP, _I64, _I64, _VP]
        lib.ge_read_range.restype = ctypes.c_int
        lib.ge_write_range.argtypes = [_VP, _I64, _I64, _VP]
        lib.ge_write_range.restype = ctypes.c_int
        lib.ge_get_step.argtypes = [_VP, ctypes.POINTER(_I64)]
        lib.ge_get_step.restype = ctypes.c_int
        lib.ge_sync.argtypes = [_VP]
        lib.ge_sync.restype = ctypes.c_int
        lib.ge_destroy.argtypes = [_VP]
        lib.ge_destroy.restype = None
        lib.ge_solve.argtypes = [_I64, _D, _D, _D, ctypes.c_int, ctypes.c_int, _I32, _I64, _VP, _VP, _VP]
        lib.ge_solve.restype = ctypes.c_int
        _PI64 = ctypes.POINTER(ctypes.c_int64)
        _PD = ctypes.POINTER(ctypes.c_double)
        lib.ge_batch_create.argtypes = [ctypes.POINTER(_VP), _I32, _PI64, _PD, _PD, _PD, _PI64, _I64,
                                        ctypes.c_int, _VP]
        lib.ge_batch_create.restype = ctypes.c_int
        lib.ge_batch_set_depth.argtypes = [_VP, _I32]
        lib.ge_batch_set_depth.restype = ctypes.c_int
        lib.ge_batch_set_kernel.argtypes = [_VP, ctypes.c_int]
        lib.ge_batch_set_kernel.restype = ctypes.c_int
        lib.ge_batch_get_depth.argtypes = [_VP, ctypes.POINTER(_I32)]
        lib.ge_batch_get_depth.restype = ctypes.c_int
        lib.ge_batch_set_geometry.argtypes = [_VP, _I32, _I32]
        lib.ge_batch_set_geometry.restype = ctypes.c_int
        lib.ge_batch_get_geometry.argtypes = [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]
        lib.ge_batch_get_geometry.restype = ctypes.c_int
        lib.ge_batch_set_persistent.argtypes = [_VP, _I32]
        lib.ge_batch_set_persistent.restype = ctypes.c_int
        lib.ge_batch_get_persistent.argtypes = [_VP, ctypes.POINTER(_I32)]
        lib.ge_batch_get_persistent.restype = ctypes.c_int
        lib.ge_batch_tune.argtypes = [_VP, _VP, _I64, ctypes.POINTER(_I32)]
        lib.ge_batch_tune.restype = ctypes.c_int
        lib.ge_batch_run.argtypes = [_VP, _VP, _I64]
        lib.ge_batch_run.restype = ctypes.c_int
        lib.ge_batch_sync.argtypes = [_VP]
        lib.ge_batch_sync.restype = ctypes.c_int
        lib.ge_batch_destroy.argtypes = [_VP]
        lib.ge_batch_destroy.restype = None
        lib.ge_solve_batch.argtypes = [_I32, _PI64, _PD, _PD, _PD, _PI64, _I64, _VP, _VP, _I64, ctypes.c_int, _VP]
        lib.ge_solve_batch.restype = ctypes.c_int
        lib.ge_solve_noalloc.argtypes = [_I64, _D, _D, _D, ctypes.c_int, _I32, _I64, _VP, _VP, _VP]
        lib.ge_solve_noalloc.restype = ctypes.c_int
        lib.ge_probe_fma.argtypes = [_I32, _I32, _I32, _I64, _VP, _VP]
        lib.ge_probe_fma.restype = ctypes.c_int
        lib.ge_set_int_pipes.argtypes = [_VP, _I32]
        lib.ge_set_int_pipes.restype = ctypes.c_int
        lib.ge_fp64_int_share.argtypes = [ctypes.POINTER(ctypes.c_double)]
        lib.ge_fp64_int_share.restype = ctypes.c_int
        lib.ge_emu_fma_check.argtypes = [ctypes.c_double, _VP, _VP, _I64, _VP, _VP]
        lib.ge_emu_fma_check.restype = ctypes.c_int
        lib.ge_sno_create.argtypes = [ctypes.POINTER(_VP), _I32, _I32, _I32, _I32, _I32, _I32, ctypes.c_uint64, _VP]
        lib.ge_sno_create.restype = ctypes.c_int
        lib.ge_sno_set_tensor_cores.argtypes = [_VP, _I32]
        lib.ge_sno_set_tensor_cores.restype = ctypes.c_int
        lib.ge_sno_get_tensor_cores.argtypes = [_VP, ctypes.POINTER(_I32)]
        lib.ge_sno_get_tensor_cores.restype = ctypes.c_int
        lib.ge_sno_sync.argtypes = [_VP]
        lib.ge_sno_sync.restype = ctypes.c_int
        lib.ge_sno_num_params.argtypes = [_VP, ctypes.POINTER(_I64)]
        lib.ge_sno_num_params.restype = ctypes.c_int
        lib.ge_sno_get_params.argtypes = [_VP, _VP]
        lib.ge_sno_get_params.restype = ctypes.c_int
        lib.ge_sno_set_params.argtypes = [_VP, _VP]
        lib.ge_sno_set_params.restype = ctypes.c_int
        lib.ge_sno_set_precision.argtypes = [_VP, _I32]
        lib.ge_sno_set_precision.restype = ctypes.c_int
        lib.ge_sno_forward.argtypes = [_VP, _I32, _VP, _VP, _VP, _VP, _VP]
        lib.ge_sno_forward.restype = ctypes.c_int
        lib.ge_sno_loss_grad.argtypes = [_VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP]
        lib.ge_sno_loss_grad.restype = ctypes.c_int
        lib.ge_sno_adam_step.argtypes = [_VP, ctypes.c_float]
        lib.ge_sno_adam_step.restype = ctypes.c_int
        lib.ge_sno_train_step.argtypes = [_VP, _I32, _VP, _VP, _VP, _VP, _VP, ctypes.c_float, _VP]
        lib.ge_sno_train_step.restype = ctypes.c_int
        lib.ge_sno_destroy.argtypes = [_VP]
        lib.ge_sno_destroy.restype = None
        lib.ge_sno_rows_nonfinite.argtypes = [_VP, _VP, _I64, _VP]
        lib.ge_sno_rows_gather.argtypes = [_VP, _VP, _I64, _VP, _I64, _VP]
        lib.ge_sno_rows_scatter.argtypes = [_VP, _VP, _I64, _VP, _VP, _I64]
        lib.ge_sno_rows_rel_err.argtypes = [_VP, _VP, _I64, _VP, _VP, _I64, _VP]
        for fn in ("ge_sno_rows_nonfinite", "ge_sno_rows_gather", "ge_sno_rows_scatter", "ge_sno_rows_rel_err"):
            getattr(lib, fn).restype = ctypes.c_int
        lib.ge_get_kernel.argtypes = [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I32)]
        lib.ge_get_kernel.restype = ctypes.c_int
        lib.ge_tune.argtypes = [_VP, _I64, ctypes.POINTER(_I32)]
        lib.ge_tune.restype = ctypes.c_int
        lib.ge_debug_stall.argtypes = [_VP, _I64]
        lib.ge_debug_stall.restype = ctypes.c_int
        lib.ge_batch_debug_stall.argtypes = [_VP, _I64]
        lib.ge_batch_debug_stall.restype = ctypes.c_int
        lib.ge_batch_check.argtypes = [_VP, _VP, _VP]
        lib.ge_batch_check.restype = ctypes.c_int
        lib.ge_status_str.argtypes = [ctypes.c_int]
        lib.ge_status_str.restype = ctypes.c_char_p
        lib.ge_last_error.argtypes = []
        lib.ge_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(st: int, where: str):
    if st != GE_OK:
        lib = load()
        raise GeError(st, where, lib.ge_last_error().decode(errors="replace"))


def _dptr(x) -> int | None:
    """Device pointer of a CUDA tensor (or an int), None for None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return x.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_of(prec: int):
    import torch
    return torch.float64 if prec == GE_F64 else torch.float32


class Ctx:
    """Owner of a ``ge_ctx*``; destroyed explicitly or when collected."""

    def __init__(self, handle: int, n: int, prec: int):
        self.handle = handle
        self.n = n
        self.prec = prec

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                ge_destroy(self)
            except Exception:
                pass


def ge_create(n: int, r: float, beta_l: float, beta_r: float, prec: int, u0=None, stream=None) -> Ctx:
    lib = load()
    h = _VP()
    if u0 is not None and (u0.numel() != n or u0.dtype != dtype_of(prec)):
        raise ValueError("u0 must hold n elements of the precision's dtype")
    _check(lib.ge_create(ctypes.byref(h), int(n), float(r), float(beta_l), float(beta_r), int(prec),
                         _dptr(u0), _stream_handle(stream)), "ge_create")
    return Ctx(h.value, int(n), int(prec))


def ge_set_kernel(ctx: Ctx, kernel: int, depth: int = 0):
    _check(load().ge_set_kernel(ctx.handle, int(kernel), int(depth)), "ge_set_kernel")


def ge_get_kernel(ctx: Ctx):
    """(kernel, steps per launch of the tiled kernel)."""
    k, d = ctypes.c_int(), _I32()
    _check(load().ge_get_kernel(ctx.handle, ctypes.byref(k), ctypes.byref(d)), "ge_get_kernel")
    return int(k.value), int(d.value)


def ge_tune(ctx: Ctx, steps: int) -> int:
    d = _I32()
    _check(load().ge_tune(ctx.handle, int(steps), ctypes.byref(d)), "ge_tune")
    return int(d.value)


def ge_set_subdomain_width(ctx: Ctx, k: int):
    _check(load().ge_set_subdomain_width(ctx.handle, int(k)), "ge_set_subdomain_width")


def ge_step_n(ctx: Ctx, steps: int):
    _check(load().ge_step_n(ctx.handle, int(steps)), "ge_step_n")


def ge_read_state(ctx: Ctx, out):
    if out.numel() < ctx.n or out.dtype != dtype_of(ctx.prec):
        raise ValueError("output tensor too small or of the wrong dtype")
    _check(load().ge_read_state(ctx.handle, _dptr(out)), "ge_read_state")


def ge_write_state(ctx: Ctx, src, step_count: int):
    if src.numel() < ctx.n or src.dtype != dtype_of(ctx.prec):
        raise ValueError("state tensor too small or of the wrong dtype")
    _check(load().ge_write_state(ctx.handle, _dptr(src), int(step_count)), "ge_write_state")


def ge_read_range(ctx: Ctx, offset: int, count: int, dst):
    """dst (CUDA tensor of at least `count` elements) <- points [offset, offset + count)."""
    if dst.numel() < count or dst.dtype != dtype_of(ctx.prec):
        raise ValueError("destination too small or of the wrong dtype")
    _check(load().ge_read_range(ctx.handle, int(offset), int(count), _dptr(dst)), "ge_read_range")


def ge_write_range(ctx: Ctx, offset: int, count: int, src):
    """Points [offset, offset + count) <- src (CUDA tensor); the step counter stays."""
    if src.numel() < count or src.dtype != dtype_of(ctx.prec):
        raise ValueError("source too small or of the wrong dtype")
    _check(load().ge_write_range(ctx.handle, int(offset), int(count), _dptr(src)), "ge_write_range")


def ge_get_step(ctx: Ctx) -> int:
    v = _I64()
    _check(load().ge_get_step(ctx.handle, ctypes.byref(v)), "ge_get_step")
    return int(v.value)


def ge_sync(ctx: Ctx):
    _check(load().ge_sync(ctx.handle), "ge_sync")


def ge_destroy(ctx: Ctx):
    if ctx.handle:
        load().ge_destroy(ctx.handle)
        ctx.handle = None


def ge_debug_stall(ctx: Ctx, cycles: int):
    _check(load().ge_debug_stall(ctx.handle, int(cycles)), "ge_debug_stall")


def ge_solve(n: int, r: float, beta_l: float, beta_r: float, prec: int, kernel: int, depth: int,
             steps: int, u0_host: np.ndarray, u_out_host: np.ndarray, stream=None):
    """One-shot solve from host memory (numpy arrays of n float64/float32)."""
    dt = np.float64 if prec == GE_F64 else np.float32
    for a in (u0_host, u_out_host):
        if a.dtype != dt or a.size < n or not a.flags.c_contiguous:
            raise ValueError("host buffers must be contiguous arrays of n elements of the precision's dtype")
    _check(load().ge_solve(int(n), float(r), float(beta_l), float(beta_r), int(prec), int(kernel),
                           int(depth), int(steps), u0_host.ctypes.data, u_out_host.ctypes.data,
                           _stream_handle(stream)), "ge_solve")


class Batch:
    """Owner of a ``ge_batch*`` plan."""

    def __init__(self, handle: int, total: int, prec: int, n_problems: int = 0):
        self.handle = handle
        self.total = total
        self.prec = prec
        self.n_problems = n_problems

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                ge_batch_destroy(self)
            except Exception:
                pass


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _batch_arrays(n, r, beta_l, beta_r, offsets):
    arrs = [_i64(n), _f64(r), _f64(beta_l), _f64(beta_r), _i64(offsets)]
    if len({a.size for a in arrs}) != 1:
        raise ValueError("n, r, beta_l, beta_r and offsets must have one entry per problem")
    return arrs


def ge_batch_create(n, r, beta_l, beta_r, offsets, total: int, prec: int, stream=None) -> Batch:
    a_n, a_r, a_bl, a_br, a_off = _batch_arrays(n, r, beta_l, beta_r, offsets)
    h = _VP()
    P64 = ctypes.POINTER(ctypes.c_int64)
    PD = ctypes.POINTER(ctypes.c_double)
    _check(load().ge_batch_create(ctypes.byref(h), a_n.size, a_n.ctypes.data_as(P64), a_r.ctypes.data_as(PD),
                                  a_bl.ctypes.data_as(PD), a_br.ctypes.data_as(PD), a_off.ctypes.data_as(P64),
                                  int(total), int(prec), _stream_handle(stream)), "ge_batch_create")
    return Batch(h.value, int(total), int(prec), int(a_n.size))


def ge_batch_set_depth(plan: Batch, depth: int):
    _check(load().ge_batch_set_depth(plan.handle, int(depth)), "ge_batch_set_depth")


def ge_batch_set_kernel(plan: Batch, kernel: int):
    _check(load().ge_batch_set_kernel(plan.handle, int(kernel)), "ge_batch_set_kernel")


def ge_batch_set_geometry(plan: Batch, tile_rows: int, ctas_per_sm: int):
    """Rows per tile (256 or 128; 0 = 256) and CTAs per SM (0 = as many as fit)."""
    _check(load().ge_batch_set_geometry(plan.handle, int(tile_rows), int(ctas_per_sm)), "ge_batch_set_geometry")


def ge_batch_get_geometry(plan: Batch):
    """(rows per tile, CTAs per SM) of the plan's launches."""
    tr, c = _I32(), _I32()
    _check(load().ge_batch_get_geometry(plan.handle, ctypes.byref(tr), ctypes.byref(c)), "ge_batch_get_geometry")
    return int(tr.value), int(c.value)


def ge_batch_set_persistent(plan: Batch, on: int):
    """1: a run of more than `depth` steps as one persistent launch (plain FP32 plans)."""
    _check(load().ge_batch_set_persistent(plan.handle, int(on)), "ge_batch_set_persistent")


def ge_batch_get_persistent(plan: Batch) -> int:
    v = _I32()
    _check(load().ge_batch_get_persistent(plan.handle, ctypes.byref(v)), "ge_batch_get_persistent")
    return int(v.value)


def ge_batch_get_depth(plan: Batch) -> int:
    v = _I32()
    _check(load().ge_batch_get_depth(plan.handle, ctypes.byref(v)), "ge_batch_get_depth")
    return int(v.value)


def ge_batch_tune(plan: Batch, u, steps: int) -> int:
    v = _I32()
    _check(load().ge_batch_tune(plan.handle, _dptr(u), int(steps), ctypes.byref(v)), "ge_batch_tune")
    return int(v.value)


def ge_batch_run(plan: Batch, u, steps: int):
    if u.numel() < plan.total or u.dtype != dtype_of(plan.prec):
        raise ValueError("packed buffer too small or of the wrong dtype")
    _check(load().ge_batch_run(plan.handle, _dptr(u), int(steps)), "ge_batch_run")


def ge_batch_sync(plan: Batch):
    _check(load().ge_batch_sync(plan.handle), "ge_batch_sync")


def ge_batch_check(plan: Batch, u, status):
    """Per-problem status (GE_OK / GE_ENONFINITE) of the packed buffer u into
    `status` (CUDA int32 tensor with one entry per problem)."""
    import torch
    if status.dtype != torch.int32 or status.numel() < plan.n_problems:
        raise ValueError("status must be an int32 CUDA tensor with one entry per problem")
    if u.numel() < plan.total or u.dtype != dtype_of(plan.prec):
        raise ValueError("packed buffer too small or of the wrong dtype")
    _check(load().ge_batch_check(plan.handle, _dptr(u), _dptr(status)), "ge_batch_check")


def ge_batch_debug_stall(plan: Batch, cycles: int):
    _check(load().ge_batch_debug_stall(plan.handle, int(cycles)), "ge_batch_debug_stall")


def ge_batch_destroy(plan: Batch):
    if plan.handle:
        load().ge_batch_destroy(plan.handle)
        plan.handle = None


def ge_solve_batch(n, r, beta_l, beta_r, offsets, total: int, u, steps: int, prec: int, stream=None, status=None):
    """One-shot batched solve in place in u; `status` (optional CUDA int32
    tensor, one entry per problem) receives GE_OK / GE_ENONFINITE."""
    import torch
    a_n, a_r, a_bl, a_br, a_off = _batch_arrays(n, r, beta_l, beta_r, offsets)
    if u.numel() < total or u.dtype != dtype_of(prec):
        raise ValueError("packed buffer too small or of the wrong dtype")
    if status is not None and (status.dtype != torch.int32 or status.numel() < a_n.size):
        raise ValueError("status must be an int32 CUDA tensor with one entry per problem")
    P64 = ctypes.POINTER(ctypes.c_int64)
    PD = ctypes.POINTER(ctypes.c_double)
    _check(load().ge_solve_batch(a_n.size, a_n.ctypes.data_as(P64), a_r.ctypes.data_as(PD),
                                 a_bl.ctypes.data_as(PD), a_br.ctypes.data_as(PD), a_off.ctypes.data_as(P64),
                                 int(total), _dptr(u), _dptr(status), int(steps), int(prec),
                                 _stream_handle(stream)),
           "ge_solve_batch")


def ge_solve_noalloc(n: int, r: float, beta_l: float, beta_r: float, prec: int, depth: int, steps: int,
                     u0, u_out, stream=None):
    """Tiled solve that allocates no device memory (fixed working memory in
    the library; n <= 1,048,576).  u0 / u_out: CUDA tensors of n elements."""
    for a in (u0, u_out):
        if a.numel() < n or a.dtype != dtype_of(prec):
            raise ValueError("buffers must hold n elements of the precision's dtype")
    _check(load().ge_solve_noalloc(int(n), float(r), float(beta_l), float(beta_r), int(prec), int(depth),
                                   int(steps), _dptr(u0), _dptr(u_out), _stream_handle(stream)),
           "ge_solve_noalloc")


PROBE_THREADS = 256


def ge_set_int_pipes(ctx: Ctx, on: int):
    _check(load().ge_set_int_pipes(ctx.handle, int(on)), "ge_set_int_pipes")


def ge_fp64_int_share() -> float:
    """Share of the FP64 tiled kernel's interior updates done on the integer pipes."""
    v = ctypes.c_double()
    _check(load().ge_fp64_int_share(ctypes.byref(v)), "ge_fp64_int_share")
    return float(v.value)


def ge_emu_fma_check(g: float, p, x, counts, stream=None):
    """Integer-pipe FP64 multiply-add against the FP64 unit on p, x (device
    float64 tensors of equal length); counts: device int64 tensor of 3."""
    n = p.numel()
    if x.numel() != n or counts.numel() < 3:
        raise ValueError("p and x must have equal length; counts needs 3 elements")
    _check(load().ge_emu_fma_check(float(g), _dptr(p), _dptr(x), int(n), _dptr(counts), _stream_handle(stream)),
           "ge_emu_fma_check")


def ge_probe_fma(prec: int, blocks: int, chains: int, iters: int, sink, stream=None) -> int:
    """Register-only multiply-add throughput probe (GE_F64: DFMA, GE_F32:
    FFMA), `chains` (4, 8, 16, 32) independent chains per thread; sink: CUDA
    tensor of blocks * 256 elements of the precision's dtype.  Returns the
    multiply-adds the launch does."""
    if sink.numel() < blocks * PROBE_THREADS or sink.dtype != dtype_of(prec):
        raise ValueError("sink must hold blocks * 256 elements of the precision's dtype")
    _check(load().ge_probe_fma(int(prec), int(blocks), int(chains), int(iters), _dptr(sink),
                               _stream_handle(stream)), "ge_probe_fma")
    return int(blocks) * PROBE_THREADS * int(chains) * int(iters)


class Sno:
    """Owner of a ``ge_sno*`` surrogate model."""

    def __init__(self, handle: int, n: int, width: int, modes: int, layers: int, hidden: int, max_batch: int):
        self.handle = handle
        self.n, self.width, self.modes, self.layers, self.hidden = n, width, modes, layers, hidden
        self.max_batch = max_batch

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                ge_sno_destroy(self)
            except Exception:
                pass


def _f32_dev(x, count: int, what: str):
    import torch
    if x is None or x.dtype != torch.float32 or x.numel() < count:
        raise ValueError(f"{what} must be a CUDA float32 tensor of at least {count} elements")
    return _dptr(x)


def _rows(model: "Sno", x, what: str, dtype=None) -> int:
    """Row count of a contiguous CUDA [rows, n] (or flat) tensor of the model's row length."""
    import torch
    dtype = dtype or torch.float32
    if x is None or not x.is_cuda or x.dtype != dtype or not x.is_contiguous() or x.numel() % model.n:
        raise ValueError(f"{what} must be a contiguous CUDA {dtype} tensor of whole rows of {model.n}")
    return x.numel() // model.n


def _idx(idx, what: str = "idx") -> int:
    import torch
    if idx is None or not idx.is_cuda or idx.dtype != torch.int64 or not idx.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA int64 tensor")
    return idx.numel()


def ge_sno_rows_nonfinite(model: "Sno", u, flags):
    """flags (CUDA int32, one per row) <- 1 where the row of u holds NaN/Inf."""
    import torch
    rows = _rows(model, u, "u")
    if flags.dtype != torch.int32 or flags.numel() < rows or not flags.is_cuda:
        raise ValueError("flags must be a CUDA int32 tensor with one entry per row")
    _check(load().ge_sno_rows_nonfinite(model.handle, _dptr(u), rows, _dptr(flags)), "ge_sno_rows_nonfinite")


def ge_sno_rows_gather(model: "Sno", src, idx, dst):
    """dst row i <- src row idx[i]."""
    count = _idx(idx)
    if _rows(model, dst, "dst") < count:
        raise ValueError("dst holds fewer rows than idx")
    _check(load().ge_sno_rows_gather(model.handle, _dptr(src), _rows(model, src, "src"), _dptr(idx), count,
                                     _dptr(dst)), "ge_sno_rows_gather")


def ge_sno_rows_scatter(model: "Sno", dst, idx, src):
    """dst row idx[i] <- src row i."""
    count = _idx(idx)
    if _rows(model, src, "src") < count:
        raise ValueError("src holds fewer rows than idx")
    _check(load().ge_sno_rows_scatter(model.handle, _dptr(dst), _rows(model, dst, "dst"), _dptr(idx), _dptr(src),
                                      count), "ge_sno_rows_scatter")


def ge_sno_rows_rel_err(model: "Sno", a, idx, ref, err):
    """err[i] (CUDA float32) <- ||a row idx[i] - ref row i|| / ||ref row i||."""
    import torch
    count = _idx(idx)
    if _rows(model, ref, "ref") < count:
        raise ValueError("ref holds fewer rows than idx")
    if err.dtype != torch.float32 or err.numel() < count or not err.is_cuda:
        raise ValueError("err must be a CUDA float32 tensor with one entry per index")
    _check(load().ge_sno_rows_rel_err(model.handle, _dptr(a), _rows(model, a, "a"), _dptr(idx), _dptr(ref), count,
                                      _dptr(err)), "ge_sno_rows_rel_err")


def ge_sno_create(n: int, width: int, modes: int, layers: int, hidden: int, max_batch: int, seed: int = 0,
                  stream=None) -> Sno:
    h = _VP()
    _check(load().ge_sno_create(ctypes.byref(h), int(n), int(width), int(modes), int(layers), int(hidden),
                                int(max_batch), int(seed), _stream_handle(stream)), "ge_sno_create")
    return Sno(h.value, int(n), int(width), int(modes), int(layers), int(hidden), int(max_batch))


def ge_sno_num_params(model: Sno) -> int:
    v = _I64()
    _check(load().ge_sno_num_params(model.handle, ctypes.byref(v)), "ge_sno_num_params")
    return int(v.value)


def ge_sno_get_params(model: Sno, dst):
    _check(load().ge_sno_get_params(model.handle, _f32_dev(dst, ge_sno_num_params(model), "dst")),
           "ge_sno_get_params")


def ge_sno_set_params(model: Sno, src):
    _check(load().ge_sno_set_params(model.handle, _f32_dev(src, ge_sno_num_params(model), "src")),
           "ge_sno_set_params")


def ge_sno_set_precision(model: Sno, split: int):
    _check(load().ge_sno_set_precision(model.handle, int(split)), "ge_sno_set_precision")


def ge_sno_set_tensor_cores(model: Sno, on: int):
    """1: fused layers and projection of inference on tcgen05 (where the shape allows); 0: mma.sync only."""
    _check(load().ge_sno_set_tensor_cores(model.handle, int(on)), "ge_sno_set_tensor_cores")


def ge_sno_get_tensor_cores(model: Sno) -> int:
    v = _I32()
    _check(load().ge_sno_get_tensor_cores(model.handle, ctypes.byref(v)), "ge_sno_get_tensor_cores")
    return int(v.value)


def ge_sno_sync(model: Sno):
    _check(load().ge_sno_sync(model.handle), "ge_sno_sync")


def _sno_inputs(model: Sno, batch: int, u0, r, beta_l, beta_r):
    return (_f32_dev(u0, batch * model.n, "u0"), _f32_dev(r, batch, "r"), _f32_dev(beta_l, batch, "beta_l"),
            _f32_dev(beta_r, batch, "beta_r"))


def ge_sno_forward(model: Sno, batch: int, u0, r, beta_l, beta_r, pred):
    args = _sno_inputs(model, batch, u0, r, beta_l, beta_r)
    _check(load().ge_sno_forward(model.handle, int(batch), *args, _f32_dev(pred, batch * model.n, "pred")),
           "ge_sno_forward")


def ge_sno_loss_grad(model: Sno, batch: int, u0, r, beta_l, beta_r, target, loss=None, grads=None):
    args = _sno_inputs(model, batch, u0, r, beta_l, beta_r)
    _check(load().ge_sno_loss_grad(model.handle, int(batch), *args,
                                   _f32_dev(target, batch * model.n, "target"),
                                   None if loss is None else _f32_dev(loss, batch, "loss"),
                                   None if grads is None else _f32_dev(grads, ge_sno_num_params(model), "grads")),
           "ge_sno_loss_grad")


def ge_sno_adam_step(model: Sno, lr: float):
    _check(load().ge_sno_adam_step(model.handle, float(lr)), "ge_sno_adam_step")


def ge_sno_train_step(model: Sno, batch: int, u0, r, beta_l, beta_r, target, lr: float, loss=None):
    args = _sno_inputs(model, batch, u0, r, beta_l, beta_r)
    _check(load().ge_sno_train_step(model.handle, int(batch), *args,
                                    _f32_dev(target, batch * model.n, "target"), float(lr),
                                    None if loss is None else _f32_dev(loss, batch, "loss")),
           "ge_sno_train_step")


def ge_sno_destroy(model: Sno):
    if model.handle:
        load().ge_sno_destroy(model.handle)
        model.handle = None


def ge_status_str(status: int) -> str:
    return load().ge_status_str(int(status)).decode()


def ge_last_error() -> str:
    return load().ge_last_error().decode(errors="replace")
