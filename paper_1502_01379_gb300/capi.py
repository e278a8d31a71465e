"""Thin ctypes binding of libbfly.so (include/bfly.h), same names as the C ABI.

Argument marshalling only: every step of the apply runs in the library's CUDA
kernels.  Vectors are passed as torch tensors (device or host) or raw
addresses; a batch of nrhs vectors of length N is a (nrhs, N) complex64
tensor, i.e. the ABI's column-major N x nrhs layout with ld = N.  Streams are
torch.cuda.Stream objects, raw cudaStream_t handles, or None for torch's
current stream.  If the library has not been built, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

BF_OK, BF_ERR_INVALID, BF_ERR_CUDA, BF_ERR_NOMEM, BF_ERR_UNSUPPORTED, BF_ERR_TIMEOUT, BF_ERR_CORRUPT = range(7)
BF_C64, BF_C128 = 1, 2

EXPORTS = ("bf_plan_create", "bf_apply", "bf_apply_adjoint", "bf_plan_destroy", "bf_plan_check",
           "bf_plan_device_bytes", "bf_plan_set_profiling", "bf_plan_kernel_times", "bf_status_string",
           "bf_apply_static_scratch", "bf_diff_create", "bf_diff_destroy", "bf_diff_stride",
           "bf_diff_saved_bytes", "bf_diff_forward", "bf_diff_backward", "bf_batch_create", "bf_batch_apply",
           "bf_batch_check", "bf_batch_items", "bf_batch_destroy", "bf_plan_set_precision", "bf_quad_create",
           "bf_quad_apply", "bf_quad_device_bytes", "bf_quad_passes", "bf_quad_destroy", "bf_quad_tc_passes",
           "bf_quad_set_precision", "bf_quad_check", "bf_sketch_products", "bf_factor_file_check",
           "bf_plan_create_from_file", "bf_crc32")
BF_PREC_FP32, BF_PREC_TF32, BF_PREC_BF16X3, BF_PREC_BF16, BF_PREC_BF16X6 = 0, 1, 2, 3, 4
BF_BATCH_EACH, BF_BATCH_GROUPED, BF_BATCH_GRAPH = 0, 1, 2


class BfError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {bf_status_string(status)} (status {status})")
        self.status = status


class BfArgumentError(BfError, ValueError):
    """An argument the wrapper rejects before calling the library (status
    BF_ERR_INVALID, as the C ABI would report it, but raised for checks the
    ABI cannot make: buffer sizes, dtypes and devices)."""

    def __init__(self, msg: str):
        RuntimeError.__init__(self, f"{msg}: BF_ERR_INVALID (status {BF_ERR_INVALID})")
        self.status = BF_ERR_INVALID


class bf_desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("leaf", ctypes.c_int), ("r", ctypes.c_int), ("nrhs_max", ctypes.c_int)]


class bf_factors(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("VL", ctypes.c_void_p), ("H", ctypes.POINTER(ctypes.c_void_p)),
                ("S", ctypes.c_void_p), ("G", ctypes.POINTER(ctypes.c_void_p)), ("UL", ctypes.c_void_p)]


class bf_dfactors(ctypes.Structure):
    _fields_ = [("VL", ctypes.c_void_p), ("H", ctypes.POINTER(ctypes.c_void_p)), ("S", ctypes.c_void_p),
                ("G", ctypes.POINTER(ctypes.c_void_p)), ("UL", ctypes.c_void_p)]


bf_dgrads = bf_dfactors   # same shape: device pointers (written by the backward pass)


class bf_batch_config(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("slot_kb", ctypes.c_int), ("stages", ctypes.c_int),
                ("route_min_rhs", ctypes.c_int), ("route_min_L", ctypes.c_int)]


class bf_sketch_desc(ctypes.Structure):
    _fields_ = [("log2N", ctypes.c_int), ("nb", ctypes.c_int), ("k", ctypes.c_int), ("node0", ctypes.c_int),
                ("nodes", ctypes.c_int), ("lo", ctypes.c_longlong), ("hi", ctypes.c_longlong),
                ("adjoint", ctypes.c_int)]


class bf_diff_desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("leaf", ctypes.c_int), ("r", ctypes.c_int), ("nrhs_max", ctypes.c_int),
                ("stride", ctypes.c_int), ("saved_budget", ctypes.c_size_t)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libbfly.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libbfly.so not found at {p}: build it with paper_1502_01379_gb300.build.build()")
    L = ctypes.CDLL(p)
    vp, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    sig = {
        "bf_plan_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(bf_desc), ctypes.POINTER(bf_factors), vp]),
        "bf_apply": (i, [vp, vp, vp, i, ll, vp]),
        "bf_apply_adjoint": (i, [vp, vp, vp, i, ll, vp]),
        "bf_plan_destroy": (i, [vp]),
        "bf_plan_check": (i, [vp, vp]),
        "bf_plan_device_bytes": (ctypes.c_size_t, [vp]),
        "bf_plan_set_profiling": (i, [vp, i]),
        "bf_plan_kernel_times": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double)]),
        "bf_status_string": (ctypes.c_char_p, [i]),
        "bf_apply_static_scratch": (i, [vp, vp, vp, i, ll, i, vp]),
        "bf_batch_create": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(bf_desc), ctypes.POINTER(bf_factors),
                                ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i),
                                ctypes.POINTER(ll), ctypes.POINTER(bf_batch_config), vp]),
        "bf_batch_apply": (i, [vp, i, i, vp]),
        "bf_plan_set_precision": (i, [vp, i]),
        "bf_batch_check": (i, [vp, vp]),
        "bf_batch_items": (i, [vp]),
        "bf_batch_destroy": (i, [vp]),
        "bf_quad_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(bf_desc), ctypes.POINTER(bf_factors), vp]),
        "bf_quad_apply": (i, [vp, vp, vp, i, ll, i, vp]),
        "bf_quad_device_bytes": (ctypes.c_size_t, [vp]),
        "bf_quad_passes": (i, [vp]),
        "bf_quad_destroy": (i, [vp]),
        "bf_quad_tc_passes": (i, [vp]),
        "bf_quad_set_precision": (i, [vp, i]),
        "bf_quad_check": (i, [vp, vp]),
        "bf_sketch_products": (i, [ctypes.POINTER(bf_sketch_desc), vp, vp, vp, vp]),
        "bf_factor_file_check": (i, [ctypes.c_char_p, ctypes.POINTER(bf_desc), ctypes.POINTER(i)]),
        "bf_plan_create_from_file": (i, [ctypes.POINTER(vp), ctypes.c_char_p, i, vp]),
        "bf_crc32": (ctypes.c_uint, [vp, ctypes.c_size_t, ctypes.c_uint]),
        "bf_diff_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(bf_diff_desc)]),
        "bf_diff_destroy": (i, [vp]),
        "bf_diff_stride": (i, [vp]),
        "bf_diff_saved_bytes": (ctypes.c_size_t, [vp, i]),
        "bf_diff_forward": (i, [vp, ctypes.POINTER(bf_dfactors), vp, vp, i, ll, vp, vp]),
        "bf_diff_backward": (i, [vp, ctypes.POINTER(bf_dfactors), vp, vp, i, ll, vp, ctypes.POINTER(bf_dfactors),
                                 vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def bf_status_string(status: int) -> str:
    return load().bf_status_string(int(status)).decode()


def _check(status: int, what: str) -> None:
    if status != BF_OK:
        raise BfError(status, what)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _addr(x) -> int:
    """Address of a raw pointer, numpy array or torch tensor; arrays must be
    contiguous (the ABI reads them as dense row-major buffers)."""
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return int(x.ctypes.data)
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return int(x.data_ptr())


class Plan:
    """Owns a bf_plan handle and the host arrays kept alive during creation."""

    def __init__(self, handle: int, N: int, L: int, n0: int, r: int, nrhs_max: int, device: int | None = None):
        self.handle, self.N, self.L, self.n0, self.r, self.nrhs_max = handle, N, L, n0, r, nrhs_max
        self.device = device          # CUDA device index the plan was created on

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self) -> None:
        if getattr(self, "handle", None):
            load().bf_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = None


def _host_factors(factors):
    """bf_factors of host arrays (complex64 or complex128); returns (struct, keep-alive)."""
    c128 = np.asarray(factors.VL).dtype == np.complex128
    cdt, rdt = (np.complex128, np.float64) if c128 else (np.complex64, np.float32)
    keep = [np.ascontiguousarray(factors.VL, cdt), np.ascontiguousarray(factors.UL, cdt),
            np.ascontiguousarray(factors.S, rdt)]
    Hs = [np.ascontiguousarray(a, cdt) for a in factors.H]
    Gs = [np.ascontiguousarray(a, cdt) for a in factors.G]
    nh = max(1, len(Hs))
    h_arr = (ctypes.c_void_p * nh)(*[a.ctypes.data for a in Hs])
    g_arr = (ctypes.c_void_p * nh)(*[a.ctypes.data for a in Gs])
    f = bf_factors(BF_C128 if c128 else BF_C64, keep[0].ctypes.data,
                   ctypes.cast(h_arr, ctypes.POINTER(ctypes.c_void_p)), keep[2].ctypes.data,
                   ctypes.cast(g_arr, ctypes.POINTER(ctypes.c_void_p)), keep[1].ctypes.data)
    return f, (keep, Hs, Gs, h_arr, g_arr)


def bf_plan_create(factors, nrhs_max: int = 1, stream=None) -> Plan:
    """Create a plan from factors in canonical layout (any object with L, n0,
    r, VL, H, S, G, UL as numpy arrays; complex64 or complex128)."""
    f, keep = _host_factors(factors)
    d = bf_desc(int(factors.L), int(factors.n0), int(factors.r), int(nrhs_max))
    h = ctypes.c_void_p()
    _check(load().bf_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.byref(f),
                                 ctypes.c_void_p(_stream_handle(stream))), "bf_plan_create")
    del keep
    return Plan(h.value, int(factors.n0) << int(factors.L), int(factors.L), int(factors.n0),
                int(factors.r), int(nrhs_max), _current_device())


def _current_device():
    """torch's current CUDA device index, or None without CUDA."""
    try:
        import torch
        return int(torch.cuda.current_device()) if torch.cuda.is_available() else None
    except Exception:
        return None


def _check_vec(what: str, v, plan, nrhs: int, ld: int, device_only: bool) -> None:
    """The kernels read and write (nrhs - 1) * ld + N complex64 entries through
    a bare pointer, and the C ABI cannot see the buffer's size: check dtype,
    device and element count here, before the call.  Raw integer addresses
    are the caller's responsibility."""
    if isinstance(v, int):
        return
    need = (nrhs - 1) * ld + plan.N if nrhs > 0 else 0
    if isinstance(v, np.ndarray):
        if v.dtype != np.complex64:
            raise BfArgumentError(f"{what}: complex64 array required, got {v.dtype}")
        if device_only:
            raise BfArgumentError(f"{what}: a device tensor is required (host arrays are not accepted here)")
        if v.size < need:
            raise BfArgumentError(f"{what}: holds {v.size} entries, the call needs (nrhs-1)*ld+N = {need}")
        return
    import torch
    if not isinstance(v, torch.Tensor):
        raise BfArgumentError(f"{what}: expected a torch tensor, numpy array or integer address, got {type(v).__name__}")
    if v.dtype != torch.complex64:
        raise BfArgumentError(f"{what}: complex64 tensor required, got {v.dtype}")
    if v.is_cuda:
        if plan.device is not None and v.device.index != plan.device:
            raise BfArgumentError(f"{what}: tensor on cuda:{v.device.index}, plan on cuda:{plan.device}")
    elif device_only:
        raise BfArgumentError(f"{what}: a device tensor is required (host tensors are not accepted here)")
    if v.numel() < need:
        raise BfArgumentError(f"{what}: holds {v.numel()} entries, the call needs (nrhs-1)*ld+N = {need}")


def _vec_args(plan, x, y, nrhs, ld, device_only: bool = False):
    if nrhs is None:
        nrhs = 1 if isinstance(x, int) or x.ndim == 1 else int(x.shape[0])
    if ld is None:
        ld = plan.N
    nrhs, ld = int(nrhs), int(ld)
    if nrhs < 0 or ld < plan.N:
        raise BfArgumentError(f"nrhs must be >= 0 and ld >= N = {plan.N} (got nrhs={nrhs}, ld={ld})")
    _check_vec("input", x, plan, nrhs, ld, device_only)
    _check_vec("output", y, plan, nrhs, ld, device_only)
    return _addr(x), _addr(y), nrhs, ld


def bf_apply(plan: Plan, x, y, nrhs: int | None = None, ld: int | None = None, stream=None) -> None:
    """y = K_bf x (asynchronous on `stream`)."""
    xi, yi, n, l = _vec_args(plan, x, y, nrhs, ld)
    _check(load().bf_apply(ctypes.c_void_p(plan.handle), ctypes.c_void_p(xi), ctypes.c_void_p(yi), n, l,
                           ctypes.c_void_p(_stream_handle(stream))), "bf_apply")


def bf_apply_adjoint(plan: Plan, x, y, nrhs: int | None = None, ld: int | None = None, stream=None) -> None:
    """y = K_bf^* x (asynchronous on `stream`)."""
    xi, yi, n, l = _vec_args(plan, x, y, nrhs, ld)
    _check(load().bf_apply_adjoint(ctypes.c_void_p(plan.handle), ctypes.c_void_p(xi), ctypes.c_void_p(yi), n, l,
                                   ctypes.c_void_p(_stream_handle(stream))), "bf_apply_adjoint")


class QuadPlan:
    """Owns a bf_quad handle (2D factorization on quadtrees)."""

    def __init__(self, handle: int, N: int, L: int, n0: int, r: int, nrhs_max: int, device: int | None = None):
        self.handle, self.N, self.L, self.n0, self.r, self.nrhs_max = handle, N, L, n0, r, nrhs_max
        self.device = device          # CUDA device index the plan was created on

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self) -> None:
        if getattr(self, "handle", None):
            load().bf_quad_destroy(ctypes.c_void_p(self.handle))
            self.handle = None


def bf_quad_create(factors, nrhs_max: int = 1, stream=None) -> QuadPlan:
    """Create a 2D plan from quadtree factors in canonical layout (an object
    with L, n0, r, VL, H, S, G, UL; complex64 or complex128)."""
    f, keep = _host_factors(factors)
    d = bf_desc(int(factors.L), int(factors.n0), int(factors.r), int(nrhs_max))
    h = ctypes.c_void_p()
    _check(load().bf_quad_create(ctypes.byref(h), ctypes.byref(d), ctypes.byref(f),
                                 ctypes.c_void_p(_stream_handle(stream))), "bf_quad_create")
    del keep
    return QuadPlan(h.value, int(factors.n0) << (2 * int(factors.L)), int(factors.L), int(factors.n0),
                    int(factors.r), int(nrhs_max), _current_device())


def bf_quad_apply(plan: QuadPlan, x, y, nrhs: int | None = None, ld: int | None = None, adjoint: bool = False,
                  stream=None) -> None:
    """y = K_bf x (or K_bf^* x) for a 2D plan; device tensors (asynchronous)."""
    xi, yi, n, l = _vec_args(plan, x, y, nrhs, ld, device_only=True)
    _check(load().bf_quad_apply(ctypes.c_void_p(plan.handle), ctypes.c_void_p(xi), ctypes.c_void_p(yi), n, l,
                                1 if adjoint else 0, ctypes.c_void_p(_stream_handle(stream))), "bf_quad_apply")


def bf_quad_device_bytes(plan: QuadPlan) -> int:
    return int(load().bf_quad_device_bytes(ctypes.c_void_p(plan.handle)))


def bf_quad_passes(plan: QuadPlan) -> int:
    return int(load().bf_quad_passes(ctypes.c_void_p(plan.handle)))


def bf_quad_tc_passes(plan: QuadPlan) -> int:
    return int(load().bf_quad_tc_passes(ctypes.c_void_p(plan.handle)))


def bf_quad_set_precision(plan: QuadPlan, precision: int) -> None:
    """Operand precision of a 2D plan's tensor-core levels (the rungs of bf_plan_set_precision)."""
    _check(load().bf_quad_set_precision(ctypes.c_void_p(plan.handle), int(precision)), "bf_quad_set_precision")


def bf_quad_check(plan: QuadPlan, stream=None) -> None:
    """Raises BfError(BF_ERR_TIMEOUT) if a tensor-core wait expired since the last check."""
    _check(load().bf_quad_check(ctypes.c_void_p(plan.handle), ctypes.c_void_p(_stream_handle(stream))),
           "bf_quad_check")


def bf_quad_destroy(plan: QuadPlan) -> None:
    plan.destroy()


def bf_plan_set_precision(plan: Plan, precision: int) -> None:
    """Operand precision of the tensor-core core: BF_PREC_FP32 (3xTF32, the
    default), BF_PREC_TF32, BF_PREC_BF16X6 (BF16 hi/mid/lo split),
    BF_PREC_BF16X3 (BF16 hi/lo split) or BF_PREC_BF16."""
    _check(load().bf_plan_set_precision(ctypes.c_void_p(plan.handle), int(precision)), "bf_plan_set_precision")


def bf_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def bf_plan_check(plan: Plan, stream=None) -> None:
    """Raise BfError(BF_ERR_TIMEOUT) if a kernel gave up on a bounded wait."""
    _check(load().bf_plan_check(ctypes.c_void_p(plan.handle), ctypes.c_void_p(_stream_handle(stream))),
           "bf_plan_check")


def bf_plan_device_bytes(plan: Plan) -> int:
    return int(load().bf_plan_device_bytes(ctypes.c_void_p(plan.handle)))


def bf_plan_set_profiling(plan: Plan, enable: bool) -> None:
    _check(load().bf_plan_set_profiling(ctypes.c_void_p(plan.handle), 1 if enable else 0), "bf_plan_set_profiling")


def bf_plan_kernel_times(plan: Plan) -> dict:
    """{'down': (launches, ms), 'up': (launches, ms)} since the last call."""
    dl, ul = ctypes.c_int(), ctypes.c_int()
    dm, um = ctypes.c_double(), ctypes.c_double()
    _check(load().bf_plan_kernel_times(ctypes.c_void_p(plan.handle), ctypes.byref(dl), ctypes.byref(dm),
                                       ctypes.byref(ul), ctypes.byref(um)), "bf_plan_kernel_times")
    return {"down": (dl.value, dm.value), "up": (ul.value, um.value)}


def bf_apply_static_scratch(plan: Plan, x, y, nrhs: int | None = None, ld: int | None = None,
                            adjoint: bool = False, stream=None) -> None:
    """y = K_bf x (or K_bf^* x) without any device allocation: the
    intermediate vector lives in the library's fixed 16 MiB device array.
    Device tensors only; calls that overlap on the GPU race."""
    xi, yi, n, l = _vec_args(plan, x, y, nrhs, ld, device_only=True)
    _check(load().bf_apply_static_scratch(ctypes.c_void_p(plan.handle), ctypes.c_void_p(xi), ctypes.c_void_p(yi),
                                          n, l, 1 if adjoint else 0, ctypes.c_void_p(_stream_handle(stream))),
           "bf_apply_static_scratch")


# ------------------------------------------------------------- differentiation
class DiffPlan:
    """Owns a bf_diff handle (reverse-mode plan)."""

    def __init__(self, handle: int, L: int, n0: int, r: int, nrhs_max: int):
        self.handle, self.L, self.n0, self.r, self.nrhs_max = handle, L, n0, r, nrhs_max
        self.N = n0 << L

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self) -> None:
        if getattr(self, "handle", None):
            load().bf_diff_destroy(ctypes.c_void_p(self.handle))
            self.handle = None


def bf_diff_create(L: int, leaf: int, r: int, nrhs_max: int, stride: int = 0, saved_budget: int = 0) -> DiffPlan:
    d = bf_diff_desc(int(L), int(leaf), int(r), int(nrhs_max), int(stride), int(saved_budget))
    h = ctypes.c_void_p()
    _check(load().bf_diff_create(ctypes.byref(h), ctypes.byref(d)), "bf_diff_create")
    return DiffPlan(h.value, int(L), int(leaf), int(r), int(nrhs_max))


def bf_diff_destroy(plan: DiffPlan) -> None:
    plan.destroy()


def bf_diff_stride(plan: DiffPlan) -> int:
    return int(load().bf_diff_stride(ctypes.c_void_p(plan.handle)))


def bf_diff_saved_bytes(plan: DiffPlan, nrhs: int) -> int:
    return int(load().bf_diff_saved_bytes(ctypes.c_void_p(plan.handle), int(nrhs)))


def _dfactors(VL, H, S, G, UL):
    """bf_dfactors of device tensors (or addresses); returns (struct, keep-alive)."""
    nh = max(1, len(H))
    h_arr = (ctypes.c_void_p * nh)(*[_addr(a) for a in H])
    g_arr = (ctypes.c_void_p * nh)(*[_addr(a) for a in G])
    f = bf_dfactors(_addr(VL), ctypes.cast(h_arr, ctypes.POINTER(ctypes.c_void_p)), _addr(S),
                    ctypes.cast(g_arr, ctypes.POINTER(ctypes.c_void_p)), _addr(UL))
    return f, (h_arr, g_arr)


def bf_diff_forward(plan: DiffPlan, factors, g, u, saved, nrhs: int | None = None, ld: int | None = None,
                    stream=None) -> None:
    """u = K_bf g keeping checkpoints in `saved`; factors = (VL, H, S, G, UL) device tensors."""
    f, keep = _dfactors(*factors)
    n = (1 if g.ndim == 1 else int(g.shape[0])) if nrhs is None else int(nrhs)
    _check(load().bf_diff_forward(ctypes.c_void_p(plan.handle), ctypes.byref(f), ctypes.c_void_p(_addr(g)),
                                  ctypes.c_void_p(_addr(u)), n, int(ld or plan.N), ctypes.c_void_p(_addr(saved)),
                                  ctypes.c_void_p(_stream_handle(stream))), "bf_diff_forward")
    del keep


def bf_diff_backward(plan: DiffPlan, factors, ubar, gbar, saved, grads, nrhs: int | None = None,
                     ld: int | None = None, stream=None) -> None:
    """gbar = K_bf^* ubar and the factor gradients into grads = (VL, H, S, G, UL)."""
    f, keep = _dfactors(*factors)
    gr, keep2 = _dfactors(*grads)
    n = (1 if ubar.ndim == 1 else int(ubar.shape[0])) if nrhs is None else int(nrhs)
    _check(load().bf_diff_backward(ctypes.c_void_p(plan.handle), ctypes.byref(f), ctypes.c_void_p(_addr(ubar)),
                                   ctypes.c_void_p(_addr(gbar)), n, int(ld or plan.N),
                                   ctypes.c_void_p(_addr(saved)), ctypes.byref(gr),
                                   ctypes.c_void_p(_stream_handle(stream))), "bf_diff_backward")
    del keep, keep2


# ----------------------------------------------------------------- batches
class Batch:
    """Owns a bf_batch handle; keeps the bound vectors alive."""

    def __init__(self, handle: int, n: int, keep):
        self.handle, self.n, self._keep = handle, n, keep

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def destroy(self) -> None:
        if getattr(self, "handle", None):
            load().bf_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None


def bf_batch_create(factors_list, ins, outs, nrhs, T: int = 1, slot_kb: int = 0, stages: int = 0,
                    route_min_rhs: int = 0, route_min_L: int = 0, stream=None) -> Batch:
    """A batch of operators (factors in canonical layout, host arrays) bound to
    device vectors ins[o], outs[o] of shape (nrhs[o], N_o) complex64.
    Operators with at least ``route_min_rhs`` vectors (0: 8; negative: none)
    and depth at least ``route_min_L`` (0: 6) run their own multi-RHS passes."""
    n = len(factors_list)
    descs = (bf_desc * n)()
    facs = (bf_factors * n)()
    keep = []
    for o, F in enumerate(factors_list):
        descs[o] = bf_desc(int(F.L), int(F.n0), int(F.r), int(nrhs[o]))
        f, k = _host_factors(F)
        facs[o] = f
        keep.append(k)
    in_arr = (ctypes.c_void_p * n)(*[_addr(x) for x in ins])
    out_arr = (ctypes.c_void_p * n)(*[_addr(x) for x in outs])
    nr = (ctypes.c_int * n)(*[int(x) for x in nrhs])
    lds = (ctypes.c_longlong * n)(*[int(F.n0) << int(F.L) for F in factors_list])
    cfg = bf_batch_config(int(T), int(slot_kb), int(stages), int(route_min_rhs), int(route_min_L))
    h = ctypes.c_void_p()
    _check(load().bf_batch_create(ctypes.byref(h), n, descs, facs, in_arr, out_arr, nr, lds, ctypes.byref(cfg),
                                  ctypes.c_void_p(_stream_handle(stream))), "bf_batch_create")
    del keep
    return Batch(h.value, n, (list(ins), list(outs)))


def bf_batch_apply(batch: Batch, adjoint: bool = False, mode: int = BF_BATCH_GRAPH, stream=None) -> None:
    _check(load().bf_batch_apply(ctypes.c_void_p(batch.handle), 1 if adjoint else 0, int(mode),
                                 ctypes.c_void_p(_stream_handle(stream))), "bf_batch_apply")


def bf_batch_check(batch: Batch, stream=None) -> None:
    _check(load().bf_batch_check(ctypes.c_void_p(batch.handle), ctypes.c_void_p(_stream_handle(stream))),
           "bf_batch_check")


def bf_batch_items(batch: Batch) -> int:
    return int(load().bf_batch_items(ctypes.c_void_p(batch.handle)))


def bf_batch_destroy(batch: Batch) -> None:
    batch.destroy()


# ------------------------------------------------------------ sketch products
def bf_sketch_products(log2N: int, nb: int, blocks, out, lo: int, hi: int, node0: int = 0,
                       adjoint: bool = False, c_fixed=None, stream=None) -> None:
    """Products of K(x_j, xi_k) = exp(2 pi i (x_j xi_k + c_j |xi_k|)) (or K^*)
    with sketch blocks, rows [lo, hi) of the result (include/bfly.h).
    ``blocks``: (nodes, nb, k) complex64 device tensor; ``out``: (nodes, k,
    hi - lo) complex64 device tensor; ``c_fixed``: (N,) int64 device tensor
    holding c_j 2^64 as unsigned bits, or None for c = 0."""
    import torch
    for name, t, shape in (("blocks", blocks, None), ("out", out, None)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
            raise BfArgumentError(f"{name}: contiguous complex64 device tensor required")
    nodes, nbb, k = blocks.shape
    if nbb != nb or tuple(out.shape) != (nodes, k, hi - lo):
        raise BfArgumentError(f"shapes: blocks {tuple(blocks.shape)}, out {tuple(out.shape)}, nb {nb}, rows {hi - lo}")
    if c_fixed is not None and (not isinstance(c_fixed, torch.Tensor) or c_fixed.dtype != torch.int64 or
                                not c_fixed.is_cuda or c_fixed.numel() != (1 << log2N)):
        raise BfArgumentError("c_fixed: (N,) int64 device tensor required")
    d = bf_sketch_desc(int(log2N), int(nb), int(k), int(node0), int(nodes), int(lo), int(hi), 1 if adjoint else 0)
    _check(load().bf_sketch_products(ctypes.byref(d), ctypes.c_void_p(0 if c_fixed is None else c_fixed.data_ptr()),
                                     ctypes.c_void_p(blocks.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(_stream_handle(stream))), "bf_sketch_products")


# ------------------------------------------------------------------ factor files
FACTOR_FILE_VERSION = 1


def bf_crc32(data: bytes, crc: int = 0) -> int:
    """The library's CRC-32 (the factor files' checksum) of a bytes object."""
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    return int(load().bf_crc32(ctypes.cast(buf, ctypes.c_void_p), len(data), crc))


def bf_factor_file_save(factors, path: str, dtype=np.complex64) -> int:
    """Writes a factor file (the layout of include/bfly.h: 64-byte header with
    magic, version, dtype, shape, payload size and CRC-32s; payload VL, H, S,
    G, UL in canonical order) for `bf_plan_create_from_file`.  The checksum is
    zlib's CRC-32, the same function as the library's.  Returns the bytes
    written."""
    import struct
    import zlib
    cdt = np.dtype(dtype)
    if cdt not in (np.dtype(np.complex64), np.dtype(np.complex128)):
        raise ValueError("dtype must be complex64 or complex128")
    rdt = np.float32 if cdt == np.complex64 else np.float64
    S = np.ascontiguousarray(factors.S, rdt).tobytes()
    S += b"\0" * (-len(S) % 8)
    parts = [np.ascontiguousarray(factors.VL, cdt)] + [np.ascontiguousarray(a, cdt) for a in factors.H] + \
        [S] + [np.ascontiguousarray(a, cdt) for a in factors.G] + [np.ascontiguousarray(factors.UL, cdt)]
    crc, size = 0, 0
    for a in parts:
        b = memoryview(a if isinstance(a, bytes) else a.reshape(-1).view(np.uint8))
        crc = zlib.crc32(b, crc)
        size += b.nbytes
    head = b"BFLYFAC\0" + struct.pack("<IIiiiIQI", FACTOR_FILE_VERSION, BF_C64 if cdt == np.complex64 else BF_C128,
                                      int(factors.L), int(factors.n0), int(factors.r), 0, size, crc)
    head += struct.pack("<I", zlib.crc32(head)) + b"\0" * 16
    with open(path, "wb") as f:
        f.write(head)
        for a in parts:
            f.write(a if isinstance(a, bytes) else a.reshape(-1).view(np.uint8).data)
    return len(head) + size


def bf_factor_file_check(path: str):
    """(L, leaf, r, dtype) of a verified factor file; raises BfError
    (BF_ERR_CORRUPT, BF_ERR_UNSUPPORTED or BF_ERR_INVALID) otherwise."""
    d = bf_desc()
    dt = ctypes.c_int()
    _check(load().bf_factor_file_check(os.fsencode(path), ctypes.byref(d), ctypes.byref(dt)), "bf_factor_file_check")
    return d.L, d.leaf, d.r, dt.value


def bf_plan_create_from_file(path: str, nrhs_max: int = 1, stream=None) -> Plan:
    """A plan from a factor file (verified before any CUDA call)."""
    L, leaf, r, _ = bf_factor_file_check(path)
    h = ctypes.c_void_p()
    _check(load().bf_plan_create_from_file(ctypes.byref(h), os.fsencode(path), int(nrhs_max),
                                           ctypes.c_void_p(_stream_handle(stream))), "bf_plan_create_from_file")
    return Plan(h.value, leaf << L, L, leaf, r, int(nrhs_max), _current_device())
