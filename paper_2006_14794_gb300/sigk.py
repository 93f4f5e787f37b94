"""Thin Python binding of libsigk (include/sigk.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
only checks tensors, allocates outputs with PyTorch, and passes device
pointers and the current CUDA stream through ``ctypes``.  Importing it does
not need a GPU; calling it needs the built ``libsigk.so`` and fails loudly when
it is missing (there is no CPU fallback).

Names follow the C ABI: ``pairs``, ``gram``, ``pairs_varlen``,
``pairs_surface``, ``pairs_backward``, ``gram_backward``, ``gram_value_and_grad``, ``mmd2``,
``scale_grad``; the autograd wrappers are
``SigKernelPairs``, ``SigKernelGram`` and ``mmd2_loss``.
"""
from __future__ import annotations

import ctypes
import os
from typing import NamedTuple, Optional, Union

import torch

from . import build as _build

SIGK_OK, SIGK_EINVAL, SIGK_ENOMEM_WS, SIGK_ECUDA, SIGK_ETIMEOUT, SIGK_EUNSUPPORTED = range(6)
SIGK_F32, SIGK_F64 = 0, 1
REC_AUTO, REC_CHAIN, REC_PLAIN, REC_STRIP, REC_BAND = 0, 1, 2, 3, 4
COEF_AUTO, COEF_FMA, COEF_TC, COEF_TC5 = 0, 1, 2, 3
OP_PAIRS, OP_GRAM, OP_PAIRS_VARLEN, OP_PAIRS_BACKWARD, OP_GRAM_BACKWARD, OP_PAIRS_SURFACE = range(6)

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


SCHEME_EXPLICIT, SCHEME_IMPLICIT = 0, 1
KERNEL_LINEAR, KERNEL_RBF = 0, 1
SCHEMES = {"explicit": SCHEME_EXPLICIT, "implicit": SCHEME_IMPLICIT}
STATIC_KERNELS = {"linear": KERNEL_LINEAR, "rbf": KERNEL_RBF}


class SigkOpts(ctypes.Structure):
    _fields_ = [("rec", _int), ("symmetric", _int), ("fault_inject", _int),
                ("rows_per_lane", _int), ("coef_path", _int), ("orient", _int),
                ("scheme", _int), ("static_kernel", _int), ("sigma", ctypes.c_double),
                ("accumulate", _int), ("reserved", _int * 1)]


class Variant(NamedTuple):
    """What a call solves (the fields of sigk_opts that change the result):
    the finite-difference scheme ("explicit", or "implicit": the four-point
    quadrature of the remark after the scheme, Sec. 3.1) and the static kernel
    that lifts the paths ("linear": the paths as given, or "rbf" with bandwidth
    sigma, Sec. 2.2)."""
    scheme: str = "explicit"
    static_kernel: str = "linear"
    sigma: float = 1.0

    def key(self) -> str:
        """'' for the paper's main variant, else a tag for caches."""
        if self.scheme == "explicit" and self.static_kernel == "linear":
            return ""
        return "%s/%s/%r" % (self.scheme, self.static_kernel,
                             float(self.sigma) if self.static_kernel == "rbf" else 0.0)


DEFAULT_VARIANT = Variant()


def _variant(variant) -> Variant:
    if variant is None:
        return DEFAULT_VARIANT
    if not isinstance(variant, Variant):
        raise TypeError("variant must be a sigk.Variant")
    if variant.scheme not in SCHEMES or variant.static_kernel not in STATIC_KERNELS:
        raise ValueError("unknown scheme or static kernel: %r" % (variant,))
    return variant


class Schedule(NamedTuple):
    """How a call is scheduled (the fields of sigk_opts that pick the kernels):
    rec (REC_*), rows_per_lane (4, 8, 16; 0 = default: the band height of the
    chained and band kernels, the strip height of the strip path), the strip
    path's coefficient kernel (COEF_*) and which path its rows refine (orient:
    0 auto, 1 longer, 2 shorter).  Every schedule computes the same scheme;
    they differ in speed only."""
    rec: int = REC_AUTO
    rows_per_lane: int = 0
    coef_path: int = COEF_AUTO
    orient: int = 0


_lib = None

# (name, restype, argtypes) of every symbol include/sigk.h declares
SIGNATURES = [
    ("sigk_workspace_bytes", ctypes.c_size_t,
     [_int, _i64, _i64, _i64, _i64, _i64, _int, _int, _vp]),
    ("sigk_pairs", _int, [_vp, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp, _vp, _vp,
                          ctypes.c_size_t, _vp]),
    ("sigk_gram", _int, [_vp, _vp, _i64, _i64, _i64, _i64, _i64, _int, _int, _vp, _vp, _vp,
                         ctypes.c_size_t, _vp]),
    ("sigk_pairs_varlen", _int, [_vp, _vp, _vp, _vp, _i64, _i64, _i64, _int, _int, _vp, _vp,
                                 _vp, ctypes.c_size_t, _vp]),
    ("sigk_pairs_surface", _int, [_vp, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp, _vp, _vp, _vp,
                                  ctypes.c_size_t, _vp]),
    ("sigk_pairs_backward", _int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _int, _int, _vp, _vp,
                                   _vp, _vp, ctypes.c_size_t, _vp]),
    ("sigk_gram_backward", _int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _int, _int, _vp,
                                  _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    ("sigk_gram_value_and_grad", _int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _int, _int, _vp,
                                        _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    ("sigk_pairs_backward_noalloc", _int, [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _int, _int,
                                           _vp, _vp, _vp]),
    ("sigk_mmd2", _int, [_vp, _vp, _vp, _i64, _i64, _int, _vp, _vp]),
    ("sigk_scale_grad", _int, [_vp, _vp, _vp, _i64, _int, _vp]),
    ("sigk_support_reduction", _int, [_vp, _vp, _vp, _i64, ctypes.c_double, ctypes.c_double, _int,
                                      _int, _vp, _vp]),
    ("sigk_mmd2_backward", _int, [_vp, _i64, _i64, _int, _vp, _vp, _vp, _vp]),
    ("sigk_stream_status", _int, [_vp, _vp]),
    ("sigk_strerror", ctypes.c_char_p, [_int]),
    ("sigk_version", ctypes.c_char_p, []),
]


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """The loaded libsigk.so.  Builds it in-tree when missing (needs nvcc)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError("libsigk.so is not built: %s" % path)
            _build.build()
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SigkError(RuntimeError):
    """A libsigk call returned an error; ``status`` is its sigk_status code."""

    def __init__(self, msg: str, status: int = -1):
        super().__init__(msg)
        self.status = status


def _check(status: int, what: str):
    if status != SIGK_OK:
        msg = lib().sigk_strerror(status).decode()
        raise SigkError("%s failed: %s (status %d)" % (what, msg, status), status)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return SIGK_F32
    if t.dtype == torch.float64:
        return SIGK_F64
    raise TypeError("sigk works on float32 or float64 tensors, got %s" % t.dtype)


def _dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor (libsigk has no CPU path)" % name)
    return t.contiguous()


def _stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _opts(rec: int = REC_AUTO, symmetric: bool = False, fault_inject: bool = False,
          schedule: Optional[Schedule] = None, variant: Optional[Variant] = None,
          accumulate: bool = False):
    o = SigkOpts()
    o.rec = int(rec)
    v = _variant(variant)
    o.scheme = SCHEMES[v.scheme]
    o.static_kernel = STATIC_KERNELS[v.static_kernel]
    o.sigma = float(v.sigma) if v.static_kernel == "rbf" else 0.0
    if schedule is not None:
        o.rec = int(schedule.rec)
        o.rows_per_lane = int(schedule.rows_per_lane)
        o.coef_path = int(schedule.coef_path)
        o.orient = int(schedule.orient)
    o.symmetric = 1 if symmetric else 0
    o.fault_inject = 1 if fault_inject else 0
    o.accumulate = 1 if accumulate else 0
    return o


def _resolve(schedule, op, *shape_args, variant=None):
    """schedule may be None, a Schedule, or "tuned": look the shape up in the
    tuner's cache (timing the candidates on a miss)."""
    if isinstance(schedule, str):
        if schedule != "tuned":
            raise ValueError("schedule must be a Schedule, None or 'tuned'")
        from . import tune
        return tune.lookup(op, *shape_args, variant=_variant(variant))
    return schedule


def _status(ws, device):
    """Reads the workspace status word after the stream drains; raises on a
    device-side timeout."""
    if ws is None:
        return
    _check(lib().sigk_stream_status(_stream(device), ws.data_ptr()), "device status")


def _ptr(t):
    return None if t is None else t.data_ptr()


def _workspace(op, b, b2, L, M, d, lam, dt, o, device):
    n = lib().sigk_workspace_bytes(op, b, b2, L, M, d, lam, dt, ctypes.byref(o))
    if n == 0:
        return None, 0
    return torch.empty(n, dtype=torch.uint8, device=device), n


def pairs(X: torch.Tensor, Y: torch.Tensor, dyadic_order: int, rec: int = REC_AUTO,
          check_status: bool = False, fault_inject: bool = False,
          schedule: Union[Schedule, str, None] = None,
          variant: Optional[Variant] = None) -> torch.Tensor:
    """out[b] = k(X_b, Y_b).  X: [B, L, d], Y: [B, M, d] (same dtype, same CUDA device).
    check_status: synchronise and raise SigkError if a bounded device wait
    expired (strip path only).  fault_inject: test switch of sigk_opts.
    schedule: a Schedule (overrides rec) or "tuned" (the tuner's choice).
    variant: the scheme and static kernel (default: explicit, linear)."""
    X, Y = _dev(X, "X"), _dev(Y, "Y")
    if X.dim() != 3 or Y.dim() != 3 or X.shape[0] != Y.shape[0] or X.shape[2] != Y.shape[2]:
        raise ValueError("pairs wants X [B,L,d] and Y [B,M,d]")
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must share a dtype")
    B, L, d = X.shape
    M = Y.shape[1]
    dt = _dtype_code(X)
    out = torch.empty(B, dtype=X.dtype, device=X.device)
    schedule = _resolve(schedule, "pairs", X, Y, dyadic_order, variant=variant)
    o = _opts(rec, fault_inject=fault_inject, schedule=schedule, variant=variant)
    ws, nws = _workspace(OP_PAIRS, B, 0, L, M, d, dyadic_order, dt, o, X.device)
    _check(lib().sigk_pairs(X.data_ptr(), Y.data_ptr(), B, L, M, d, int(dyadic_order), dt,
                            ctypes.byref(o), out.data_ptr(), _ptr(ws), nws, _stream(X.device)),
           "sigk_pairs")
    if check_status:
        _status(ws, X.device)
    return out


def gram(X: torch.Tensor, Y: torch.Tensor, dyadic_order: int, rec: int = REC_AUTO,
         symmetric: bool = False, check_status: bool = False,
         schedule: Union[Schedule, str, None] = None,
         variant: Optional[Variant] = None) -> torch.Tensor:
    """out[i, j] = k(X_i, Y_j).  With symmetric=True, Y must be X and only the
    upper triangle is solved (then mirrored).  schedule, variant: as for pairs."""
    X, Y = _dev(X, "X"), _dev(Y, "Y")
    if X.dim() != 3 or Y.dim() != 3 or X.shape[2] != Y.shape[2]:
        raise ValueError("gram wants X [Bx,L,d] and Y [By,M,d]")
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must share a dtype")
    Bx, L, d = X.shape
    By, M = Y.shape[0], Y.shape[1]
    dt = _dtype_code(X)
    out = torch.empty(Bx, By, dtype=X.dtype, device=X.device)
    schedule = _resolve(schedule, "gram", X, Y, dyadic_order, variant=variant)
    o = _opts(rec, symmetric, schedule=schedule, variant=variant)
    ws, nws = _workspace(OP_GRAM, Bx, By, L, M, d, dyadic_order, dt, o, X.device)
    _check(lib().sigk_gram(X.data_ptr(), Y.data_ptr(), Bx, By, L, M, d, int(dyadic_order), dt,
                           ctypes.byref(o), out.data_ptr(), _ptr(ws), nws, _stream(X.device)),
           "sigk_gram")
    if check_status:
        _status(ws, X.device)
    return out


def pairs_varlen(Xp: torch.Tensor, x_off: torch.Tensor, Yp: torch.Tensor, y_off: torch.Tensor,
                 dyadic_order: int, max_len: int, rec: int = REC_AUTO, check_status: bool = False,
                 fault_inject: bool = False,
                 schedule: Union[Schedule, str, None] = None,
                 variant: Optional[Variant] = None) -> torch.Tensor:
    """Pairs of uneven lengths: Xp [sum L, d] with int64 offsets x_off [B+1] (on the GPU).
    schedule, variant: as for pairs."""
    Xp, Yp = _dev(Xp, "Xp"), _dev(Yp, "Yp")
    x_off, y_off = _dev(x_off, "x_off"), _dev(y_off, "y_off")
    if x_off.dtype != torch.int64 or y_off.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    B = x_off.shape[0] - 1
    d = Xp.shape[1]
    dt = _dtype_code(Xp)
    out = torch.empty(B, dtype=Xp.dtype, device=Xp.device)
    schedule = _resolve(schedule, "pairs_varlen", Xp, x_off, Yp, y_off, dyadic_order, max_len,
                        variant=variant)
    o = _opts(rec, fault_inject=fault_inject, schedule=schedule, variant=variant)
    ws, nws = _workspace(OP_PAIRS_VARLEN, B, 0, max_len, max_len, d, dyadic_order, dt, o,
                         Xp.device)
    _check(lib().sigk_pairs_varlen(Xp.data_ptr(), x_off.data_ptr(), Yp.data_ptr(),
                                   y_off.data_ptr(), B, d, int(max_len), int(dyadic_order), dt,
                                   ctypes.byref(o), out.data_ptr(), _ptr(ws), nws,
                                   _stream(Xp.device)), "sigk_pairs_varlen")
    if check_status:
        _status(ws, Xp.device)
    return out


def pairs_surface(X: torch.Tensor, Y: torch.Tensor, dyadic_order: int, rec: int = REC_AUTO,
                  schedule: Optional[Schedule] = None, variant: Optional[Variant] = None):
    """(k [B], surf [B, L, M]): the solution at the sample-grid nodes,
    surf[b, i, j] ~ k_{X_b, Y_b}(s_i, t_j) (row and column 0 are 1,
    surf[:, -1, -1] = k)."""
    X, Y = _dev(X, "X"), _dev(Y, "Y")
    if X.dim() != 3 or Y.dim() != 3 or X.shape[0] != Y.shape[0] or X.shape[2] != Y.shape[2]:
        raise ValueError("pairs_surface wants X [B,L,d] and Y [B,M,d]")
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must share a dtype")
    B, L, d = X.shape
    M = Y.shape[1]
    dt = _dtype_code(X)
    out = torch.empty(B, dtype=X.dtype, device=X.device)
    surf = torch.empty(B, L, M, dtype=X.dtype, device=X.device)
    o = _opts(rec, schedule=schedule, variant=variant)
    ws, nws = _workspace(OP_PAIRS_SURFACE, B, 0, L, M, d, dyadic_order, dt, o, X.device)
    _check(lib().sigk_pairs_surface(X.data_ptr(), Y.data_ptr(), B, L, M, d, int(dyadic_order), dt,
                                    ctypes.byref(o), out.data_ptr(), surf.data_ptr(), _ptr(ws), nws,
                                    _stream(X.device)), "sigk_pairs_surface")
    return out, surf


def version() -> str:
    return lib().sigk_version().decode()


def pairs_backward(grad_out: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, dyadic_order: int,
                   need_dx: bool = True, need_dy: bool = True, rec: int = REC_AUTO,
                   schedule: Optional[Schedule] = None, variant: Optional[Variant] = None,
                   check_status: bool = False, dX: Optional[torch.Tensor] = None,
                   dY: Optional[torch.Tensor] = None, accumulate: bool = False):
    """(dX, dY) with dX[b] = grad_out[b] dk(X_b, Y_b)/dX_b (None when not needed).
    check_status: as for pairs (waits for the stream, raises on a device-side
    timeout).  dX / dY: output buffers to use (else new ones); accumulate:
    add the gradients to what they hold."""
    X, Y, grad_out = _dev(X, "X"), _dev(Y, "Y"), _dev(grad_out, "grad_out")
    B, L, d = X.shape
    M = Y.shape[1]
    dt = _dtype_code(X)
    grad_out = grad_out.to(X.dtype)
    dX, dY = _grad_buffers(X, Y, need_dx, need_dy, dX, dY, accumulate)
    o = _opts(rec, schedule=schedule, variant=variant, accumulate=accumulate)
    ws, nws = _workspace(OP_PAIRS_BACKWARD, B, 0, L, M, d, dyadic_order, dt, o, X.device)
    _check(lib().sigk_pairs_backward(grad_out.data_ptr(), X.data_ptr(), Y.data_ptr(), B, L, M, d,
                                     int(dyadic_order), dt, ctypes.byref(o), _ptr(dX), _ptr(dY),
                                     _ptr(ws), nws, _stream(X.device)), "sigk_pairs_backward")
    if check_status:
        _status(ws, X.device)
    return dX, dY


def gram_backward(grad_out: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, dyadic_order: int,
                  need_dx: bool = True, need_dy: bool = True, rec: int = REC_AUTO,
                  schedule: Optional[Schedule] = None, symmetric: bool = False,
                  variant: Optional[Variant] = None, dX: Optional[torch.Tensor] = None,
                  dY: Optional[torch.Tensor] = None, accumulate: bool = False):
    """(dX, dY): dX[i] = sum_j grad_out[i,j] dk(X_i,Y_j)/dX_i, dY[j] likewise.
    symmetric=True (Y is X): (dX, None) with dX the derivative of
    sum_ij grad_out[i,j] k(X_i, X_j) through both arguments, from the pairs
    i <= j only (f32, band form; SigkError with SIGK_EUNSUPPORTED otherwise).
    dX / dY, accumulate: as for pairs_backward."""
    X, Y, grad_out = _dev(X, "X"), _dev(Y, "Y"), _dev(grad_out, "grad_out")
    Bx, L, d = X.shape
    By, M = Y.shape[0], Y.shape[1]
    dt = _dtype_code(X)
    grad_out = grad_out.to(X.dtype).contiguous()
    if symmetric:
        need_dx, need_dy = True, False
    dX, dY = _grad_buffers(X, Y, need_dx, need_dy, dX, dY, accumulate)
    o = _opts(rec, symmetric=symmetric, schedule=schedule, variant=variant, accumulate=accumulate)
    ws, nws = _workspace(OP_GRAM_BACKWARD, Bx, By, L, M, d, dyadic_order, dt, o, X.device)
    _check(lib().sigk_gram_backward(grad_out.data_ptr(), X.data_ptr(), Y.data_ptr(), Bx, By, L, M,
                                    d, int(dyadic_order), dt, ctypes.byref(o), _ptr(dX), _ptr(dY),
                                    _ptr(ws), nws, _stream(X.device)), "sigk_gram_backward")
    return dX, dY


def gram_value_and_grad(grad_out: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, dyadic_order: int,
                        need_dx: bool = True, need_dy: bool = True, rec: int = REC_AUTO,
                        schedule: Optional[Schedule] = None, symmetric: bool = False,
                        variant: Optional[Variant] = None, dX: Optional[torch.Tensor] = None,
                        dY: Optional[torch.Tensor] = None, accumulate: bool = False):
    """(K, dX, dY) in one pass: K as gram computes it and (dX, dY) as
    gram_backward computes them for grad_out, for a grad_out known before K (a
    loss linear in the Gram).  The band backward's forward sweep writes K.
    dX / dY: output buffers to use (else new ones); accumulate: add the
    gradients to what they hold.  SigkError with SIGK_EUNSUPPORTED where the
    backward is not the band form; the caller then calls gram and
    gram_backward."""
    X, Y, grad_out = _dev(X, "X"), _dev(Y, "Y"), _dev(grad_out, "grad_out")
    Bx, L, d = X.shape
    By, M = Y.shape[0], Y.shape[1]
    dt = _dtype_code(X)
    grad_out = grad_out.to(X.dtype).contiguous()
    if symmetric:
        need_dx, need_dy = True, False
    out = torch.empty(Bx, By, dtype=X.dtype, device=X.device)
    dX, dY = _grad_buffers(X, Y, need_dx, need_dy, dX, dY, accumulate)
    o = _opts(rec, symmetric=symmetric, schedule=schedule, variant=variant, accumulate=accumulate)
    ws, nws = _workspace(OP_GRAM_BACKWARD, Bx, By, L, M, d, dyadic_order, dt, o, X.device)
    _check(lib().sigk_gram_value_and_grad(grad_out.data_ptr(), X.data_ptr(), Y.data_ptr(), Bx, By, L, M,
                                          d, int(dyadic_order), dt, ctypes.byref(o), out.data_ptr(),
                                          _ptr(dX), _ptr(dY), _ptr(ws), nws, _stream(X.device)),
           "sigk_gram_value_and_grad")
    return out, dX, dY


def _out_buffer(t: torch.Tensor, like: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.shape != like.shape or t.dtype != like.dtype or \
            t.device != like.device or not t.is_contiguous():
        raise ValueError("%s must be a contiguous tensor shaped like its input" % name)
    return t


def _grad_buffers(X, Y, need_dx, need_dy, dX, dY, accumulate):
    """The backward's output buffers: the caller's (checked), else new ones."""
    if accumulate and ((need_dx and dX is None) or (need_dy and dY is None)):
        raise ValueError("accumulate wants the dX / dY buffers to add into")
    dX = (_out_buffer(dX, X, "dX") if dX is not None else torch.empty_like(X)) if need_dx else None
    dY = (_out_buffer(dY, Y, "dY") if dY is not None else torch.empty_like(Y)) if need_dy else None
    return dX, dY


def scale_grad(grad: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """grad[0] * g, for input gradients g formed with a unit upstream
    derivative (sigk_scale_grad)."""
    g = _dev(g, "g")
    grad = _dev(grad.reshape(1).to(g.dtype), "grad")
    out = torch.empty_like(g)
    _check(lib().sigk_scale_grad(grad.data_ptr(), g.data_ptr(), out.data_ptr(), g.numel(), _dtype_code(g),
                                 _stream(g.device)), "sigk_scale_grad")
    return out


def mmd2(Kxx: torch.Tensor, Kyy: torch.Tensor, Kxy: torch.Tensor) -> torch.Tensor:
    """Unbiased MMD^2 from the three Gram matrices (one element tensor)."""
    Kxx, Kyy, Kxy = _dev(Kxx, "Kxx"), _dev(Kyy, "Kyy"), _dev(Kxy, "Kxy")
    m, n = Kxx.shape[0], Kyy.shape[0]
    out = torch.empty(1, dtype=Kxx.dtype, device=Kxx.device)
    _check(lib().sigk_mmd2(Kxx.data_ptr(), Kyy.data_ptr(), Kxy.data_ptr(), m, n, _dtype_code(Kxx),
                           out.data_ptr(), _stream(Kxx.device)), "sigk_mmd2")
    return out


def mmd2_backward(grad: torch.Tensor, m: int, n: int, dtype, device):
    grad = _dev(grad.reshape(1).to(dtype), "grad")
    gxx = torch.empty(m, m, dtype=dtype, device=device)
    gyy = torch.empty(n, n, dtype=dtype, device=device)
    gxy = torch.empty(m, n, dtype=dtype, device=device)
    _check(lib().sigk_mmd2_backward(grad.data_ptr(), m, n, _dtype_code(gxx), gxx.data_ptr(),
                                    gyy.data_ptr(), gxy.data_ptr(), _stream(device)),
           "sigk_mmd2_backward")
    return gxx, gyy, gxy


def support_reduction(K: torch.Tensor, alpha: torch.Tensor, beta0: torch.Tensor, gamma: float,
                      lam: float, iters: int):
    """Moments-matching support reduction (Sec. 5.3): proximal gradient
    descent on (alpha - beta)^T K (alpha - beta) + lam |beta|_1 from beta0.
    Returns (beta after `iters` steps, loss history [iters + 1])."""
    K, alpha = _dev(K, "K"), _dev(alpha, "alpha")
    N = K.shape[0]
    if K.shape != (N, N) or alpha.shape != (N,) or tuple(beta0.shape) != (N,):
        raise ValueError("support_reduction wants K [N,N], alpha [N], beta0 [N]")
    dt = _dtype_code(K)
    alpha = alpha.to(K.dtype).contiguous()
    beta = _dev(beta0, "beta0").to(K.dtype).clone().contiguous()
    loss = torch.empty(iters + 1, dtype=K.dtype, device=K.device)
    _check(lib().sigk_support_reduction(K.data_ptr(), alpha.data_ptr(), beta.data_ptr(), N, float(gamma),
                                        float(lam), int(iters), dt, loss.data_ptr(), _stream(K.device)),
           "sigk_support_reduction")
    return beta, loss


class SigKernelPairs(torch.autograd.Function):
    """k(X_b, Y_b) with the adjoint sweep as its backward."""

    @staticmethod
    def forward(ctx, X, Y, dyadic_order, variant=None):
        ctx.save_for_backward(X, Y)
        ctx.lam = dyadic_order
        ctx.variant = variant
        return pairs(X, Y, dyadic_order, variant=variant)

    @staticmethod
    def backward(ctx, g):
        X, Y = ctx.saved_tensors
        dX, dY = pairs_backward(g, X, Y, ctx.lam, ctx.needs_input_grad[0], ctx.needs_input_grad[1],
                                variant=ctx.variant)
        return dX, dY, None, None


class SigKernelGram(torch.autograd.Function):
    """k(X_i, Y_j) with the adjoint sweep as its backward.  Given the same
    tensor twice (a Gram of X with itself) it solves only the pairs i <= j,
    forward and (where the band form applies) backward."""

    @staticmethod
    def forward(ctx, X, Y, dyadic_order, variant=None):
        ctx.save_for_backward(X, Y)
        ctx.lam = dyadic_order
        ctx.sym = X is Y
        ctx.variant = variant
        return gram(X, Y, dyadic_order, symmetric=ctx.sym, variant=variant)

    @staticmethod
    def backward(ctx, g):
        X, Y = ctx.saved_tensors
        if ctx.sym and ctx.needs_input_grad[0] and ctx.needs_input_grad[1]:
            try:
                dX, _ = gram_backward(g, X, X, ctx.lam, symmetric=True, variant=ctx.variant)
                return dX, None, None, None
            except SigkError as e:
                if e.status != SIGK_EUNSUPPORTED:
                    raise
        dX, dY = gram_backward(g, X, Y, ctx.lam, ctx.needs_input_grad[0], ctx.needs_input_grad[1],
                               variant=ctx.variant)
        return dX, dY, None, None


class _MMD2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Kxx, Kyy, Kxy):
        ctx.shape = (Kxx.shape[0], Kyy.shape[0], Kxx.dtype, Kxx.device)
        return mmd2(Kxx, Kyy, Kxy)

    @staticmethod
    def backward(ctx, g):
        m, n, dt, dev = ctx.shape
        return mmd2_backward(g, m, n, dt, dev)


class _MMD2Fused(torch.autograd.Function):
    """MMD^2 and its gradient in one forward: the loss is linear in the three
    Grams, so dL/dK is a constant matrix (sigk_mmd2_backward of 1) before any
    Gram is known, and each Gram's values and input gradient come from one
    sigk_gram_value_and_grad call; the Kxy call adds its gradients into those
    of Kxx and Kyy.  The backward scales the stored gradients by the upstream
    derivative (sigk_scale_grad)."""

    @staticmethod
    def forward(ctx, X, Y, dyadic_order, variant):
        m, n = X.shape[0], Y.shape[0]
        need_x, need_y = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        one = torch.ones(1, dtype=X.dtype, device=X.device)
        gxx, gyy, gxy = mmd2_backward(one, m, n, X.dtype, X.device)
        # a Gram whose paths need no gradient is only evaluated
        if need_x:
            Kxx, dX, _ = gram_value_and_grad(gxx, X, X, dyadic_order, symmetric=True, variant=variant)
        else:
            Kxx, dX = gram(X, X, dyadic_order, symmetric=True, variant=variant), None
        if need_y:
            Kyy, dY, _ = gram_value_and_grad(gyy, Y, Y, dyadic_order, symmetric=True, variant=variant)
        else:
            Kyy, dY = gram(Y, Y, dyadic_order, symmetric=True, variant=variant), None
        Kxy, dX, dY = gram_value_and_grad(gxy, X, Y, dyadic_order, need_x, need_y, variant=variant,
                                          dX=dX, dY=dY, accumulate=True)
        ctx.save_for_backward(dX, dY)
        return mmd2(Kxx, Kyy, Kxy)

    @staticmethod
    def backward(ctx, g):
        dX, dY = ctx.saved_tensors
        return (scale_grad(g, dX) if dX is not None else None,
                scale_grad(g, dY) if dY is not None else None, None, None)


def mmd2_loss(X: torch.Tensor, Y: torch.Tensor, dyadic_order: int,
              variant: Optional[Variant] = None) -> torch.Tensor:
    """Differentiable unbiased MMD^2 between two batches of paths, built from
    three signature-kernel Gram matrices.  When a gradient is wanted and the
    backward runs in the band form, each Gram's values and gradient come from
    one fused call (_MMD2Fused); otherwise the Grams' own autograd functions."""
    if torch.is_grad_enabled() and (X.requires_grad or Y.requires_grad):
        try:
            return _MMD2Fused.apply(X, Y, dyadic_order, variant)[0]
        except SigkError as e:
            if e.status != SIGK_EUNSUPPORTED:
                raise
    Kxx = SigKernelGram.apply(X, X, dyadic_order, variant)
    Kyy = SigKernelGram.apply(Y, Y, dyadic_order, variant)
    Kxy = SigKernelGram.apply(X, Y, dyadic_order, variant)
    return _MMD2.apply(Kxx, Kyy, Kxy)[0]


class Graphed:
    """One library call captured into a CUDA graph with static input and output
    buffers: ``g = graphed(pairs_varlen, Xp, x_off, Yp, y_off, 1, max_len=512)``
    then ``out = g(Xp2, x_off2, Yp2, y_off2)`` copies the new inputs into the
    captured buffers (same shapes) and replays the whole call (its memsets,
    planning, coefficient and sweep kernels) as one graph launch.  The
    workspace is allocated once, inside the capture's memory pool."""

    def __init__(self, fn, *args, **kwargs):
        self.static_in = [a.clone() if isinstance(a, torch.Tensor) else a for a in args]
        self.kwargs = kwargs
        dev = next(a.device for a in args if isinstance(a, torch.Tensor))
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(2):   # warm-up outside the capture (attributes, module load)
                fn(*self.static_in, **kwargs)
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self.static_out = fn(*self.static_in, **kwargs)

    def __call__(self, *args):
        for dst, src in zip(self.static_in, args):
            if isinstance(dst, torch.Tensor):
                dst.copy_(src, non_blocking=True)
        self.graph.replay()
        return self.static_out

    def replay(self):
        """Replays the captured call on the inputs already in the static buffers."""
        self.graph.replay()
        return self.static_out


def graphed(fn, *args, **kwargs) -> Graphed:
    return Graphed(fn, *args, **kwargs)
