"""Python binding of libosbf.so (the C ABI in include/osbf.h).

Argument marshalling only: every pass of the filter runs in the library's CUDA
kernels.  Tensors must be CUDA tensors, contiguous, in NCHW (H x W and P x H x W
are accepted as N = C = 1 and N = 1).  Work is enqueued on the current torch
stream of the tensor's device.  If the library is not built, every call raises:
there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libosbf.so")

OSBF_MAX_RADIUS = 16
OSBF_MAX_DEPTH = 8
_STATUS = {0: "OSBF_OK", 1: "OSBF_EINVAL", 2: "OSBF_ENOMEM", 3: "OSBF_ECUDA", 4: "OSBF_EUNSUPPORTED",
           5: "OSBF_ETIMEOUT"}
_DTYPE = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2, torch.uint8: 3}
_TIE = {"paper": 0, "appendix": 1}
_VARIANT = {"auto": 0, "tile": 1, "strip": 2}


class OSBFError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.status_name = _STATUS.get(status, str(status))
        super().__init__(f"{self.status_name}: {message}")


class _Options(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("tie", ctypes.c_int), ("maps", ctypes.c_void_p),
                ("variant", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class _Job(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("r", ctypes.c_int), ("iters", ctypes.c_int)]


_lib = None
_lock = threading.Lock()
_ctxs: dict[int, ctypes.c_void_p] = {}


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libosbf.so is not built ({LIB_PATH}); run paper_2108_05021_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
        L.osbf_create.argtypes = [ctypes.POINTER(vp), i]
        L.osbf_create.restype = st
        L.osbf_destroy.argtypes = [vp]
        L.osbf_destroy.restype = None
        L.osbf_last_error.argtypes = [vp]
        L.osbf_last_error.restype = ctypes.c_char_p
        L.osbf_last_launch_count.argtypes = [vp]
        L.osbf_last_launch_count.restype = i
        L.osbf_version.restype = ctypes.c_char_p
        L.osbf_filter.argtypes = [vp, vp, vp, i, i, i, i, i, i, i, vp]
        L.osbf_filter.restype = st
        L.osbf_filter_ex.argtypes = [vp, vp, vp, i, i, i, i, i, i, i, ctypes.POINTER(_Options), vp]
        L.osbf_filter_ex.restype = st
        L.osbf_filter_fast.argtypes = [vp, vp, vp, i, i, i, i, i, i, vp, vp]
        L.osbf_filter_fast.restype = st
        L.osbf_filter_3d.argtypes = [vp, vp, vp, i, i, i, i, i, i, i, vp, vp]
        L.osbf_filter_3d.restype = st
        L.osbf_filter_gauss.argtypes = [vp, vp, vp, i, i, i, i, i, ctypes.c_double, i, vp, vp]
        L.osbf_filter_gauss.restype = st
        L.osbf_filter_host.argtypes = [vp, vp, vp, i, i, i, i, i, i, i, vp]
        L.osbf_filter_host.restype = st
        L.osbf_filter_backward.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, vp]
        L.osbf_filter_backward.restype = st
        L.osbf_filter_checkpointed.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, i, vp]
        L.osbf_filter_checkpointed.restype = st
        L.osbf_filter_backward_checkpointed.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, i, vp]
        L.osbf_filter_backward_checkpointed.restype = st
        L.osbf_filter_batched.argtypes = [vp, ctypes.POINTER(_Job), i, vp]
        L.osbf_filter_batched.restype = st
        L.osbf_autotune.argtypes = [vp, i, i, i, i, i, i]
        L.osbf_autotune.restype = st
        L.osbf_tuned.argtypes = [vp, i, i, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.osbf_tuned.restype = st
        L.osbf_set_tuned.argtypes = [vp, i, i, i, i, i, i, i]
        L.osbf_set_tuned.restype = st
        L.osbf_autotune_batched.argtypes = [vp, ctypes.POINTER(_Job), i, vp]
        L.osbf_autotune_batched.restype = st
        L.osbf_batched_policy.argtypes = [vp, ctypes.POINTER(_Job), i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.osbf_batched_policy.restype = i
        L.osbf_frame_pitch.argtypes = [i, i]
        L.osbf_frame_pitch.restype = i
        L.osbf_maps_pitch.argtypes = [i, i]
        L.osbf_maps_pitch.restype = i
        L.osbf_check.argtypes = [vp]
        L.osbf_check.restype = st
        L.osbf_batched_latencies.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong), i]
        L.osbf_batched_latencies.restype = i
        L.osbf_set_wait_timeout.argtypes = [vp, ctypes.c_ulonglong]
        L.osbf_set_wait_timeout.restype = st
        _lib = L
    return _lib


def _destroy_all():
    if _lib is None:
        return
    for c in list(_ctxs.values()):
        _lib.osbf_destroy(c)
    _ctxs.clear()


atexit.register(_destroy_all)


def context(device: int) -> ctypes.c_void_p:
    """The library context of a CUDA device (created on first use, kept until exit)."""
    with _lock:
        c = _ctxs.get(device)
        if c is None:
            c = ctypes.c_void_p()
            st = lib().osbf_create(ctypes.byref(c), device)
            if st != 0:
                raise OSBFError(st, f"osbf_create(device={device}) failed")
            _ctxs[device] = c
        return c


def _check(st: int, ctx: ctypes.c_void_p):
    if st != 0:
        msg = lib().osbf_last_error(ctx)
        raise OSBFError(st, msg.decode() if msg else "")


def _stream(device: int) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _nchw(x: torch.Tensor):
    if x.dim() == 2:
        return 1, 1, x.shape[0], x.shape[1]
    if x.dim() == 3:
        return 1, x.shape[0], x.shape[1], x.shape[2]
    if x.dim() == 4:
        return tuple(x.shape)
    raise ValueError("expected an H x W, P x H x W or N x C x H x W tensor")


def _require_cuda(*ts: torch.Tensor):
    for t in ts:
        if not t.is_cuda:
            raise ValueError("the library works on CUDA tensors only (use filter_host for host buffers)")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def version() -> str:
    return lib().osbf_version().decode()


def last_launch_count(device: int = 0) -> int:
    """Kernel launches enqueued by the last filter call on this device's context."""
    return lib().osbf_last_launch_count(context(device))


def maps_pitch(W: int, r: int) -> int:
    """Bytes per selection-map row: W + 2r rounded up to a multiple of 16."""
    return lib().osbf_maps_pitch(W, r)


def maps_shape(x: torch.Tensor, r: int, iters: int):
    """Shape of the selection maps of osbf_filter_ex: (iters, N*C, H+2r, maps_pitch(W, r));
    the first W+2r bytes of each row hold the window indices (maps_frames() views them)."""
    N, C, H, W = _nchw(x)
    return (iters, N * C, H + 2 * r, maps_pitch(W, r))


def maps_frames(maps, W: int, r: int):
    """The frame columns of selection maps (a view without the row padding)."""
    return maps[..., : W + 2 * r]


def filter(x: torch.Tensor, r: int, iters: int, *, depth: int = 0, tie: str = "paper",
           maps: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
           variant: str = "auto") -> torch.Tensor:
    """Forward One-Sided Box Filter (osbf_filter_ex).  uint8 input gives float32 output.
    variant: the float32 single-pass kernel ("auto", "tile" or "strip")."""
    _require_cuda(x)
    N, C, H, W = _nchw(x)
    if x.dtype not in _DTYPE:
        raise TypeError(f"unsupported dtype {x.dtype}")
    odt = torch.float32 if x.dtype == torch.uint8 else x.dtype
    if out is None:
        out = torch.empty(x.shape, dtype=odt, device=x.device)
    _require_cuda(out)
    if out.dtype != odt or out.shape != x.shape:
        raise ValueError("out has the wrong dtype or shape")
    opts = _Options(depth, _TIE[tie], None, _VARIANT[variant], (ctypes.c_int * 3)())
    if maps is not None:
        _require_cuda(maps)
        if maps.dtype != torch.uint8 or tuple(maps.shape) != maps_shape(x, r, iters):
            raise ValueError(f"maps must be uint8 of shape {maps_shape(x, r, iters)}")
        opts.maps = maps.data_ptr()
    dev = x.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_ex(ctx, x.data_ptr(), out.data_ptr(), N, C, H, W, r, iters, _DTYPE[x.dtype],
                                ctypes.byref(opts), _stream(dev)), ctx)
    return out


def filter_fast(x: torch.Tensor, r: int, iters: int, *, maps: Optional[torch.Tensor] = None,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """The fast approximation (osbf_filter_fast; Algorithm 3, Eq. (app)) on float32 NCHW input."""
    _require_cuda(x)
    N, C, H, W = _nchw(x)
    if x.dtype != torch.float32:
        raise TypeError("filter_fast takes float32")
    if out is None:
        out = torch.empty_like(x)
    _require_cuda(out)
    if out.dtype != torch.float32 or out.shape != x.shape:
        raise ValueError("out has the wrong dtype or shape")
    mp = None
    if maps is not None:
        _require_cuda(maps)
        if maps.dtype != torch.uint8 or tuple(maps.shape) != maps_shape(x, r, iters):
            raise ValueError(f"maps must be uint8 of shape {maps_shape(x, r, iters)}")
        mp = maps.data_ptr()
    dev = x.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_fast(ctx, x.data_ptr(), out.data_ptr(), N, C, H, W, r, iters, mp, _stream(dev)), ctx)
    return out


def filter_gauss(x: torch.Tensor, r: int, sigma: float, iters: int, *, maps: Optional[torch.Tensor] = None,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """The one-sided Gaussian filter (osbf_filter_gauss; Algorithm 1 with the one-sided
    Gaussian kernels of Sec. "Separable Kernels") on float32 NCHW input."""
    _require_cuda(x)
    N, C, H, W = _nchw(x)
    if x.dtype != torch.float32:
        raise TypeError("filter_gauss takes float32")
    if out is None:
        out = torch.empty_like(x)
    _require_cuda(out)
    if out.dtype != torch.float32 or out.shape != x.shape:
        raise ValueError("out has the wrong dtype or shape")
    mp = None
    if maps is not None:
        _require_cuda(maps)
        if maps.dtype != torch.uint8 or tuple(maps.shape) != maps_shape(x, r, iters):
            raise ValueError(f"maps must be uint8 of shape {maps_shape(x, r, iters)}")
        mp = maps.data_ptr()
    dev = x.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_gauss(ctx, x.data_ptr(), out.data_ptr(), N, C, H, W, r, float(sigma), iters, mp,
                                   _stream(dev)), ctx)
    return out


def maps3d_shape(x: torch.Tensor, r: int, iters: int):
    """Shape of the 3D filter's selection maps: (iters, N*C, D+2r, H+2r, W+2r)."""
    N, C, D, H, W = x.shape
    return (iters, N * C, D + 2 * r, H + 2 * r, W + 2 * r)


def filter3d(x: torch.Tensor, r: int, iters: int, *, maps: Optional[torch.Tensor] = None,
             out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """The 3D filter (osbf_filter_3d; Sec. "Higher Dimension Case") on float32 N x C x D x H x W."""
    _require_cuda(x)
    if x.dim() != 5 or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("filter3d takes a contiguous float32 N x C x D x H x W tensor")
    N, C, D, H, W = x.shape
    if out is None:
        out = torch.empty_like(x)
    _require_cuda(out)
    if out.dtype != torch.float32 or out.shape != x.shape:
        raise ValueError("out has the wrong dtype or shape")
    mp = None
    if maps is not None:
        _require_cuda(maps)
        if maps.dtype != torch.uint8 or tuple(maps.shape) != maps3d_shape(x, r, iters):
            raise ValueError(f"maps must be uint8 of shape {maps3d_shape(x, r, iters)}")
        mp = maps.data_ptr()
    dev = x.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_3d(ctx, x.data_ptr(), out.data_ptr(), N, C, D, H, W, r, iters, mp, _stream(dev)), ctx)
    return out


def filter_host(x: torch.Tensor, r: int, iters: int, *, out: Optional[torch.Tensor] = None,
                device: int = 0) -> torch.Tensor:
    """osbf_filter_host: host (ideally pinned) input and output; returns once `out` is filled."""
    if x.is_cuda or not x.is_contiguous():
        raise ValueError("filter_host takes a contiguous host tensor")
    N, C, H, W = _nchw(x)
    odt = torch.float32 if x.dtype == torch.uint8 else x.dtype
    if out is None:
        out = torch.empty(x.shape, dtype=odt, pin_memory=x.is_pinned())
    ctx = context(device)
    with torch.cuda.device(device):
        _check(lib().osbf_filter_host(ctx, x.data_ptr(), out.data_ptr(), N, C, H, W, r, iters, _DTYPE[x.dtype],
                                      _stream(device)), ctx)
    return out


def backward(grad_out: torch.Tensor, maps: torch.Tensor, r: int, iters: int,
             out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """osbf_filter_backward: vector-Jacobian product with the selections frozen to `maps`."""
    _require_cuda(grad_out, maps)
    if grad_out.dtype != torch.float32:
        raise TypeError("grad_out must be float32")
    N, C, H, W = _nchw(grad_out)
    if maps.dtype != torch.uint8 or tuple(maps.shape) != maps_shape(grad_out, r, iters):
        raise ValueError(f"maps must be uint8 of shape {maps_shape(grad_out, r, iters)}")
    if out is None:
        out = torch.empty_like(grad_out)
    dev = grad_out.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_backward(ctx, grad_out.data_ptr(), out.data_ptr(), maps.data_ptr(), N, C, H, W, r,
                                      iters, _stream(dev)), ctx)
    return out


def checkpoint_count(iters: int, interval: int) -> int:
    return (iters + interval - 1) // interval


def frame_pitch(W: int, r: int) -> int:
    return lib().osbf_frame_pitch(W, r)


def check(device: int = 0) -> None:
    """osbf_check: raise if a bounded device-side wait of this context gave up."""
    ctx = context(device)
    _check(lib().osbf_check(ctx), ctx)


def filter_checkpointed(x: torch.Tensor, r: int, iters: int, interval: int):
    """Forward that keeps a padded frame every `interval` passes; returns (out, checkpoints).

    checkpoints: K x N*C x (H+2r) x frame_pitch(W, r) float32 (the valid width is W + 2r)."""
    _require_cuda(x)
    N, C, H, W = _nchw(x)
    ck = torch.empty((checkpoint_count(iters, interval), N * C, H + 2 * r, frame_pitch(W, r)),
                     dtype=torch.float32, device=x.device)
    out = torch.empty_like(x)
    dev = x.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_checkpointed(ctx, x.data_ptr(), out.data_ptr(), ck.data_ptr(), interval, N, C, H, W, r,
                                          iters, _stream(dev)), ctx)
    return out, ck


def backward_checkpointed(grad_out: torch.Tensor, checkpoints: torch.Tensor, r: int, iters: int,
                          interval: int) -> torch.Tensor:
    _require_cuda(grad_out, checkpoints)
    N, C, H, W = _nchw(grad_out)
    out = torch.empty_like(grad_out)
    dev = grad_out.device.index
    ctx = context(dev)
    _check(lib().osbf_filter_backward_checkpointed(ctx, grad_out.data_ptr(), out.data_ptr(), checkpoints.data_ptr(),
                                                   interval, N, C, H, W, r, iters, _stream(dev)), ctx)
    return out


def _jobs(inputs, radii, iters, outputs):
    n = len(inputs)
    jobs = (_Job * n)()
    dev = None
    for k, (t, o, r, it) in enumerate(zip(inputs, outputs, radii, iters)):
        _require_cuda(t, o)
        if t.dim() != 2 or t.dtype != torch.float32 or o.shape != t.shape or o.dtype != t.dtype:
            raise ValueError("batched jobs are H x W float32 images")
        dev = t.device.index if dev is None else dev
        jobs[k] = _Job(t.data_ptr(), o.data_ptr(), t.shape[0], t.shape[1], int(r), int(it))
    return jobs, n, 0 if dev is None else dev


def batched(inputs: Sequence[torch.Tensor], radii: Sequence[int], iters: Sequence[int],
            outputs: Optional[Sequence[torch.Tensor]] = None) -> list:
    """osbf_filter_batched: many H x W float32 images of different sizes, radii and pass counts."""
    if outputs is None:
        outputs = [torch.empty_like(t) for t in inputs]
    jobs, n, dev = _jobs(inputs, radii, iters, outputs)
    ctx = context(dev)
    _check(lib().osbf_filter_batched(ctx, jobs, n, _stream(dev)), ctx)
    return list(outputs)


def autotune_batched(inputs: Sequence[torch.Tensor], radii: Sequence[int], iters: Sequence[int],
                     outputs: Sequence[torch.Tensor]) -> None:
    """osbf_autotune_batched: time the batch's layout policies, record the fastest for these jobs."""
    jobs, n, dev = _jobs(inputs, radii, iters, outputs)
    ctx = context(dev)
    _check(lib().osbf_autotune_batched(ctx, jobs, n, _stream(dev)), ctx)


def batched_policy(inputs: Sequence[torch.Tensor], radii: Sequence[int], iters: Sequence[int],
                   outputs: Sequence[torch.Tensor]):
    """The tuned policy of these jobs as (order, ctas_per_sm), or None if none is recorded."""
    jobs, n, dev = _jobs(inputs, radii, iters, outputs)
    o, c = ctypes.c_int(), ctypes.c_int()
    found = lib().osbf_batched_policy(context(dev), jobs, n, ctypes.byref(o), ctypes.byref(c))
    return (o.value, c.value) if found else None


def set_tuned(dtype: torch.dtype, planes: int, H: int, W: int, r: int, depth: int, variant: str,
              device: int = 0) -> None:
    """osbf_set_tuned: record a forward choice (depth, "tile" or "strip") without timing."""
    ctx = context(device)
    _check(lib().osbf_set_tuned(ctx, _DTYPE[dtype], planes, H, W, r, depth, _VARIANT[variant]), ctx)


def set_wait_timeout(ns: int, device: int = 0) -> None:
    """Bound of the batched launch's device-side dependency wait (0 = default 2 s)."""
    ctx = context(device)
    _check(lib().osbf_set_wait_timeout(ctx, int(ns)), ctx)


def batched_latencies(n: int, device: int = 0) -> list:
    """Per-image latencies (seconds) of the last batched call's persistent launch."""
    buf = (ctypes.c_ulonglong * max(n, 1))()
    k = lib().osbf_batched_latencies(context(device), buf, n)
    return [buf[i] * 1e-9 for i in range(k)]


def autotune(dtype: torch.dtype, planes: int, H: int, W: int, r: int, iters: int, device: int = 0) -> None:
    """osbf_autotune: time the forward's candidates (tile kernel at each fused depth, strip
    kernel) on a synthetic image and record the fastest for (dtype, r, size class)."""
    ctx = context(device)
    with torch.cuda.device(device):
        _check(lib().osbf_autotune(ctx, _DTYPE[dtype], planes, H, W, r, iters), ctx)


def tuned(dtype: torch.dtype, planes: int, H: int, W: int, r: int, device: int = 0):
    """The recorded tuned choice as (depth, variant name), or (0, "auto") if none."""
    d, v = ctypes.c_int(), ctypes.c_int()
    ctx = context(device)
    _check(lib().osbf_tuned(ctx, _DTYPE[dtype], planes, H, W, r, ctypes.byref(d), ctypes.byref(v)), ctx)
    return d.value, {0: "auto", 1: "tile", 2: "strip"}[v.value]


class OSBFFunction(torch.autograd.Function):
    """Autograd wrapper: forward keeps every pass's selection map (1 byte per frame
    pixel and pass) or, with `checkpoint_interval`, a frame every that many passes;
    backward is the library's adjoint kernel (selection treated as constant)."""

    @staticmethod
    def forward(ctx, x, r: int, iters: int, checkpoint_interval: int = 0):
        if checkpoint_interval and checkpoint_interval > 0:
            out, ck = filter_checkpointed(x.contiguous(), r, iters, checkpoint_interval)
            ctx.save_for_backward(ck)
            ctx.mode = "checkpoint"
        else:
            maps = torch.empty(maps_shape(x, r, iters), dtype=torch.uint8, device=x.device)
            out = filter(x.contiguous(), r, iters, maps=maps)
            ctx.save_for_backward(maps)
            ctx.mode = "maps"
        ctx.r, ctx.iters, ctx.interval = r, iters, checkpoint_interval
        return out

    @staticmethod
    def backward(ctx, g):
        (saved,) = ctx.saved_tensors
        g = g.contiguous()
        if ctx.mode == "maps":
            gi = backward(g, saved, ctx.r, ctx.iters)
        else:
            gi = backward_checkpointed(g, saved, ctx.r, ctx.iters, ctx.interval)
        return gi, None, None, None


def osbf(x: torch.Tensor, r: int, iters: int, checkpoint_interval: int = 0) -> torch.Tensor:
    """Differentiable One-Sided Box Filter on float32 CUDA tensors."""
    return OSBFFunction.apply(x, r, iters, checkpoint_interval)
