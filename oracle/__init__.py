"""CPU oracle for the One-Sided Box Filter -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 (int64 for 8-bit input) implementation of Algorithm 2 with
the appendix's boundary rule, by direct summation over each one-sided window
(Eq. (6)-(13)), of the fast approximation (Algorithm 3, Eq. (app)), of the 3D
filter (Sec. "Higher Dimension Case"), and of the one-sided Gaussian filter
(Algorithm 1 with the kernels of Sec. "Separable Kernels").  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it; the CUDA library never imports it and shares no
code with it.  The arithmetic lives in ``osbf_oracle.c``; this module only
builds that file with gcc and marshals numpy arrays into it.

Parity pins live in ``tests/test_oracle_pins.py``.  Every oracle function is
pinned there except the storage-rounding helper's bf16 subnormal range, which
no workload reaches.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osbf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

STORE = {None: 0, "none": 0, "f32": 1, "f16": 2, "bf16": 3}
TIE = {"paper": 0, "appendix": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math).  Returns the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, ll, vp = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
        lib.oracle_round_storage.restype = d
        lib.oracle_round_storage.argtypes = [d, i]
        lib.oracle_round_storage_array.argtypes = [vp, ctypes.c_long, i]
        lib.oracle_threads.restype = i
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_pad_replicate_f64.argtypes = [vp, vp, i, i, i, i]
        lib.oracle_crop_f64.argtypes = [vp, vp, i, i, i, i]
        lib.oracle_window_means_f64.argtypes = [vp, vp, i, i, i, i]
        lib.oracle_iterate_frame_f64.restype = i
        lib.oracle_iterate_frame_f64.argtypes = [vp, i, i, i, i, i, i, vp, vp, vp, d, vp, i]
        lib.oracle_filter_f64.restype = i
        lib.oracle_filter_f64.argtypes = [vp, vp, i, i, i, i, i, i, vp, vp, vp, d, vp, i]
        lib.oracle_fast_filter_f64.restype = i
        lib.oracle_fast_filter_f64.argtypes = [vp, vp, i, i, i, i, i, i, vp, vp, vp, d, vp]
        lib.oracle_filter3d_f64.restype = i
        lib.oracle_filter3d_f64.argtypes = [vp, vp, i, i, i, i, i, i, vp, vp, d, vp]
        lib.oracle_gauss_filter_f64.restype = i
        lib.oracle_gauss_filter_f64.argtypes = [vp, vp, i, i, i, i, i, i, d, vp, vp, d, vp]
        lib.oracle_gauss_iterate_frame_f64.restype = i
        lib.oracle_gauss_iterate_frame_f64.argtypes = [vp, i, i, i, i, i, i, d, vp, vp, d, vp]
        lib.oracle_filter_region_f64.restype = i
        lib.oracle_filter_region_f64.argtypes = [vp, i, i, i, i, i, i, i, i, i, vp, vp, i, d, vp]
        lib.oracle_u8_first_pass.restype = i
        lib.oracle_u8_first_pass.argtypes = [vp, vp, vp, i, i, i, i, i]
        lib.oracle_adjoint_f64.restype = i
        lib.oracle_adjoint_f64.argtypes = [vp, vp, vp, i, i, i, i, i]
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _planes(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x)
    if x.ndim == 2:
        return x[None]
    if x.ndim == 3:
        return x
    if x.ndim == 4:
        return x.reshape(-1, x.shape[-2], x.shape[-1])
    raise ValueError("expected H x W, P x H x W or N x C x H x W")


def _check(st: int):
    if st != 0:
        raise RuntimeError(f"oracle error {st}")


def threads() -> int:
    return _load().oracle_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def round_storage(x: np.ndarray, storage: str) -> np.ndarray:
    """Round FP64 values to f32 / f16 / bf16 (nearest, ties to even); returns FP64."""
    a = np.ascontiguousarray(x, dtype=np.float64).copy()
    _load().oracle_round_storage_array(_ptr(a), a.size, STORE[storage])
    return a


def pad_replicate(x: np.ndarray, r: int) -> np.ndarray:
    x3 = np.ascontiguousarray(_planes(x), dtype=np.float64)
    P, H, W = x3.shape
    f = np.empty((P, H + 2 * r, W + 2 * r), dtype=np.float64)
    _load().oracle_pad_replicate_f64(_ptr(x3), _ptr(f), P, H, W, r)
    return f


def window_means(frame: np.ndarray, r: int) -> np.ndarray:
    """The eight window means (N1..N8) at every frame pixel: shape 8 x P x FH x FW."""
    f = np.ascontiguousarray(_planes(frame), dtype=np.float64)
    P, FH, FW = f.shape
    out = np.empty((8, P, FH, FW), dtype=np.float64)
    _load().oracle_window_means_f64(_ptr(f), _ptr(out), P, FH, FW, r)
    return out


def iterate_frame(frame: np.ndarray, r: int, iters: int, tie: str = "paper", want_maps: bool = False,
                  want_gaps: bool = False, hint: Optional[np.ndarray] = None, hint_thresh: float = 1e-6,
                  storage: Optional[str] = None):
    """Run `iters` passes on padded frames (P x FH x FW).  Returns a dict."""
    f = np.ascontiguousarray(_planes(frame), dtype=np.float64).copy()
    P, FH, FW = f.shape
    maps = np.zeros((iters, P, FH, FW), dtype=np.uint8) if (want_maps or hint is not None) else None
    gaps = np.zeros((iters, P, FH, FW), dtype=np.float64) if want_gaps else None
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, P, FH, FW)
    nh = ctypes.c_longlong(0)
    _check(_load().oracle_iterate_frame_f64(_ptr(f), P, FH, FW, r, iters, TIE[tie], _ptr(maps), _ptr(gaps),
                                            _ptr(h), float(hint_thresh), ctypes.addressof(nh), STORE[storage]))
    return {"frame": f, "maps": maps, "gaps": gaps, "n_hinted": int(nh.value)}


def filter(x: np.ndarray, r: int, iters: int, tie: str = "paper", want_maps: bool = False,
           want_gaps: bool = False, hint: Optional[np.ndarray] = None, hint_thresh: float = 1e-6,
           storage: Optional[str] = None):
    """The whole filter (pad, `iters` passes, crop) on H x W, P x H x W or N x C x H x W input.

    Returns a dict with "out" (same shape as x, FP64), "maps" / "gaps"
    (iters x P x FH x FW, when asked for) and "n_hinted".
    """
    shape = np.asarray(x).shape
    x3 = np.ascontiguousarray(_planes(x), dtype=np.float64)
    P, H, W = x3.shape
    FH, FW = H + 2 * r, W + 2 * r
    out = np.empty_like(x3)
    maps = np.zeros((iters, P, FH, FW), dtype=np.uint8) if (want_maps or hint is not None) else None
    gaps = np.zeros((iters, P, FH, FW), dtype=np.float64) if want_gaps else None
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, P, FH, FW)
    nh = ctypes.c_longlong(0)
    _check(_load().oracle_filter_f64(_ptr(x3), _ptr(out), P, H, W, r, iters, TIE[tie], _ptr(maps), _ptr(gaps),
                                     _ptr(h), float(hint_thresh), ctypes.addressof(nh), STORE[storage]))
    return {"out": out.reshape(shape), "maps": maps, "gaps": gaps, "n_hinted": int(nh.value)}


def fast_filter(x: np.ndarray, r: int, iters: int, tie: str = "paper", want_maps: bool = False,
                want_gaps: bool = False, hint: Optional[np.ndarray] = None, hint_thresh: float = 1e-6):
    """The fast approximation (Algorithm 3, Eq. (app)): pad, `iters` passes, crop.

    Same shapes and return dict as filter(); FP64, no storage rounding.
    """
    shape = np.asarray(x).shape
    x3 = np.ascontiguousarray(_planes(x), dtype=np.float64)
    P, H, W = x3.shape
    FH, FW = H + 2 * r, W + 2 * r
    out = np.empty_like(x3)
    maps = np.zeros((iters, P, FH, FW), dtype=np.uint8) if (want_maps or hint is not None) else None
    gaps = np.zeros((iters, P, FH, FW), dtype=np.float64) if want_gaps else None
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, P, FH, FW)
    nh = ctypes.c_longlong(0)
    _check(_load().oracle_fast_filter_f64(_ptr(x3), _ptr(out), P, H, W, r, iters, TIE[tie], _ptr(maps), _ptr(gaps),
                                          _ptr(h), float(hint_thresh), ctypes.addressof(nh)))
    return {"out": out.reshape(shape), "maps": maps, "gaps": gaps, "n_hinted": int(nh.value)}


def filter3d(x: np.ndarray, r: int, iters: int, want_maps: bool = False, hint: Optional[np.ndarray] = None,
             hint_thresh: float = 1e-6):
    """The 3D filter (Sec. "Higher Dimension Case") on D x H x W, P x D x H x W or
    N x C x D x H x W input: pad every axis by r, `iters` passes over 14 windows, crop.
    Returns {"out", "maps" (iters x P x FD x FH x FW, window 1..14), "n_hinted"}."""
    a = np.asarray(x)
    shape = a.shape
    x4 = np.ascontiguousarray(a.reshape((-1,) + shape[-3:]), dtype=np.float64)
    P, D, H, W = x4.shape
    FD, FH, FW = D + 2 * r, H + 2 * r, W + 2 * r
    out = np.empty_like(x4)
    maps = np.zeros((iters, P, FD, FH, FW), dtype=np.uint8) if (want_maps or hint is not None) else None
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, P, FD, FH, FW)
    nh = ctypes.c_longlong(0)
    _check(_load().oracle_filter3d_f64(_ptr(x4), _ptr(out), P, D, H, W, r, iters, _ptr(maps), _ptr(h),
                                       float(hint_thresh), ctypes.addressof(nh)))
    return {"out": out.reshape(shape), "maps": maps, "n_hinted": int(nh.value)}


def gauss_filter(x: np.ndarray, r: int, iters: int, sigma: float, tie: str = "paper", want_maps: bool = False,
                 hint: Optional[np.ndarray] = None, hint_thresh: float = 1e-6):
    """The one-sided Gaussian filter (Algorithm 1, Phi = weighted mean with the kernels of
    Sec. "Separable Kernels"): pad, `iters` passes, crop.  Same shapes and dict as filter()."""
    shape = np.asarray(x).shape
    x3 = np.ascontiguousarray(_planes(x), dtype=np.float64)
    P, H, W = x3.shape
    FH, FW = H + 2 * r, W + 2 * r
    out = np.empty_like(x3)
    maps = np.zeros((iters, P, FH, FW), dtype=np.uint8) if (want_maps or hint is not None) else None
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, P, FH, FW)
    nh = ctypes.c_longlong(0)
    _check(_load().oracle_gauss_filter_f64(_ptr(x3), _ptr(out), P, H, W, r, iters, TIE[tie], float(sigma), _ptr(maps),
                                           _ptr(h), float(hint_thresh), ctypes.addressof(nh)))
    return {"out": out.reshape(shape), "maps": maps, "n_hinted": int(nh.value)}


def gauss_iterate_frame(frame: np.ndarray, r: int, iters: int, sigma: float, tie: str = "paper",
                        hint: Optional[np.ndarray] = None, hint_thresh: float = 1e-6) -> np.ndarray:
    """`iters` one-sided Gaussian passes on already padded frames (P x FH x FW), zeros
    outside them; no padding or crop.  A (2r+1)^2 patch of a frame, zero where it leaves
    the frame, gives one pass's value at its centre pixel.  hint: iters x P x FH x FW
    window indices adopted at near ties (0 = none), as in filter()."""
    f = np.ascontiguousarray(_planes(frame), dtype=np.float64).copy()
    P, FH, FW = f.shape
    h = None if hint is None else np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, P, FH, FW)
    _check(_load().oracle_gauss_iterate_frame_f64(_ptr(f), P, FH, FW, r, iters, TIE[tie], float(sigma), None, _ptr(h),
                                                  float(hint_thresh), None))
    return f.reshape(np.asarray(frame).shape)


def filter_region(plane: np.ndarray, r: int, iters: int, y0: int, y1: int, x0: int, x1: int,
                  tie: str = "paper", hint: Optional[np.ndarray] = None, hint_thresh: float = 1e-6,
                  return_hinted: bool = False):
    """Exact output of one H x W plane on [y0, y1) x [x0, x1), from the dependency cone only.

    `hint`: optional selection maps of this plane's whole frame, iters x (H+2r) x (W+2r)
    (any array supporting the buffer protocol, e.g. a numpy memmap or array).
    """
    p = np.ascontiguousarray(plane, dtype=np.float64)
    H, W = p.shape
    out = np.empty((y1 - y0, x1 - x0), dtype=np.float64)
    h = None
    if hint is not None:
        h = np.ascontiguousarray(hint, dtype=np.uint8).reshape(iters, H + 2 * r, W + 2 * r)
    nh = ctypes.c_longlong(0)
    _check(_load().oracle_filter_region_f64(_ptr(p), H, W, r, iters, TIE[tie], y0, y1, x0, x1, _ptr(out), _ptr(h),
                                            W + 2 * r, float(hint_thresh), ctypes.addressof(nh)))
    return (out, int(nh.value)) if return_hinted else out


def u8_first_pass(x: np.ndarray, r: int, tie: str = "paper"):
    """Exact integer first pass on 8-bit input.  Returns (frame float32 P x FH x FW, map uint8)."""
    x3 = np.ascontiguousarray(_planes(x), dtype=np.uint8)
    P, H, W = x3.shape
    FH, FW = H + 2 * r, W + 2 * r
    frame = np.empty((P, FH, FW), dtype=np.float32)
    m = np.empty((P, FH, FW), dtype=np.uint8)
    _check(_load().oracle_u8_first_pass(_ptr(x3), _ptr(frame), _ptr(m), P, H, W, r, TIE[tie]))
    return frame, m


def crop(frame: np.ndarray, r: int) -> np.ndarray:
    f = _planes(frame)
    FH, FW = f.shape[-2:]
    return f[:, r:FH - r, r:FW - r]


def adjoint(grad_out: np.ndarray, maps: np.ndarray, r: int, iters: int) -> np.ndarray:
    """Transpose of the filter with selections frozen to `maps` (iters x P x FH x FW)."""
    shape = np.asarray(grad_out).shape
    g3 = np.ascontiguousarray(_planes(grad_out), dtype=np.float64)
    P, H, W = g3.shape
    m = np.ascontiguousarray(maps, dtype=np.uint8).reshape(iters, P, H + 2 * r, W + 2 * r)
    gi = np.empty_like(g3)
    _check(_load().oracle_adjoint_f64(_ptr(g3), _ptr(m), _ptr(gi), P, H, W, r, iters))
    return gi.reshape(shape)
