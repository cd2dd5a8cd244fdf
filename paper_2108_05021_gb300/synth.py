"""Seeded synthetic inputs shaped like the One-Sided Box Filter paper's workloads.

The paper smooths natural photographs, a checkerboard and an MRI volume
(Sec. "Edge and Corner Preserving", Sec. "Comparison with Edge Preserving
Methods"); none of those images ships with it, so every run here draws a
piecewise-constant scene plus noise instead:

* a 0.5 background;
* ``n_rect`` axis-aligned rectangles, each given by two sorted uniform draws per
  axis (a pixel belongs to it when its centre lies in the half-open box);
* ``n_tri`` triangles with three uniform vertices (a pixel belongs to it when its
  centre lies inside, i.e. all three edge functions are >= 0 once the triangle is
  oriented counter-clockwise);
* painting order: rectangles, then triangles; later shapes overwrite earlier
  ones; every region takes a level drawn uniformly from [0, 1];
* i.i.d. N(0, sigma^2) noise, then clamping to [0, 1].

Every channel of an N x C stack is drawn independently from one PCG64 stream.
This module holds none of the filter's arithmetic: it only produces inputs, and
both the CUDA path's tests and the CPU oracle's tests receive the same arrays.
"""
from __future__ import annotations

import numpy as np

__all__ = ["piecewise_plane", "piecewise_stack", "to_u8", "checkerboard", "round_to_storage"]


def _paint_plane(rng: np.random.Generator, H: int, W: int, n_rect: int, n_tri: int) -> np.ndarray:
    img = np.full((H, W), 0.5, dtype=np.float32)
    for _ in range(n_rect):
        y0, y1 = np.sort(rng.uniform(0.0, H, size=2))
        x0, x1 = np.sort(rng.uniform(0.0, W, size=2))
        level = np.float32(rng.uniform(0.0, 1.0))
        # pixel centres c = i + 0.5 with y0 <= c < y1
        r0, r1 = int(np.ceil(y0 - 0.5)), int(np.ceil(y1 - 0.5))
        c0, c1 = int(np.ceil(x0 - 0.5)), int(np.ceil(x1 - 0.5))
        img[max(r0, 0):min(r1, H), max(c0, 0):min(c1, W)] = level
    for _ in range(n_tri):
        vx = rng.uniform(0.0, W, size=3)
        vy = rng.uniform(0.0, H, size=3)
        level = np.float32(rng.uniform(0.0, 1.0))
        # orient counter-clockwise in (x, y) with the usual cross product sign
        cross = (vx[1] - vx[0]) * (vy[2] - vy[0]) - (vy[1] - vy[0]) * (vx[2] - vx[0])
        if cross < 0:
            vx[[1, 2]] = vx[[2, 1]]
            vy[[1, 2]] = vy[[2, 1]]
        r0 = max(int(np.floor(vy.min() - 0.5)), 0)
        r1 = min(int(np.ceil(vy.max() + 0.5)), H)
        c0 = max(int(np.floor(vx.min() - 0.5)), 0)
        c1 = min(int(np.ceil(vx.max() + 0.5)), W)
        if r0 >= r1 or c0 >= c1:
            continue
        cy = (np.arange(r0, r1, dtype=np.float64) + 0.5)[:, None]
        cx = (np.arange(c0, c1, dtype=np.float64) + 0.5)[None, :]
        inside = np.ones((r1 - r0, c1 - c0), dtype=bool)
        for k in range(3):
            ax, ay = vx[k], vy[k]
            bx, by = vx[(k + 1) % 3], vy[(k + 1) % 3]
            inside &= ((bx - ax) * (cy - ay) - (by - ay) * (cx - ax)) >= 0.0
        img[r0:r1, c0:c1][inside] = level
    return img


def piecewise_plane(H: int, W: int, seed: int, sigma: float = 0.05,
                    n_rect: int = 40, n_tri: int = 20) -> np.ndarray:
    """One H x W float32 plane in [0, 1] (see the module docstring)."""
    return piecewise_stack(1, 1, H, W, seed, sigma, n_rect, n_tri)[0, 0]


def piecewise_stack(N: int, C: int, H: int, W: int, seed: int, sigma: float = 0.05,
                    n_rect: int = 40, n_tri: int = 20) -> np.ndarray:
    """An N x C x H x W float32 stack; each plane drawn independently, in order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((N, C, H, W), dtype=np.float32)
    for n in range(N):
        for c in range(C):
            img = _paint_plane(rng, H, W, n_rect, n_tri)
            if sigma > 0:
                img += np.float32(sigma) * rng.standard_normal((H, W), dtype=np.float32)
            np.clip(img, 0.0, 1.0, out=img)
            out[n, c] = img
    return out


def to_u8(x: np.ndarray) -> np.ndarray:
    """The 8-bit copy round(255 x) of a [0, 1] image (ties to even, as numpy rounds)."""
    return np.rint(np.asarray(x, dtype=np.float64) * 255.0).clip(0, 255).astype(np.uint8)


def checkerboard(H: int, W: int, square: int, lo: float = 0.25, hi: float = 0.75,
                 phase_y: int = 0, phase_x: int = 0) -> np.ndarray:
    """A noise-free checkerboard of ``square`` x ``square`` cells (float32)."""
    yy = (np.arange(H)[:, None] + phase_y) // square
    xx = (np.arange(W)[None, :] + phase_x) // square
    return np.where((yy + xx) % 2 == 0, lo, hi).astype(np.float32)


def round_to_storage(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round float32 values to a 16-bit storage type and return them as float32.

    Used to build inputs that are exactly representable in f16 / bf16 storage.
    """
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    return t.to(tdt).to(torch.float32).numpy()
