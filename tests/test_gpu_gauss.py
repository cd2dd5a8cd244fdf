"""GPU parity of the one-sided Gaussian filter (osbf_filter_gauss; Algorithm 1 with the
one-sided Gaussian kernels of Sec. "Separable Kernels") against the oracle's gauss_filter.

Bar: with the GPU's selections as hints at near ties (best two |mean - U| within 1e-6
in FP64), every pixel within 1e-5 of the FP64 oracle after several passes (float32
weights and sums over at most (r+1)(2r+1) taps of values in [0, 1]); the map-writing and
the plain launches agree bit for bit.  At the 4096 x 4096 x 3, r = 8 size: sampled pixels
of one pass against the oracle on their own (2r+1)^2 patches, and the checkerboard
invariant after several passes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TIE_THRESH = 1e-6
TOL = 1e-5


def sigma_for(r):
    return 0.6 + 0.35 * r


def run(x_np, r, sigma, iters, want_maps=True):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    maps = torch.zeros(osbf.maps_shape(x, r, iters), dtype=torch.uint8, device=DEV) if want_maps else None
    out = osbf.filter_gauss(x, r, sigma, iters, maps=maps)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (osbf.maps_frames(maps, x.shape[-1], r).cpu().numpy() if want_maps else None)


def check(x_np, r, sigma, iters):
    out, maps = run(x_np, r, sigma, iters)
    ref = oracle.gauss_filter(x_np.astype(np.float64), r, iters, sigma, hint=maps, hint_thresh=TIE_THRESH)
    err = np.abs(out - ref["out"]).max()
    assert err <= TOL, (r, sigma, iters, err)
    plain, _ = run(x_np, r, sigma, iters, want_maps=False)
    np.testing.assert_array_equal(out, plain)
    return out, maps, ref


@pytest.mark.parametrize("r", list(range(1, 17)))
def test_gauss_matches_oracle(r):
    x = synth.piecewise_stack(1, 2, 45, 140, seed=r, sigma=0.05)   # two tiles across, ragged
    _, maps, ref = check(x, r, sigma_for(r), 3)
    # the selections agree wherever the oracle's choice is clear
    assert ref["n_hinted"] <= 1e-3 * maps.size


@pytest.mark.parametrize("sigma", [0.3, 1.0, 3.0, 1e4, float("inf")])
def test_gauss_sigmas(sigma):
    x = synth.piecewise_stack(1, 1, 60, 250, seed=11, sigma=0.05)
    check(x, 5, sigma, 3)


def test_gauss_infinite_sigma_is_the_box_filter():
    """sigma = +inf: flat weights, the one-sided box filter (against the box oracle)."""
    x = synth.piecewise_stack(1, 1, 50, 130, seed=3, sigma=0.05)
    for r in (2, 8):
        out, maps = run(x, r, float("inf"), 3)
        ref = oracle.filter(x.astype(np.float64), r, 3, hint=maps, hint_thresh=TIE_THRESH)
        assert np.abs(out - ref["out"]).max() <= TOL


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1, 1, 1, 9), (1, 1, 7, 1), (1, 2, 5, 6), (2, 1, 33, 129),
                                   (1, 1, 70, 256), (1, 3, 97, 230)])
def test_gauss_shapes(shape):
    x = synth.piecewise_stack(*shape, seed=7, sigma=0.05)
    for r in (1, 4, 9):
        check(x, r, sigma_for(r), 2)


def test_gauss_many_tiles():
    x = synth.piecewise_stack(1, 1, 300, 520, seed=21, sigma=0.05)
    check(x, 8, 3.0, 4)


def test_gauss_full_size_sampled_one_pass():
    """4096 x 4096 x 3, r = 8, sigma = 3: one pass in the benchmark's launch configuration;
    400 sampled pixels (edges and corners included) against the oracle on their patches."""
    r, sigma = 8, 3.0
    x_np = synth.piecewise_stack(1, 3, 4096, 4096, seed=5, sigma=0.05)
    x = torch.from_numpy(x_np).to(DEV)
    maps = torch.zeros(osbf.maps_shape(x, r, 1), dtype=torch.uint8, device=DEV)
    out = osbf.filter_gauss(x, r, sigma, 1, maps=maps)
    torch.cuda.synchronize()
    out_np = out.cpu().numpy()
    sel = osbf.maps_frames(maps, 4096, r).cpu().numpy()[0]
    rng = np.random.default_rng(0)
    pts = [(c, y, xx) for c in range(3) for y in (0, 1, 4095) for xx in (0, 7, 4095)]
    pts += [(int(rng.integers(3)), int(rng.integers(4096)), int(rng.integers(4096))) for _ in range(400 - len(pts))]
    err = 0.0
    for c, y, xx in pts:
        # frame rows / columns around frame pixel (y + r, x + r): the replicate-padded input
        # inside the frame, zeros outside it
        fy = np.arange(y - r, y + r + 1)
        fx = np.arange(xx - r, xx + r + 1)
        inside = ((fy >= -r) & (fy < 4096 + r))[:, None] & ((fx >= -r) & (fx < 4096 + r))[None, :]
        src = x_np[0, c][np.clip(fy, 0, 4095)][:, np.clip(fx, 0, 4095)].astype(np.float64)
        patch = np.where(inside, src, 0.0)
        s = sel[c, y + r, xx + r]
        assert 1 <= s <= 8
        hint = np.zeros((1, 1, 2 * r + 1, 2 * r + 1), dtype=np.uint8)
        hint[0, 0, r, r] = s
        want = oracle.gauss_iterate_frame(patch, r, 1, sigma, hint=hint, hint_thresh=TIE_THRESH)[r, r]
        err = max(err, abs(float(out_np[0, c, y, xx]) - want))
    assert err <= TOL, err


def test_gauss_full_size_checkerboard_invariant():
    """Corners and edges preserved at 4096 x 4096 x 3, r = 8, 10 passes: every pixel has a
    quadrant inside its own 16 x 16 cell, whose weighted mean is the pixel value."""
    r = 8
    cb = synth.checkerboard(4096, 4096, 2 * r)
    x = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(cb, (1, 3, 4096, 4096)))).to(DEV)
    out = osbf.filter_gauss(x, r, 3.0, 10)
    torch.cuda.synchronize()
    assert (out - x).abs().max().item() <= 1e-5


def test_gauss_trivial_and_status_codes():
    x = torch.from_numpy(synth.piecewise_stack(1, 1, 20, 24, seed=1, sigma=0.05)).to(DEV)
    for r, it in ((0, 3), (3, 0)):
        np.testing.assert_array_equal(osbf.filter_gauss(x, r, 1.0, it).cpu().numpy(), x.cpu().numpy())
    maps = torch.zeros(osbf.maps_shape(x, 0, 2), dtype=torch.uint8, device=DEV)
    osbf.filter_gauss(x, 0, 1.0, 2, maps=maps)
    assert bool((osbf.maps_frames(maps, 24, 0) == 1).all())
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter_gauss(x, 17, 3.0, 1)
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    for r, s in ((-1, 1.0), (2, 0.0), (2, -1.0), (2, float("nan"))):
        with pytest.raises(osbf.OSBFError) as e:
            osbf.filter_gauss(x, r, s, 1)
        assert e.value.status_name == "OSBF_EINVAL"
    with pytest.raises(TypeError):
        osbf.filter_gauss(x.half(), 2, 1.0, 1)
