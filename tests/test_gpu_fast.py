"""GPU parity of the fast approximation (osbf_filter_fast; Sec. "Fast Approximation to
One-sided Box Filter", Algorithm 3, Eq. (app)) against the oracle's fast_filter.

Same bar as the exact filter: with the GPU's selections as hints at near ties (best two
|d_i| within 1e-6), every pixel within 1e-5 of the FP64 oracle after several passes;
the map-writing and the plain launches agree bit for bit.
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


def run(x_np, r, iters, want_maps=True):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    maps = torch.zeros(osbf.maps_shape(x, r, iters), dtype=torch.uint8, device=DEV) if want_maps else None
    out = osbf.filter_fast(x, r, iters, maps=maps)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (osbf.maps_frames(maps, x.shape[-1], r).cpu().numpy() if want_maps else None)


def check(x_np, r, iters):
    out, maps = run(x_np, r, iters)
    ref = oracle.fast_filter(x_np.astype(np.float64), r, iters, hint=maps, hint_thresh=TIE_THRESH)
    err = np.abs(out - ref["out"]).max()
    assert err <= TOL, (r, iters, err)
    plain, _ = run(x_np, r, iters, want_maps=False)
    np.testing.assert_array_equal(out, plain)
    return out


@pytest.mark.parametrize("r", list(range(1, 17)))
def test_fast_matches_oracle(r):
    x = synth.piecewise_stack(1, 2, 45, 140, seed=r, sigma=0.05)
    check(x, r, 3)


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1, 1, 1, 9), (1, 1, 7, 1), (1, 2, 5, 6), (2, 1, 33, 129),
                                   (1, 1, 70, 256)])
def test_fast_shapes(shape):
    x = synth.piecewise_stack(*shape, seed=7, sigma=0.05)
    for r in (1, 4):
        check(x, r, 2)


def test_fast_output_paths():
    """W % 4 == 0 and r % 4 == 0: the last pass writes the cropped output from registers;
    otherwise it writes a frame and a crop follows.  Both against the oracle, many tiles."""
    for (H, W, r) in [(96, 300, 4), (96, 302, 4), (96, 300, 3), (257, 260, 8)]:
        x = synth.piecewise_stack(1, 1, H, W, seed=H + W + r, sigma=0.05)
        check(x, r, 4)


@pytest.mark.parametrize("r", [2, 8])
def test_fast_checkerboard_is_a_fixed_point(r):
    """Corners and edges are preserved (every pixel has a quadrant inside its own cell),
    at a size spanning many tiles; values as in the exact filter's invariant test."""
    cb = synth.checkerboard(512, 768, 4 * r)[None, None]
    out, _ = run(cb, r, 5, want_maps=False)
    np.testing.assert_array_equal(out, cb)


def test_fast_trivial_and_status_codes():
    x = torch.from_numpy(synth.piecewise_stack(1, 1, 20, 24, seed=1, sigma=0.05)).to(DEV)
    for r, it in ((0, 3), (3, 0)):
        np.testing.assert_array_equal(osbf.filter_fast(x, r, it).cpu().numpy(), x.cpu().numpy())
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter_fast(x, 17, 1)
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter_fast(x, -1, 1)
    assert e.value.status_name == "OSBF_EINVAL"
    with pytest.raises(TypeError):
        osbf.filter_fast(x.half(), 2, 1)


def test_fast_launch_plan():
    """The fast approximation shares the float32 forward's launch plan: at r % 4 == 0 and
    W % 4 == 0 the first pass pads the image itself and the last pass writes the cropped
    output (one launch per pass); otherwise a padding launch precedes the passes and a crop
    follows them.  Both plans against the oracle."""
    for (H, W, r, launches) in [(200, 512, 8, 4), (200, 302, 3, 4 + 2)]:
        x_np = synth.piecewise_stack(1, 2, H, W, seed=H + r, sigma=0.05)
        x = torch.from_numpy(x_np).to(DEV)
        osbf.filter_fast(x, r, 4)
        assert osbf.last_launch_count(0) == launches, (H, W, r)
        check(x_np, r, 4)
