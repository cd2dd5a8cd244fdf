"""GPU parity of the 3D filter (osbf_filter_3d; Sec. "Higher Dimension Case") against the
oracle's filter3d: with the GPU's selections as hints at near ties (best two |d| within
1e-6), every voxel within 1e-5 of the FP64 oracle after several passes; map-writing and
plain runs agree bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def volume(P, D, H, W, seed):
    """Piecewise-constant slabs with noise: each depth slice a synthetic 2D scene, slices
    grouped into a few blocks that share their scene (edges across depth too)."""
    rng = np.random.default_rng(seed)
    blocks = synth.piecewise_stack(1, P * 3, H, W, seed=seed, sigma=0.0)[0]
    v = np.empty((P, D, H, W), np.float32)
    for p in range(P):
        cut = sorted(rng.integers(1, max(D, 2), size=2))
        for z in range(D):
            v[p, z] = blocks[p * 3 + (0 if z < cut[0] else (1 if z < cut[1] else 2))]
    v += rng.normal(0, 0.05, v.shape).astype(np.float32)
    return np.clip(v, 0, 1)[None]


def run(x_np, r, iters, want_maps=True):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    maps = torch.zeros(osbf.maps3d_shape(x, r, iters), dtype=torch.uint8, device=DEV) if want_maps else None
    out = osbf.filter3d(x, r, iters, maps=maps)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (maps.cpu().numpy() if want_maps else None)


def check(x_np, r, iters):
    out, maps = run(x_np, r, iters)
    ref = oracle.filter3d(x_np.astype(np.float64), r, iters, hint=maps, hint_thresh=1e-6)
    err = np.abs(out - ref["out"]).max()
    assert err <= 1e-5, (r, iters, err)
    plain, _ = run(x_np, r, iters, want_maps=False)
    np.testing.assert_array_equal(out, plain)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_3d_matches_oracle(r):
    # FH, FW exceed one 32 x 64 tile; ragged edges in every axis
    check(volume(2, 9, 37, 70, seed=r), r, 2)


@pytest.mark.parametrize("shape", [(1, 1, 1, 1, 1), (1, 1, 3, 1, 5), (1, 2, 5, 6, 7), (1, 1, 2, 33, 65)])
def test_3d_shapes(shape):
    x = np.random.default_rng(sum(shape)).random(shape).astype(np.float32)
    for r in (1, 2):
        check(x, r, 2)


def test_3d_checkerboard_is_a_fixed_point():
    """Whole cells of 2r on every axis: every voxel owns an octant inside its cell (a cell
    cut thinner than r+1 at the volume's end is not a fixed point -- the zero border
    reaches it -- in the oracle either)."""
    r, c = 2, 4
    zz, yy, xx = np.mgrid[0:3 * c, 0:5 * c, 0:9 * c]
    cb = np.where(((zz // c) + (yy // c) + (xx // c)) % 2 == 0, 0.25, 0.75).astype(np.float32)[None, None]
    out, _ = run(cb, r, 4, want_maps=False)
    np.testing.assert_array_equal(out, cb)
    np.testing.assert_array_equal(oracle.filter3d(cb.astype(np.float64), r, 4)["out"], cb)


def test_3d_trivial_and_status_codes():
    x = torch.from_numpy(np.random.default_rng(0).random((1, 1, 4, 6, 8)).astype(np.float32)).to(DEV)
    for r, it in ((0, 2), (2, 0)):
        np.testing.assert_array_equal(osbf.filter3d(x, r, it).cpu().numpy(), x.cpu().numpy())
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter3d(x, 5, 1)
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter3d(x, -1, 1)
    assert e.value.status_name == "OSBF_EINVAL"
    with pytest.raises(ValueError):
        osbf.filter3d(x[0], 1, 1)
