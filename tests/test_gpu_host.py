"""osbf_filter_host (host buffers, planes in up to four chunks whose copies overlap the
filtering of their neighbours) against the device-buffer forward: bit-identical results
for every plane count (uneven chunks included), storage type and pinned / pageable
buffers, and status codes passed through."""
import numpy as np
import pytest
import torch

from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def device_result(x_host, r, iters):
    return osbf.filter(x_host.to(DEV), r, iters).cpu()


@pytest.mark.parametrize("shape", [(1, 1, 33, 70), (1, 3, 64, 100), (5, 1, 17, 23), (2, 3, 40, 50), (3, 3, 9, 130)])
@pytest.mark.parametrize("r", [1, 3, 8])
def test_host_matches_device_f32(shape, r):
    x = torch.from_numpy(synth.piecewise_stack(*shape, seed=sum(shape) + r, sigma=0.05))
    want = device_result(x, r, 3)
    got = osbf.filter_host(x.pin_memory(), r, 3)
    assert torch.equal(got, want)
    got_pageable = osbf.filter_host(x.clone(), r, 3)
    assert torch.equal(got_pageable, want)


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16, torch.uint8])
def test_host_matches_device_other_storage(dtype):
    x32 = synth.piecewise_stack(2, 3, 37, 61, seed=4, sigma=0.05)
    x = torch.from_numpy(synth.to_u8(x32)) if dtype == torch.uint8 else torch.from_numpy(x32).to(dtype)
    want = device_result(x, 2, 2)
    got = osbf.filter_host(x.pin_memory(), 2, 2)
    assert got.dtype == want.dtype and torch.equal(got, want)


def test_host_repeated_calls_and_large_planes():
    """Back-to-back calls reuse the context's staging buffers and streams; 3 planes of
    1024 x 1536 (one chunk per plane)."""
    x = torch.from_numpy(synth.piecewise_stack(1, 3, 1024, 1536, seed=9, sigma=0.05)).pin_memory()
    want = device_result(x, 4, 5)
    out = torch.empty_like(x).pin_memory()
    for _ in range(3):
        out.zero_()
        osbf.filter_host(x, 4, 5, out=out)
        assert torch.equal(out, want)


def test_host_status_codes():
    x = torch.from_numpy(synth.piecewise_stack(1, 2, 20, 24, seed=1, sigma=0.05))
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter_host(x, 17, 1)
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter_host(x, -1, 1)
    assert e.value.status_name == "OSBF_EINVAL"
    np.testing.assert_array_equal(osbf.filter_host(x, 0, 3).numpy(), x.numpy())
    with pytest.raises(ValueError):
        osbf.filter_host(x.to(DEV), 2, 1)
