"""GPU parity of the backward (vector-Jacobian product) against the oracle's adjoint.

With every selection frozen to the maps the forward recorded, the filter is linear,
and the oracle's adjoint (oracle.adjoint) is its exact transpose in FP64 -- itself
pinned by the transpose identity and by central finite differences in
tests/test_oracle_pins.py.  The CUDA backward must match it to float32 accuracy:
|delta| <= 1e-5 * (1 + max |grad|) on every pixel.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def fwd_with_maps(x_np, r, iters):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    maps = torch.zeros(osbf.maps_shape(x, r, iters), dtype=torch.uint8, device=DEV)
    out = osbf.filter(x, r, iters, maps=maps)
    return x, out, maps


def check_adjoint(g_gpu, g_np, maps, r, iters):
    want = oracle.adjoint(g_np.astype(np.float64), osbf.maps_frames(maps, g_np.shape[-1], r).cpu().numpy(), r, iters)
    got = g_gpu.cpu().numpy().astype(np.float64)
    tol = 1e-5 * (1.0 + np.abs(want).max())
    err = np.abs(got - want).max()
    assert err <= tol, (err, tol)
    return err


@pytest.mark.parametrize("r", list(range(1, 17)))
@pytest.mark.parametrize("shape", [(1, 1, 70, 150), (2, 1, 33, 129)])
def test_backward_matches_oracle_adjoint(shape, r):
    x_np = synth.piecewise_stack(*shape, seed=r, sigma=0.05)
    iters = 3
    x, out, maps = fwd_with_maps(x_np, r, iters)
    g_np = np.random.default_rng(r).standard_normal(x_np.shape).astype(np.float32)
    g = torch.from_numpy(g_np).to(DEV)
    gi = osbf.backward(g, maps, r, iters)
    torch.cuda.synchronize()
    check_adjoint(gi, g_np, maps, r, iters)


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1, 1, 1, 9), (1, 1, 7, 1), (1, 2, 5, 6)])
def test_backward_degenerate_shapes(shape):
    x_np = synth.piecewise_stack(*shape, seed=1, sigma=0.1)
    for r in (1, 3):
        x, out, maps = fwd_with_maps(x_np, r, 2)
        g_np = np.ones(x_np.shape, dtype=np.float32)
        gi = osbf.backward(torch.from_numpy(g_np).to(DEV), maps, r, 2)
        torch.cuda.synchronize()
        check_adjoint(gi, g_np, maps, r, 2)


def test_autograd_function():
    """The torch.autograd.Function path gives the oracle's adjoint of the recorded maps."""
    x_np = synth.piecewise_stack(1, 2, 48, 64, seed=3, sigma=0.05)
    r, iters = 2, 4
    x = torch.from_numpy(x_np).to(DEV).requires_grad_(True)
    y = osbf.osbf(x, r, iters)
    g = torch.randn_like(y)
    y.backward(g)
    maps = torch.zeros(osbf.maps_shape(x, r, iters), dtype=torch.uint8, device=DEV)
    osbf.filter(x.detach(), r, iters, maps=maps)
    check_adjoint(x.grad, g.cpu().numpy(), maps, r, iters)


def test_checkpointed_forward_and_backward():
    x_np = synth.piecewise_stack(1, 3, 64, 90, seed=4, sigma=0.05)
    r, iters = 3, 7
    x, out, maps = fwd_with_maps(x_np, r, iters)
    for interval in (1, 2, 3, 7, 10):
        out_ck, ck = osbf.filter_checkpointed(x, r, iters, interval)
        g = torch.randn_like(out)
        gi_maps = osbf.backward(g, maps, r, iters)
        gi_ck = osbf.backward_checkpointed(g, ck, r, iters, interval)
        torch.cuda.synchronize()
        a, b = out_ck.cpu().numpy(), out.cpu().numpy()
        ga, gb = gi_ck.cpu().numpy(), gi_maps.cpu().numpy()
        if interval >= iters:
            # one segment: the same fused groups as the plain call, hence the same bits
            np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(ga, gb)
        else:
            # segment boundaries regroup the fused passes: float32 summation order differs
            # (last-ulp changes), and a near tie may be decided the other way
            assert np.mean(np.abs(a - b) <= 1e-6) > 0.99 and np.mean(np.abs(a - b) <= 1e-5) > 0.995
            scale = np.abs(gb).max()
            assert np.mean(np.abs(ga - gb) <= 1e-5 * scale) > 0.99
    # the autograd wrapper in checkpoint mode
    xx = x.clone().requires_grad_(True)
    yy = osbf.osbf(xx, r, iters, checkpoint_interval=3)
    gg = torch.randn_like(yy)
    yy.backward(gg)
    gi = osbf.backward(gg, maps, r, iters).cpu().numpy()
    assert np.mean(np.abs(xx.grad.cpu().numpy() - gi) <= 1e-5 * np.abs(gi).max()) > 0.99


def test_config5_sample():
    """Differentiation config: 16 x 3 x 512 x 512, r = 3, 5 passes, MSE(osbf(noisy), clean).
    The full batch runs on the GPU; two planes are checked against the oracle adjoint."""
    N, C, H, W, r, iters = 16, 3, 512, 512, 3, 5
    noisy = synth.piecewise_stack(N, C, H, W, seed=50, sigma=0.05)
    clean = synth.piecewise_stack(N, C, H, W, seed=50, sigma=0.0)
    x = torch.from_numpy(noisy).to(DEV).requires_grad_(True)
    y = osbf.osbf(x, r, iters)
    loss = torch.mean((y - torch.from_numpy(clean).to(DEV)) ** 2)
    loss.backward()
    maps = torch.zeros(osbf.maps_shape(x, r, iters), dtype=torch.uint8, device=DEV)
    osbf.filter(x.detach(), r, iters, maps=maps)
    gy = (2.0 / y.numel()) * (y.detach() - torch.from_numpy(clean).to(DEV))
    planes = [0, 47]
    P = N * C
    m = osbf.maps_frames(maps, W, r).cpu().numpy()
    for p in planes:
        want = oracle.adjoint(gy.reshape(P, H, W)[p].cpu().numpy().astype(np.float64), m[:, p:p + 1], r, iters)
        got = x.grad.reshape(P, H, W)[p].cpu().numpy()
        # gradients of a mean are ~1e-7 in size: compare relative to their scale
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


def test_backward_status_codes():
    g = torch.zeros(1, 1, 8, 8, device=DEV)
    with pytest.raises(osbf.OSBFError) as e:
        osbf.backward(g, torch.zeros(osbf.maps_shape(g, 17, 1), dtype=torch.uint8, device=DEV), 17, 1)
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.backward(g, torch.zeros(osbf.maps_shape(g, -1, 1), dtype=torch.uint8, device=DEV), -1, 1)
    assert e.value.status_name == "OSBF_EINVAL"
    # maps of the wrong shape are refused before any launch
    with pytest.raises(ValueError):
        osbf.backward(g, torch.zeros(1, 1, 10, 10, dtype=torch.uint8, device=DEV), 1, 1)
    # maps must start on 16 bytes (the backward reads them with tensor copies)
    buf = torch.zeros(osbf.maps_shape(g, 1, 1)[-1] * 10 + 16, dtype=torch.uint8, device=DEV)
    with pytest.raises(osbf.OSBFError) as e:
        lib, ctx = osbf.lib(), osbf.context(0)
        gi = torch.empty_like(g)
        st = lib.osbf_filter_backward(ctx, g.data_ptr(), gi.data_ptr(), buf.data_ptr() + 1, 1, 1, 8, 8, 1, 1,
                                      osbf._stream(0))
        osbf._check(st, ctx)
    assert e.value.status_name == "OSBF_EINVAL"
