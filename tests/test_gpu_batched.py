"""GPU checks of the batched persistent launch.

Every job of a batch must equal its own single-image filter call bit for bit (same
sweep code, same fused depth), and one job is also checked against the CPU oracle.
The bounded dependency wait is exercised by shortening it from the host: the call
must return OSBF_ETIMEOUT, with no hang, and the context must stay usable.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def make_batch(n, seed, hw=(1, 300), radii=(0, 1, 2, 3, 4, 6, 8, 12), iters=(0, 12)):
    rng = np.random.default_rng(seed)
    ins, rs, its = [], [], []
    for k in range(n):
        H, W = (int(v) for v in rng.integers(hw[0], hw[1] + 1, size=2))
        x = synth.piecewise_stack(1, 1, H, W, seed=1000 + k, sigma=0.05)[0, 0]
        ins.append(torch.from_numpy(x).to(DEV))
        rs.append(int(rng.choice(radii)))
        its.append(int(rng.integers(iters[0], iters[1] + 1)))
    return ins, rs, its


def test_batched_matches_single_calls():
    ins, rs, its = make_batch(40, seed=1)
    outs = osbf.batched(ins, rs, its)
    torch.cuda.synchronize()
    for x, r, it, o in zip(ins, rs, its, outs):
        want = osbf.filter(x, r, it)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o.cpu().numpy(), want.cpu().numpy())


def test_batched_replay_is_deterministic_and_matches_oracle():
    ins, rs, its = make_batch(12, seed=2, hw=(20, 200), radii=(1, 2, 3), iters=(1, 6))
    a = [o.cpu().numpy() for o in osbf.batched(ins, rs, its)]
    b = [o.cpu().numpy() for o in osbf.batched(ins, rs, its)]  # replays the cached graph
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    k = 0
    x = ins[k].cpu().numpy()
    maps = torch.zeros(osbf.maps_shape(ins[k], rs[k], its[k]), dtype=torch.uint8, device=DEV)
    osbf.filter(ins[k], rs[k], its[k], maps=maps)
    ref = oracle.filter(x.astype(np.float64), rs[k], its[k], hint=osbf.maps_frames(maps, x.shape[-1], rs[k]).cpu().numpy(),
                       hint_thresh=1e-6)["out"]
    assert np.abs(a[k] - ref).max() <= 1e-5


def test_batched_config4_sample():
    """256 single-channel images, H and W uniform in [64, 2048], r in {1,2,3,4,6,8},
    passes uniform in [1, 30]; a sample of jobs is compared with single calls."""
    ins, rs, its = make_batch(256, seed=4, hw=(64, 2048), radii=(1, 2, 3, 4, 6, 8), iters=(1, 30))
    outs = osbf.batched(ins, rs, its)
    lat = osbf.batched_latencies(256)
    assert len(lat) == 256 and all(t > 0 for t in lat)
    for k in (0, 17, 101, 255):
        want = osbf.filter(ins[k], rs[k], its[k])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(outs[k].cpu().numpy(), want.cpu().numpy())


def test_batched_wait_timeout_is_reported_and_recoverable():
    ins, rs, its = make_batch(16, seed=5, hw=(100, 400), radii=(2, 4), iters=(3, 8))
    try:
        osbf.set_wait_timeout(1)  # 1 ns: any item that has to wait gives up at once
        with pytest.raises(osbf.OSBFError) as e:
            osbf.batched(ins, rs, its)
        assert e.value.status_name == "OSBF_ETIMEOUT"
    finally:
        osbf.set_wait_timeout(0)
    outs = osbf.batched(ins, rs, its)  # the context stays usable
    want = osbf.filter(ins[3], rs[3], its[3])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(outs[3].cpu().numpy(), want.cpu().numpy())


def test_batched_bad_jobs():
    x = torch.zeros(8, 8, device=DEV)
    with pytest.raises(osbf.OSBFError) as e:
        osbf.batched([x], [17], [1])
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.batched([x], [1], [1], outputs=[x])
    assert e.value.status_name == "OSBF_EINVAL"
