"""GPU checks of the tuners (through the C ABI).

osbf_autotune times the forward's candidates (the tile kernel at every fused depth that
fits, the streaming strip kernel) on a synthetic image and records the fastest; a tuned
call must apply it (its launch count shows the depth) and still match the oracle.
osbf_autotune_batched times the batched launch's layout policies on the batch itself; the
recorded policy must be replayed by later batched calls, whose results stay bit-equal to
single filter calls.  A tuned single-call choice that the persistent kernel cannot run
sends that job through a plain call.  Tuned state lives in the context: every test resets
what it set, so the other test files see the default plan.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture
def tuned_keys():
    keys = []
    yield keys
    for k in keys:  # depth 1 on the tile kernel is the untuned plan
        osbf.set_tuned(torch.float32, *k, 1, "tile")


def test_autotune_records_and_applies_a_choice(tuned_keys):
    planes, H, W, r, it = 2, 300, 400, 3, 4
    tuned_keys.append((planes, H, W, r))
    osbf.autotune(torch.float32, planes, H, W, r, it)
    depth, variant = osbf.tuned(torch.float32, planes, H, W, r)
    print(f"\ntuned for {planes}x{H}x{W}, r={r}, {it} passes: depth {depth}, {variant} kernel")
    assert depth >= 1 and variant in ("tile", "strip")
    x_np = synth.piecewise_stack(1, planes, H, W, seed=90, sigma=0.05)
    x = torch.from_numpy(x_np).to(DEV)
    plain = osbf.filter(x, r, it)
    # r = 3: a padding launch, then ceil(it / depth) launches of fused passes
    assert osbf.last_launch_count(0) == 1 + -(-it // depth)
    maps = torch.zeros(osbf.maps_shape(x, r, it), dtype=torch.uint8, device=DEV)
    withmaps = osbf.filter(x, r, it, maps=maps)
    torch.cuda.synchronize()
    assert torch.equal(plain, withmaps)
    m = osbf.maps_frames(maps, W, r).cpu().numpy()
    ref = oracle.filter(x_np.astype(np.float64), r, it, hint=m, hint_thresh=1e-6)
    assert np.abs(plain.cpu().numpy().astype(np.float64) - ref["out"]).max() <= 1e-5


def test_set_tuned_is_applied_and_validated(tuned_keys):
    planes, H, W, r, it = 1, 200, 256, 4, 6
    tuned_keys.append((planes, H, W, r))
    x = torch.from_numpy(synth.piecewise_stack(1, planes, H, W, seed=91, sigma=0.05)).to(DEV)
    osbf.set_tuned(torch.float32, planes, H, W, r, 2, "tile")
    assert osbf.tuned(torch.float32, planes, H, W, r) == (2, "tile")
    osbf.filter(x, r, it)
    assert osbf.last_launch_count(0) == 1 + it // 2  # padding launch + three fused launches
    osbf.set_tuned(torch.float32, planes, H, W, r, 1, "strip")
    a = osbf.filter(x, r, it)
    b = osbf.filter(x, r, it, variant="strip")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with pytest.raises(osbf.OSBFError) as e:
        osbf.set_tuned(torch.float32, planes, H, W, 12, 1, "strip")  # the strip kernel stops at r = 8
    assert e.value.status_name == "OSBF_EUNSUPPORTED"


def make_jobs(n, seed):
    rng = np.random.default_rng(seed)
    ins, rs, its = [], [], []
    for k in range(n):
        H, W = (int(v) for v in rng.integers(40, 400, size=2))
        ins.append(torch.from_numpy(synth.piecewise_stack(1, 1, H, W, seed=3000 + k, sigma=0.05)[0, 0]).to(DEV))
        rs.append(int(rng.choice([1, 2, 3, 4, 6, 8])))
        its.append(int(rng.integers(1, 9)))
    return ins, rs, its


def test_autotune_batched_policy_is_replayed():
    ins, rs, its = make_jobs(24, seed=7)
    outs = [torch.empty_like(t) for t in ins]
    assert osbf.batched_policy(ins, rs, its, outs) is None
    osbf.autotune_batched(ins, rs, its, outs)
    pol = osbf.batched_policy(ins, rs, its, outs)
    print(f"\ntuned batched policy (job order, CTAs per SM): {pol}")
    assert pol is not None and pol[0] in (0, 1, 2) and pol[1] >= 1
    for o in outs:
        o.zero_()
    osbf.batched(ins, rs, its, outputs=outs)  # the tuned policy's cached graph
    assert osbf.last_launch_count(0) == 1
    for x, r, it, o in zip(ins, rs, its, outs):
        want = osbf.filter(x, r, it)
        torch.cuda.synchronize()
        assert torch.equal(o, want)


def test_batched_follows_the_tuned_single_call_choice(tuned_keys):
    """A job whose size class has a tuned strip kernel runs as a plain strip call; the other
    job (another size class) stays in the persistent launch."""
    small = torch.from_numpy(synth.piecewise_stack(1, 1, 100, 120, seed=92, sigma=0.05)[0, 0]).to(DEV)
    large = torch.from_numpy(synth.piecewise_stack(1, 1, 1500, 1500, seed=93, sigma=0.05)[0, 0]).to(DEV)
    r, it = 4, 5
    tuned_keys.append((1, 100, 120, r))
    osbf.set_tuned(torch.float32, 1, 100, 120, r, 1, "strip")
    outs = osbf.batched([small, large], [r, r], [it, it])
    want_small = osbf.filter(small, r, it, variant="strip")
    want_large = osbf.filter(large, r, it, variant="tile")
    torch.cuda.synchronize()
    assert torch.equal(outs[0], want_small)
    assert torch.equal(outs[1], want_large)
