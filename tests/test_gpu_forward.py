"""GPU parity of the forward filter against the CPU oracle (through the C ABI).

Accuracy rules (all on [0, 1] images):
  * float32: max |delta| <= 1e-5 on every pixel.  Where the oracle's best two |d_i|
    differ by less than 1e-6 (a near tie that float32 cannot decide the same way
    as float64) the oracle adopts the GPU's recorded selection ("hinted" mode); the
    number of such pixels is reported.  With one pass this is the literal rule.
  * uint8, one pass: bit-exact values and selection maps.
  * float16 / bfloat16 storage: compared with the oracle that rounds to the same
    storage type after every pass, hinted within one storage ulp; max |delta| <= 2
    storage ulps at 1.0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_05021_gb300 import osbf, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
F32_TOL = 1e-5
TIE_THRESH = 1e-6


def gpu_filter(x_np, r, iters, depth=0, tie="paper", want_maps=True, dtype=torch.float32, variant="auto"):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV).to(dtype)
    maps = torch.zeros(osbf.maps_shape(x, r, iters), dtype=torch.uint8, device=DEV) if want_maps else None
    out = osbf.filter(x, r, iters, depth=depth, tie=tie, maps=maps, variant=variant)
    torch.cuda.synchronize()
    return out.float().cpu().numpy(), (osbf.maps_frames(maps, x.shape[-1], r).cpu().numpy() if want_maps else None)


# Hinted pixels: (pixel, pass) pairs where the oracle adopted the GPU's selection inside the
# near-tie band and that changed the value.  Measured on the noisy float inputs: up to
# ~2e-5 of all pixel-passes over a few passes, up to ~1.1e-3 after 30 passes (smoothed
# regions make several windows' means nearly equal).  The bound is 5e-3.
MAX_HINTED_FRAC = 5e-3


def check_f32(x_np, r, iters, depth=0, tie="paper", max_hinted_frac=MAX_HINTED_FRAC, variant="auto"):
    out, maps = gpu_filter(x_np, r, iters, depth=depth, tie=tie, variant=variant)
    ref = oracle.filter(x_np.astype(np.float64), r, iters, tie=tie, hint=maps, hint_thresh=TIE_THRESH,
                        want_gaps=True)
    err = np.abs(out.astype(np.float64) - ref["out"])
    assert err.max() <= F32_TOL, (err.max(), np.unravel_index(err.argmax(), err.shape), ref["n_hinted"])
    frame_px_passes = maps.size
    assert ref["n_hinted"] <= max(4, max_hinted_frac * frame_px_passes), (ref["n_hinted"], frame_px_passes)
    # the literal rule's count: output pixels whose last pass had its best two |d_i| within 1e-6
    literal = int((oracle.crop(ref["gaps"][-1], r) < TIE_THRESH).sum()) if iters > 0 and r > 0 else 0
    print(f"\n{x_np.shape} r={r} passes={iters}: max|d| {err.max():.3g}, hinted {ref['n_hinted']} of "
          f"{frame_px_passes} pixel-passes, near ties in the last pass {literal}")
    return out, maps, ref


# ------------------------------------------------------------------------------------------
def test_config1_512_r2_10iters():
    """512 x 512 x 1 float32, r = 2, 10 passes, sigma = 0.05, seed 0 (the correctness config)."""
    x = synth.piecewise_stack(1, 1, 512, 512, seed=0, sigma=0.05)
    out, maps, ref = check_f32(x, 2, 10)
    plain = oracle.filter(x.astype(np.float64), 2, 10)["out"]
    print(f"\nconfig1: max|d| hinted {np.abs(out - ref['out']).max():.3g}, unhinted {np.abs(out - plain).max():.3g},"
          f" hinted pixels {ref['n_hinted']}")
    # the fast variant (no maps) agrees with the map-writing one
    fast, _ = gpu_filter(x, 2, 10, want_maps=False)
    np.testing.assert_array_equal(fast, out)


def test_literal_rule_one_pass():
    """One pass: max |delta| <= 1e-5 except where the oracle's two best scores are within 1e-6."""
    x = synth.piecewise_stack(1, 2, 300, 257, seed=1, sigma=0.05)
    for r in (1, 2, 4, 8):
        out, _ = gpu_filter(x, r, 1, want_maps=False)
        ref = oracle.filter(x.astype(np.float64), r, 1, want_gaps=True)
        gap = oracle.crop(ref["gaps"][0], r).reshape(out.shape)
        err = np.abs(out - ref["out"])
        assert err[gap >= TIE_THRESH].max() <= F32_TOL
        print(f"r={r}: near-tie pixels {(gap < TIE_THRESH).sum()}, max|d| elsewhere {err[gap >= TIE_THRESH].max():.3g}")


# the two float32 single-pass kernels: "strip" covers r <= 8, "tile" every radius
VARIANTS = [("tile", r) for r in (1, 2, 3, 5, 8, 11, 16)] + [("strip", r) for r in (1, 2, 3, 5, 6, 7, 8)]


@pytest.mark.parametrize("variant,r", VARIANTS)
@pytest.mark.parametrize("shape", [(1, 2, 70, 301), (2, 1, 131, 64)])
def test_radii_ragged_tiles(shape, variant, r):
    x = synth.piecewise_stack(*shape, seed=r, sigma=0.05)
    check_f32(x, r, 3, variant=variant)


@pytest.mark.parametrize("variant,r", [("tile", 4), ("tile", 8), ("tile", 12), ("tile", 16), ("strip", 4),
                                       ("strip", 8)])
@pytest.mark.parametrize("W", [256, 258])
def test_no_maps_kernels_match_oracle(variant, r, W):
    """The kernels a plain call runs (no maps): frame-to-frame passes at r % 4 == 0 leave
    through per-warp tensor stores (r = 4) or the early-load kernel's 32-byte register
    stores (r >= 8); the last pass writes the cropped output with tensor stores on the
    output-aligned grid when W % 4 == 0 and through staged rows of the direct kernel otherwise.
    Their results equal the map-writing run bit for bit (same arithmetic, so the maps run's
    selections are the no-maps run's), and the oracle, hinted with those maps, agrees
    within 1e-5 on every pixel."""
    x = synth.piecewise_stack(1, 2, 97, W, seed=60 + r, sigma=0.05)
    plain, _ = gpu_filter(x, r, 4, want_maps=False, variant=variant)
    out, maps, ref = check_f32(x, r, 4, variant=variant)
    np.testing.assert_array_equal(plain, out)
    assert np.abs(plain.astype(np.float64) - ref["out"]).max() <= F32_TOL


@pytest.mark.parametrize("r", [4, 8, 16])
@pytest.mark.parametrize("shape", [(1, 1, 1, 4), (1, 1, 3, 8), (1, 2, 29, 4), (2, 1, 70, 132), (1, 1, 40, 300)])
def test_padding_first_pass(shape, r):
    """Float32 at r % 4 == 0 with W % 4 == 0: the first pass reads the unpadded image and
    replicates its border into the frame ring itself (no padding launch).  Images smaller
    than r, one row high and spanning several tiles: the plain call equals the map-writing
    call, which pads with a separate launch, bit for bit, and the oracle within 1e-5."""
    x = synth.piecewise_stack(*shape, seed=70 + r, sigma=0.05)
    plain, _ = gpu_filter(x, r, 3, want_maps=False)
    launches = osbf.last_launch_count(0)
    out, maps, ref = check_f32(x, r, 3, max_hinted_frac=0.05)
    np.testing.assert_array_equal(plain, out)
    assert launches == 3  # three passes, no padding launch


def test_bench_shape_sampled():
    """The benchmark's own workload and launch sequence: 1 x 3 x 4096 x 4096 float32, r = 8,
    30 passes, the bench's input (seed 0).  The plain call (the padding first pass, early-load
    passes, the tensor-store pass into the output) equals the map-writing call bit for bit
    on the whole output; 32 x 32 regions --
    the top-left frame corner, a region straddling a tile seam in both axes, an interior
    region and the bottom-right corner -- match the oracle (dependency cone only, hinted
    with the run's maps) within 1e-5."""
    r, it, H, W = 8, 30, 4096, 4096
    x_np = synth.piecewise_stack(1, 3, H, W, seed=0, sigma=0.05)
    x = torch.from_numpy(x_np).to(DEV)
    plain = osbf.filter(x, r, it)
    maps = torch.empty(osbf.maps_shape(x, r, it), dtype=torch.uint8, device=DEV)
    withmaps = osbf.filter(x, r, it, maps=maps)
    torch.cuda.synchronize()
    assert torch.equal(plain, withmaps)
    FH, FW = H + 2 * r, W + 2 * r
    m = it * r
    # tiles are 32 rows x 128 columns of the frame: image row 24 and column 120 lie on seams
    regions = [(0, 0, 0), (0, 8, 104), (1, 2000, 3000), (2, H - 32, W - 32)]
    total_hinted = 0
    for p, y0, x0 in regions:
        y1, x1 = y0 + 32, x0 + 32
        fy0, fy1 = max(0, y0 + r - m), min(FH, y1 + r + m)
        fx0, fx1 = max(0, x0 + r - m), min(FW, x1 + r + m)
        hint = np.zeros((it, FH, FW), dtype=np.uint8)  # pages outside the cone stay untouched
        hint[:, fy0:fy1, fx0:fx1] = maps[:, p, fy0:fy1, fx0:fx1].cpu().numpy()
        ref, nh = oracle.filter_region(x_np[0, p].astype(np.float64), r, it, y0, y1, x0, x1, hint=hint,
                                       hint_thresh=TIE_THRESH, return_hinted=True)
        got = plain[0, p, y0:y1, x0:x1].cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).max()
        print(f"\nplane {p} region ({y0}, {x0}): max|d| {err:.3g}, hinted {nh}")
        assert err <= F32_TOL
        total_hinted += nh
        # the oracle iterates the whole cone: (fy1 - fy0) x (fx1 - fx0) pixels, 30 passes
        assert nh <= MAX_HINTED_FRAC * (fy1 - fy0) * (fx1 - fx0) * it


@pytest.mark.parametrize("depth", [1, 2, 3, 4, 8])
def test_fused_depths(depth):
    x = synth.piecewise_stack(1, 1, 97, 260, seed=42, sigma=0.05)
    for r in (1, 2, 4):
        check_f32(x, r, 9, depth=depth)


def test_depth_invariance():
    """Fused depths differ only in FP32 summation order: equal within 1e-6 wherever every
    pass made the same selection (downstream of a near tie the choice may differ, and each
    depth on its own is checked against the oracle in test_fused_depths)."""
    import scipy.ndimage as ndi

    x = synth.piecewise_stack(1, 1, 160, 200, seed=5, sigma=0.05)
    r, iters = 2, 8
    runs = [gpu_filter(x, r, iters, depth=d) for d in (1, 2, 4, 8)]
    out0, maps0 = runs[0]
    for o, m in runs[1:]:
        # a selection that differs at pass t can change every pixel within r*(iters-1-t)
        touched = np.zeros(maps0.shape[2:], dtype=bool)
        for t in range(iters):
            flips = m[t, 0] != maps0[t, 0]
            reach = r * (iters - 1 - t)
            touched |= ndi.maximum_filter(flips, size=2 * reach + 1) if reach else flips
        clean = ~touched[r:-r, r:-r]
        diff = np.abs(o - out0)[0, 0]
        assert clean.mean() > 0.9
        assert diff[clean].max() <= 1e-6


@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (1, 1, 1, 37), (1, 1, 29, 1), (1, 1, 5, 7), (1, 3, 33, 129)])
@pytest.mark.parametrize("r", [1, 2, 16])
def test_small_and_degenerate_shapes(shape, r):
    # frames one pixel wide or high are symmetric (replicated rows or columns), so opposite
    # windows tie often: measured up to 1.6 % hinted pixel-passes, bound 5 %
    x = synth.piecewise_stack(*shape, seed=7, sigma=0.1)
    check_f32(x, r, 3, max_hinted_frac=0.05)


def test_r0_and_iters0_are_identity():
    x = synth.piecewise_stack(1, 2, 40, 50, seed=3)
    for r, it in ((0, 5), (3, 0), (0, 0)):
        out, maps = gpu_filter(x, r, it)
        np.testing.assert_array_equal(out, x)
        if it > 0:
            assert (maps == 1).all()


def test_tie_order_appendix():
    x = np.round(synth.piecewise_stack(1, 1, 90, 140, seed=8, sigma=0.05) * 16) / 16  # many exact ties
    x = x.astype(np.float32)
    for r in (1, 2, 3):
        # values on a 1/16 grid tie exactly between quadrants and half windows, whose means
        # float32 rounds differently: in-band hints are frequent here (bound 5 %)
        check_f32(x, r, 4, tie="appendix", max_hinted_frac=0.05)
        check_f32(x, r, 4, tie="paper", max_hinted_frac=0.05)


@pytest.mark.parametrize("r", [3, 4, 8, 12])
@pytest.mark.parametrize("W", [256, 301])
def test_appendix_order_single_pass(r, W):
    """The appendix tie order's float32 single-pass kernels (plain and map-writing, results
    and selections staged; every pass, also the last into the cropped output at any W):
    several planes, many tiles, plain == map-writing bit for bit, and the oracle in the
    appendix order, hinted with the run's maps, within 1e-5.  A depth-2 run (the fused-pass
    kernel) agrees with the oracle as well."""
    x = synth.piecewise_stack(1, 2, 97, W, seed=90 + r, sigma=0.05)
    plain, _ = gpu_filter(x, r, 4, tie="appendix", want_maps=False)
    out, maps, ref = check_f32(x, r, 4, tie="appendix")
    np.testing.assert_array_equal(plain, out)
    check_f32(x, r, 4, depth=2, tie="appendix")


def test_edges_corners_checkerboard_preserved():
    """Paper-stated invariants, at a size spanning many tiles."""
    for r in (2, 8):
        cb = synth.checkerboard(512, 768, 4 * r)
        out, _ = gpu_filter(cb, r, 5, want_maps=False)
        np.testing.assert_array_equal(out, cb)
        const = np.full((300, 333), 0.5, dtype=np.float32)
        out, _ = gpu_filter(const, r, 7, want_maps=False)
        np.testing.assert_array_equal(out, const)


# ------------------------------------------------------------------------------------------
# 8-bit input
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("r", [1, 2, 3, 4, 8, 16])
def test_u8_one_pass_bit_exact(r):
    x = synth.to_u8(synth.piecewise_stack(1, 2, 150, 211, seed=10 + r, sigma=0.05))
    x[0, 0, 20:40, 30:60] = 77  # plateaus: exact ties
    for tie in ("paper", "appendix"):
        out, maps = gpu_filter(x, r, 1, tie=tie, dtype=torch.uint8)
        frame, m = oracle.u8_first_pass(x, r, tie=tie)
        want = oracle.crop(frame, r).reshape(out.shape)
        np.testing.assert_array_equal(out.view(np.uint32), want.view(np.uint32))
        np.testing.assert_array_equal(maps[0], m)


def test_u8_config1_one_pass():
    x = synth.to_u8(synth.piecewise_stack(1, 1, 512, 512, seed=0, sigma=0.05))
    out, maps = gpu_filter(x, 2, 1, dtype=torch.uint8)
    frame, m = oracle.u8_first_pass(x, 2)
    np.testing.assert_array_equal(out.view(np.uint32), oracle.crop(frame, 2).reshape(out.shape).view(np.uint32))
    np.testing.assert_array_equal(maps[0], m)


def test_u8_several_passes():
    """First pass exact in integers, later passes in float32 on the 0..255 scale."""
    x = synth.to_u8(synth.piecewise_stack(1, 1, 100, 130, seed=12, sigma=0.05))
    r, iters = 2, 4
    out, maps = gpu_filter(x, r, iters, dtype=torch.uint8)
    frame, m = oracle.u8_first_pass(x, r)
    np.testing.assert_array_equal(maps[0], m)
    rest = oracle.iterate_frame(frame.astype(np.float64), r, iters - 1, hint=maps[1:], hint_thresh=255 * TIE_THRESH)
    want = oracle.crop(rest["frame"], r).reshape(out.shape)
    assert np.abs(out - want).max() <= 255 * F32_TOL


# ------------------------------------------------------------------------------------------
# 16-bit storage
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dt,name,ulp1", [(torch.float16, "f16", 2.0**-10), (torch.bfloat16, "bf16", 2.0**-7)])
def test_half_storage(dt, name, ulp1):
    # r = 1, 3, 6: tile grids shifted by 7, 5, 2 columns (halo exactly r, boxes on 16
    # bytes); W = 188 with r = 4, 8 also runs the last pass straight into the output
    cases = [(synth.round_to_storage(synth.piecewise_stack(1, 2, 150, 190, seed=21, sigma=0.03), name), r)
             for r in (1, 3, 4, 6)]
    cases += [(synth.round_to_storage(synth.piecewise_stack(1, 1, 70, 188, seed=22, sigma=0.03), name), r)
              for r in (4, 8)]
    for x, r in cases:
        out, maps = gpu_filter(x, r, 6, dtype=dt)
        fast, _ = gpu_filter(x, r, 6, dtype=dt, want_maps=False)
        np.testing.assert_array_equal(fast, out)
        # quantised values make exact |d_i| ties common; within one storage ulp the oracle
        # follows the GPU's recorded choice
        ref = oracle.filter(x.astype(np.float64), r, 6, storage=name, hint=maps, hint_thresh=ulp1)["out"]
        exact = oracle.filter(x.astype(np.float64), r, 6)["out"]
        err = np.abs(out - ref)
        frac_equal = np.mean(err == 0)
        print(f"\n{name} r={r}: vs rounded oracle max {err.max():.3g} (equal {frac_equal:.5f}, "
              f"> 1 ulp at 1.0: {(err > ulp1).sum()}); vs FP64 oracle max {np.abs(out - exact).max():.3g} "
              f"mean {np.abs(out - exact).mean():.3g}")
        # the kernel's new value is the storage rounding of the correctly rounded float32
        # quotient S_m / n_m, so it equals the oracle's rounding of the exact mean wherever
        # the float32 window sums are exact (16-bit values near 1 sum exactly; values below
        # about 2^-7 carry bits past float32's 24 when summed with large ones)
        assert frac_equal >= 0.99
        assert err.max() <= 2 * ulp1


@pytest.mark.parametrize("name", ["f32", "f16", "bf16"])
def test_precision_config_error_vs_fp64(name):
    """The storage-precision configuration (1 x 3 x 4320 x 7680, r = 4, 30 passes, noise
    sigma 0.03) on a 48 x 48 sample of plane 0 at the image centre.

    float32: the FP32 rule -- max |delta| <= 1e-5 against the FP64 oracle hinted with the
    run's own maps (near ties counted).  16-bit storage: the error against the FP64 oracle
    (not rounded to storage) is reported and bounded with a margin over the measured values
    (max / mean 1.1e-3 / 2.4e-4 for f16, 3.5e-3 / 9.1e-4 for bf16), and the selection flips
    against the float32 run -- (frame pixel, pass) pairs whose selected window differs --
    are counted over all three planes and 30 passes."""
    dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[name]
    H, W, r, it = 4320, 7680, 4, 30
    x32 = synth.piecewise_stack(1, 3, H, W, seed=3, sigma=0.03)
    xin = x32 if name == "f32" else synth.round_to_storage(x32, name)
    y0, x0, s = H // 2, W // 2, 48
    xt = torch.from_numpy(xin).to(DEV).to(dt)
    maps = torch.empty(osbf.maps_shape(xt, r, it), dtype=torch.uint8, device=DEV)
    out = osbf.filter(xt, r, it, maps=maps)
    got = out[0, 0, y0:y0 + s, x0:x0 + s].float().cpu().numpy().astype(np.float64)
    plain = oracle.filter_region(xin[0, 0].astype(np.float64), r, it, y0, y0 + s, x0, x0 + s)
    err_plain = np.abs(got - plain)
    FH, FW = H + 2 * r, W + 2 * r
    if name == "f32":
        m = it * r
        fy0, fy1, fx0, fx1 = y0 + r - m, y0 + s + r + m, x0 + r - m, x0 + s + r + m
        hint = np.zeros((it, FH, FW), dtype=np.uint8)
        hint[:, fy0:fy1, fx0:fx1] = maps[:, 0, fy0:fy1, fx0:fx1].cpu().numpy()
        ref, nh = oracle.filter_region(xin[0, 0].astype(np.float64), r, it, y0, y0 + s, x0, x0 + s, hint=hint,
                                       hint_thresh=TIE_THRESH, return_hinted=True)
        err = np.abs(got - ref)
        print(f"\nf32: hinted max {err.max():.3g} ({nh} hinted); unhinted max {err_plain.max():.3g} "
              f"mean {err_plain.mean():.3g}")
        assert err.max() <= F32_TOL
        assert nh <= MAX_HINTED_FRAC * (fy1 - fy0) * (fx1 - fx0) * it
        return
    bound = {"f16": (6e-3, 1.2e-3), "bf16": (2e-2, 5e-3)}[name]
    x_f32 = torch.from_numpy(x32).to(DEV)
    maps32 = torch.empty(osbf.maps_shape(x_f32, r, it), dtype=torch.uint8, device=DEV)
    osbf.filter(x_f32, r, it, maps=maps32)
    flips = [int((maps[t, ..., :FW] != maps32[t, ..., :FW]).sum()) for t in range(it)]
    total = 3 * FH * FW * it
    print(f"\n{name}: max {err_plain.max():.3g} mean {err_plain.mean():.3g} vs FP64; selection flips vs f32 "
          f"{sum(flips)} of {total} pixel-passes ({sum(flips) / total:.3%}); pass 1: {flips[0]}, pass 30: "
          f"{flips[-1]}")
    assert err_plain.max() <= bound[0] and err_plain.mean() <= bound[1]
    # Reported, not bounded tightly: the rounded input already changes the first pass's
    # choice where windows are close (measured 1.0 % f16, 6.5 % bf16 of pass-1 pixels), and
    # as passes flatten the image, windows with nearly equal means swap freely (25 % / 43 %
    # of all pixel-passes) at little cost in value (the error bounds above).
    assert flips[0] < 0.1 * total / it


def test_half_depth_invariance():
    """Rounding to storage after every pass makes fused depths agree exactly."""
    x = synth.round_to_storage(synth.piecewise_stack(1, 1, 120, 150, seed=4, sigma=0.03), "f16")
    a, _ = gpu_filter(x, 2, 8, depth=1, dtype=torch.float16, want_maps=False)
    b, _ = gpu_filter(x, 2, 8, depth=4, dtype=torch.float16, want_maps=False)
    assert np.mean(a == b) > 0.999


# ------------------------------------------------------------------------------------------
# argument errors come back as status codes
# ------------------------------------------------------------------------------------------
def test_status_codes():
    x = torch.zeros(1, 1, 8, 8, device=DEV)
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter(x, 17, 1)
    assert e.value.status_name == "OSBF_EUNSUPPORTED"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter(x, -1, 1)
    assert e.value.status_name == "OSBF_EINVAL"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter(x, 1, 1, out=x)
    assert e.value.status_name == "OSBF_EINVAL"
    with pytest.raises(osbf.OSBFError) as e:
        osbf.filter(x, 1, 1, depth=9)
    assert e.value.status_name == "OSBF_EINVAL"
    osbf.filter(x, 1, 1)  # the context stays usable
