"""Pins of the CPU oracle against what the paper and plain mathematics fix.

None of these tests compares the oracle with itself.  They check it against
  * a hand-derived worked example (tests/golden/spike_r1.txt);
  * a pure-Python brute force written from the set definitions of Eq. (6)-(13)
    and Algorithm 2 (tiny frames only);
  * the eight window means as 2D correlations (scipy) of the padded frame with
    indicator kernels built from the set definitions of Eq. (6)-(13), in both tie
    orders;
  * the classical box filter (scipy.ndimage.uniform_filter): half-window and
    quadrant sums must recombine into it (the separable construction of the
    section "Separable Kernels");
  * fixed points the paper states: a flat region and noise-free ideal edges,
    corners and checkerboards are preserved;
  * exact rational arithmetic (fractions) for the 8-bit rule;
  * the transpose identity <A v, w> = <v, A^T w> and central finite differences
    for the adjoint;
  * torch's own f16 / bf16 conversions for the storage rounding.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from paper_2108_05021_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------
# independent brute force: Eq. (6)-(13) as set predicates, Algorithm 2, appendix frame
# ----------------------------------------------------------------------------------
def _in_window(i, r, x, y, u, v):
    """(u, v) in N_i(x, y), u = column, v = row -- typed from Eq. (6)-(13)."""
    return {
        1: x - r <= u <= x and y <= v <= y + r,
        2: x <= u <= x + r and y <= v <= y + r,
        3: x <= u <= x + r and y - r <= v <= y,
        4: x - r <= u <= x and y - r <= v <= y,
        5: x - r <= u <= x and abs(y - v) <= r,
        6: x <= u <= x + r and abs(y - v) <= r,
        7: abs(u - x) <= r and y <= v <= y + r,
        8: abs(u - x) <= r and y - r <= v <= y,
    }[i]


def _kernel_weight(i, r):
    # weights of k1..k4 are (r+1)^-2, of k5..k8 (r+1)^-1 (2r+1)^-1
    return Fraction(1, (r + 1) ** 2) if i <= 4 else Fraction(1, (r + 1) * (2 * r + 1))


def brute_force(img, r, iters, order=(1, 2, 3, 4, 5, 6, 7, 8)):
    H, W = len(img), len(img[0])
    FH, FW = H + 2 * r, W + 2 * r
    U = [[img[min(max(fy - r, 0), H - 1)][min(max(fx - r, 0), W - 1)] for fx in range(FW)] for fy in range(FH)]
    for _ in range(iters):
        new = [[0.0] * FW for _ in range(FH)]
        for y in range(FH):
            for x in range(FW):
                best, best_ad = None, None
                for i in order:
                    s = 0.0
                    for v in range(y - r, y + r + 1):
                        for u in range(x - r, x + r + 1):
                            if 0 <= v < FH and 0 <= u < FW and _in_window(i, r, x, y, u, v):
                                s += U[v][u]
                    mean = s * float(_kernel_weight(i, r))
                    ad = abs(mean - U[y][x])
                    if best is None or ad < best_ad:
                        best, best_ad = mean, ad
                new[y][x] = best
        U = new
    return np.array([row[r:r + W] for row in U[r:r + H]])


# ----------------------------------------------------------------------------------
def test_golden_spike():
    rows = np.loadtxt(os.path.join(GOLDEN, "spike_r1.txt"), comments="#")
    for it, *expect in rows:
        got = oracle.filter(np.array([[0.0, 1.0, 0.0]]), r=1, iters=int(it))["out"]
        np.testing.assert_array_equal(got, np.array([expect]))


@pytest.mark.parametrize("r", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (4, 1), (3, 4), (5, 6)])
def test_brute_force_matches(shape, r):
    rng = np.random.default_rng(hash((shape, r)) % 2**32)
    img = rng.random(shape)
    iters = 2
    want = brute_force(img.tolist(), r, iters)
    got = oracle.filter(img, r, iters)["out"]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_brute_force_appendix_order():
    rng = np.random.default_rng(7)
    img = np.round(rng.random((4, 5)) * 4) / 4  # many exact ties
    want = brute_force(img.tolist(), 1, 2, order=(6, 5, 7, 8, 2, 1, 3, 4))
    got = oracle.filter(img, 1, 2, tie="appendix")["out"]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    want_p = brute_force(img.tolist(), 1, 2)
    got_p = oracle.filter(img, 1, 2, tie="paper")["out"]
    np.testing.assert_allclose(got_p, want_p, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------------
# window means by 2D correlation with the indicator kernels of Eq. (6)-(13)
# ----------------------------------------------------------------------------------
def window_kernels(r):
    """The eight box kernels k1..k8 as (2r+1) x (2r+1) weight arrays, each built from the
    set predicate of its window (Eq. (6)-(13)) and normalised by its pixel count (Sec.
    "One-sided Kernels for Box Filter").  Entry [dv + r, du + r] weights the pixel at row
    offset dv and column offset du from the centre."""
    ks = []
    for i in range(1, 9):
        k = np.zeros((2 * r + 1, 2 * r + 1))
        for dv in range(-r, r + 1):
            for du in range(-r, r + 1):
                k[dv + r, du + r] = 1.0 if _in_window(i, r, 0, 0, du, dv) else 0.0
        ks.append(k / k.sum())
    return ks


def correlation_filter(img, r, iters, order):
    """Algorithm 2 with each window mean taken as a 2D correlation of the frame with its
    kernel (scipy, zeros beyond the frame), on the replicate-padded frame, first argmin of
    |d_i| in `order`, cropped at the end."""
    im = np.pad(img, r, mode="edge")
    ks = window_kernels(r)
    for _ in range(iters):
        means = np.stack([ndi.correlate(im, ks[i - 1], mode="constant", cval=0.0) for i in order])
        ind = np.argmin(np.abs(means - im), axis=0)  # numpy's argmin returns the first minimum
        im = np.take_along_axis(means, ind[None], axis=0)[0]
    return im[r:-r or None, r:-r or None] if r else im


@pytest.mark.parametrize("r", [1, 2, 3, 5])
@pytest.mark.parametrize("tie,order", [("paper", (1, 2, 3, 4, 5, 6, 7, 8)), ("appendix", (6, 5, 7, 8, 2, 1, 3, 4))])
def test_correlation_semantics(r, tie, order):
    rng = np.random.default_rng(100 + r)
    img = rng.random((17, 23))
    for iters in (1, 3):
        want = correlation_filter(img, r, iters, order)
        got = oracle.filter(img, r, iters, tie=tie)["out"]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------------
# the classical box filter recovered from the one-sided sums
# ----------------------------------------------------------------------------------
def _shift_sum(f, axis, shifts):
    """sum_k f shifted by +k along `axis` (out[i] = sum_k f[i - k]), zero outside."""
    out = np.zeros_like(f)
    n = f.shape[axis]
    for k in shifts:
        src = [slice(None)] * 2
        dst = [slice(None)] * 2
        if k >= 0:
            src[axis], dst[axis] = slice(0, n - k), slice(k, n)
        else:
            src[axis], dst[axis] = slice(-k, n), slice(0, n + k)
        out[tuple(dst)] += f[tuple(src)]
    return out


@pytest.mark.parametrize("r", [0, 1, 2, 4])
def test_box_filter_recovered(r):
    rng = np.random.default_rng(200 + r)
    frame = rng.random((2, 13, 19))
    m = oracle.window_means(frame, r)
    nq, nh, nb = (r + 1) ** 2, (r + 1) * (2 * r + 1), (2 * r + 1) ** 2
    S = np.stack([m[i] * (nq if i < 4 else nh) for i in range(8)])
    for p in range(frame.shape[0]):
        f = frame[p]
        box = ndi.uniform_filter(f, size=2 * r + 1, mode="constant", cval=0.0) * nb
        row = ndi.uniform_filter1d(f, size=2 * r + 1, axis=1, mode="constant", cval=0.0) * (2 * r + 1)
        col = ndi.uniform_filter1d(f, size=2 * r + 1, axis=0, mode="constant", cval=0.0) * (2 * r + 1)
        s = S[:, p]
        np.testing.assert_allclose(s[4] + s[5] - col, box, atol=1e-10)  # left + right halves
        np.testing.assert_allclose(s[6] + s[7] - row, box, atol=1e-10)  # down + up halves
        np.testing.assert_allclose(s[0] + s[1] + s[2] + s[3] - row - col - f, box, atol=1e-10)
        # a half window is the union of its two quadrants minus their shared segment
        row_left = _shift_sum(f, axis=1, shifts=range(0, r + 1))     # f(y, x-k), k = 0..r
        col_down = _shift_sum(f, axis=0, shifts=range(-r, 1))        # f(y+k, x), k = 0..r
        np.testing.assert_allclose(s[0] + s[3] - row_left, s[4], atol=1e-10)  # N1 u N4 = N5
        np.testing.assert_allclose(s[0] + s[1] - col_down, s[6], atol=1e-10)  # N1 u N2 = N7


@pytest.mark.parametrize("r", [1, 3])
def test_window_geometry_symmetries(r):
    """Mirroring the frame permutes the eight windows as their definitions imply."""
    rng = np.random.default_rng(300 + r)
    f = rng.random((11, 14))
    m = oracle.window_means(f, r)[:, 0]
    mx = oracle.window_means(f[:, ::-1].copy(), r)[:, 0][:, :, ::-1]  # flip x
    my = oracle.window_means(f[::-1, :].copy(), r)[:, 0][:, ::-1, :]  # flip y
    mt = oracle.window_means(f.T.copy(), r)[:, 0].transpose(0, 2, 1)  # swap x and y
    flip_x = {1: 2, 2: 1, 3: 4, 4: 3, 5: 6, 6: 5, 7: 7, 8: 8}
    flip_y = {1: 4, 4: 1, 2: 3, 3: 2, 5: 5, 6: 6, 7: 8, 8: 7}
    swap = {1: 3, 3: 1, 2: 2, 4: 4, 5: 8, 8: 5, 6: 7, 7: 6}
    for i in range(1, 9):
        np.testing.assert_allclose(mx[flip_x[i] - 1], m[i - 1], atol=1e-12)
        np.testing.assert_allclose(my[flip_y[i] - 1], m[i - 1], atol=1e-12)
        np.testing.assert_allclose(mt[swap[i] - 1], m[i - 1], atol=1e-12)


def test_window_means_constant_interior():
    r = 2
    f = np.ones((9, 9))
    m = oracle.window_means(f, r)[:, 0]
    np.testing.assert_array_equal(m[:, r:-r, r:-r], np.ones((8, 5, 5)))


# ----------------------------------------------------------------------------------
# fixed points: flat regions, ideal edges, corners, checkerboards (edge preservation)
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("r", [0, 1, 2, 5])
@pytest.mark.parametrize("tie", ["paper", "appendix"])
def test_constant_is_fixed_point(r, tie):
    img = np.full((2, 7, 10), 0.5)
    out = oracle.filter(img, r, 4, tie=tie)["out"]
    np.testing.assert_array_equal(out, img)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_step_edges_and_corner_preserved(r):
    H, W = 24, 30
    v = np.full((H, W), 0.25)
    v[:, 13:] = 0.75  # vertical step at column 13 >= r
    h = np.full((H, W), 0.25)
    h[11:, :] = 0.75
    corner = np.full((H, W), 0.25)
    corner[10:, 12:] = 0.75  # L-shaped corner
    rect = np.full((H, W), 0.25)
    rect[5:5 + 2 * r + 3, 7:7 + 2 * r + 1] = 0.75  # rectangle of sides >= 2r
    for img in (v, h, corner, rect):
        out = oracle.filter(img, r, 6)["out"]
        np.testing.assert_array_equal(out, img)


@pytest.mark.parametrize("r,s", [(1, 2), (2, 4), (3, 7)])
def test_checkerboard_preserved(r, s):
    img = synth.checkerboard(4 * s, 5 * s, s).astype(np.float64)
    out = oracle.filter(img, r, 5)["out"]
    np.testing.assert_array_equal(out, img)


def test_box_filter_smooths_edges_but_osbf_does_not():
    """Contrast with the classical box filter (Fig. 1): a box filter blurs a step."""
    img = np.full((16, 16), 0.25)
    img[:, 8:] = 0.75
    box = ndi.uniform_filter(np.pad(img, 2, mode="edge"), size=5, mode="constant")[2:-2, 2:-2]
    assert np.abs(box - img).max() > 0.1
    np.testing.assert_array_equal(oracle.filter(img, 2, 3)["out"], img)


def test_noise_is_smoothed():
    """Sanity check (not a pin): one large rectangle plus noise gets closer to the clean scene."""
    img = synth.piecewise_stack(1, 1, 64, 64, seed=3, sigma=0.05, n_rect=1, n_tri=0)[0, 0].astype(np.float64)
    clean = synth.piecewise_stack(1, 1, 64, 64, seed=3, sigma=0.0, n_rect=1, n_tri=0)[0, 0].astype(np.float64)
    out = oracle.filter(img, 2, 10)["out"]
    assert np.sqrt(np.mean((out - clean) ** 2)) < 0.5 * np.sqrt(np.mean((img - clean) ** 2))


# ----------------------------------------------------------------------------------
# exact 8-bit rule
# ----------------------------------------------------------------------------------
def fraction_first_pass(img, r, order=(1, 2, 3, 4, 5, 6, 7, 8)):
    H, W = img.shape
    FH, FW = H + 2 * r, W + 2 * r
    U = [[int(img[min(max(fy - r, 0), H - 1)][min(max(fx - r, 0), W - 1)]) for fx in range(FW)] for fy in range(FH)]
    out = np.zeros((FH, FW), dtype=np.float32)
    mp = np.zeros((FH, FW), dtype=np.uint8)
    for y in range(FH):
        for x in range(FW):
            best, best_ad, best_i = None, None, None
            for i in order:
                s = sum(U[v][u] for v in range(max(0, y - r), min(FH, y + r + 1))
                        for u in range(max(0, x - r), min(FW, x + r + 1)) if _in_window(i, r, x, y, u, v))
                mean = Fraction(s) * _kernel_weight(i, r)
                ad = abs(mean - U[y][x])
                if best is None or ad < best_ad:
                    best, best_ad, best_i = mean, ad, i
            out[y, x] = np.float32(float(best))  # double rounding is innocuous here (53 >= 2*24+2)
            mp[y, x] = best_i
    return out, mp


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_u8_exact_rule(r):
    rng = np.random.default_rng(400 + r)
    img = rng.integers(0, 256, size=(5, 7), dtype=np.uint8)
    img[1:3, 2:5] = 17  # plateaus create exact ties
    frame, mp = oracle.u8_first_pass(img, r)
    want, want_map = fraction_first_pass(img, r)
    np.testing.assert_array_equal(frame[0].view(np.uint32), want.view(np.uint32))
    np.testing.assert_array_equal(mp[0], want_map)
    frame_a, mp_a = oracle.u8_first_pass(img, r, tie="appendix")
    want_a, want_map_a = fraction_first_pass(img, r, order=(6, 5, 7, 8, 2, 1, 3, 4))
    np.testing.assert_array_equal(frame_a[0].view(np.uint32), want_a.view(np.uint32))
    np.testing.assert_array_equal(mp_a[0], want_map_a)


def test_u8_spike():
    frame, _ = oracle.u8_first_pass(np.array([[0, 255, 0]], dtype=np.uint8), 1)
    assert oracle.crop(frame, 1)[0].tolist() == [[0.0, 127.5, 0.0]]


# ----------------------------------------------------------------------------------
# adjoint: transpose identity and finite differences
# ----------------------------------------------------------------------------------
def _frozen_apply(v, maps, r, iters):
    # hint_thresh = inf forces every selection to the given map: the frozen linear map A
    return oracle.filter(v, r, iters, hint=maps, hint_thresh=np.inf)["out"]


@pytest.mark.parametrize("r,iters", [(1, 1), (1, 3), (2, 2), (3, 2)])
def test_adjoint_transpose_identity(r, iters):
    rng = np.random.default_rng(500 + r * 10 + iters)
    x = rng.random((2, 9, 11))
    maps = oracle.filter(x, r, iters, want_maps=True)["maps"]
    v = rng.standard_normal(x.shape)
    w = rng.standard_normal(x.shape)
    Av = _frozen_apply(v, maps, r, iters)
    Atw = oracle.adjoint(w, maps, r, iters)
    assert abs(np.sum(Av * w) - np.sum(v * Atw)) < 1e-10 * (1 + abs(np.sum(Av * w)))


def test_frozen_map_is_the_filter_on_its_own_input():
    rng = np.random.default_rng(9)
    x = rng.random((1, 8, 8))
    res = oracle.filter(x, 2, 3, want_maps=True)
    np.testing.assert_allclose(_frozen_apply(x, res["maps"], 2, 3), res["out"], atol=1e-14)


def test_adjoint_finite_differences():
    """FP64 central differences on 1 x 1 x 32 x 32, r = 1, 2 passes, away from selection ties."""
    rng = np.random.default_rng(11)
    x = synth.piecewise_plane(32, 32, seed=5, sigma=0.05).astype(np.float64)
    w = rng.standard_normal((32, 32))
    r, iters, h = 1, 2, 1e-6
    base = oracle.filter(x, r, iters, want_maps=True)
    g = oracle.adjoint(w, base["maps"], r, iters)
    checked = 0
    for (y, xx) in itertools.product(range(0, 32, 3), range(0, 32, 3)):
        xp, xm = x.copy(), x.copy()
        xp[y, xx] += h
        xm[y, xx] -= h
        rp = oracle.filter(xp, r, iters, want_maps=True)
        rm = oracle.filter(xm, r, iters, want_maps=True)
        if not (np.array_equal(rp["maps"], base["maps"]) and np.array_equal(rm["maps"], base["maps"])):
            continue  # the perturbation flips a selection: not differentiable there
        fd = (np.sum(rp["out"] * w) - np.sum(rm["out"] * w)) / (2 * h)
        assert abs(fd - g[y, xx]) < 1e-6 * (1 + abs(g[y, xx]))
        checked += 1
    assert checked > 50


# ----------------------------------------------------------------------------------
# region oracle, hints, storage rounding
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("r,iters", [(1, 3), (2, 2), (3, 1)])
def test_region_matches_full(r, iters):
    x = synth.piecewise_plane(40, 37, seed=r + iters, sigma=0.05).astype(np.float64)
    full = oracle.filter(x, r, iters)["out"]
    for (y0, y1, x0, x1) in [(0, 5, 0, 7), (10, 20, 11, 30), (35, 40, 30, 37), (0, 40, 0, 37), (17, 18, 0, 1)]:
        np.testing.assert_array_equal(oracle.filter_region(x, r, iters, y0, y1, x0, x1), full[y0:y1, x0:x1])


def test_hint_with_own_maps_changes_nothing():
    x = synth.piecewise_plane(30, 30, seed=1).astype(np.float64)
    res = oracle.filter(x, 2, 3, want_maps=True)
    again = oracle.filter(x, 2, 3, hint=res["maps"], hint_thresh=1e-6)
    np.testing.assert_array_equal(again["out"], res["out"])
    assert again["n_hinted"] == 0


def test_hint_threshold_band():
    """Hinted mode adopts a recorded selection only where its |d| is within hint_thresh of
    the best |d| (the near-tie band), never elsewhere.

    On the plane u(y, x) = x + 2y the eight means of an interior pixel (windows inside the
    image) are closed forms: a window spanning column offsets a0..a1 and row offsets b0..b1
    has mean u + (a0 + a1)/2 + (b0 + b1), so d_1..d_8 = r/2, 3r/2, -r/2, -3r/2, -r/2, r/2,
    r, -r (Eq. (6)-(13)).  The best |d| = r/2 is shared by N1, N6 (+r/2) and N3, N5 (-r/2);
    Algorithm 2's first minimum in the paper order is N1, so one pass gives u + r/2."""
    r, H, W = 3, 20, 26
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = xx + 2 * yy
    FH, FW = H + 2 * r, W + 2 * r
    inner = (slice(r, H - r), slice(r, W - r))  # image pixels whose windows stay inside the image
    n_inner = (H - 2 * r) * (W - 2 * r)

    def run(window, thresh):
        hint = np.zeros((1, 1, FH, FW), dtype=np.uint8)
        hint[0, 0, 2 * r:FH - 2 * r, 2 * r:FW - 2 * r] = window  # frame coordinates of the inner pixels
        return oracle.filter(img, r, 1, hint=hint, hint_thresh=thresh)

    own = oracle.filter(img, r, 1)["out"]
    np.testing.assert_array_equal(own[inner], img[inner] + r / 2)
    # outside the band (gap r or r/2 > 1e-6): the oracle keeps its own choice
    for window in (2, 4, 7, 8):
        res = run(window, 1e-6)
        np.testing.assert_array_equal(res["out"], own)
        assert res["n_hinted"] == 0
    # inside the band (gap 0): a tied window of the other sign is adopted and counted
    for window in (3, 5):
        res = run(window, 1e-6)
        np.testing.assert_array_equal(res["out"][inner], img[inner] - r / 2)
        assert res["n_hinted"] == n_inner
    # a tied window with the same mean changes nothing and is not counted
    res = run(6, 1e-6)
    np.testing.assert_array_equal(res["out"], own)
    assert res["n_hinted"] == 0
    # the band is strict: with hint_thresh = r, N7 (gap r/2) is adopted, N2 (gap r) is not
    res = run(7, float(r))
    np.testing.assert_array_equal(res["out"][inner], img[inner] + r)
    assert res["n_hinted"] == n_inner
    res = run(2, float(r))
    np.testing.assert_array_equal(res["out"], own)
    assert res["n_hinted"] == 0
    # the region oracle applies the same band
    for window, thresh, want in ((3, 1e-6, img - r / 2), (2, 1e-6, img + r / 2), (7, float(r), img + r)):
        hint = np.zeros((1, FH, FW), dtype=np.uint8)
        hint[0, 2 * r:FH - 2 * r, 2 * r:FW - 2 * r] = window
        got, nh = oracle.filter_region(img, r, 1, r, H - r, r, W - r, hint=hint, hint_thresh=thresh,
                                       return_hinted=True)
        np.testing.assert_array_equal(got, want[inner])
        assert nh == (0 if window == 2 else n_inner)


def test_hint_threshold_band_fast_and_gauss():
    """The same band in the fast approximation's and the one-sided Gaussian filter's hinted
    modes.  On u = x + 2y, Eq. (app) gives the fast variant the exact filter's eight d_i
    (r/2, 3r/2, -r/2, -3r/2, -r/2, r/2, r, -r); the Gaussian windows give mu, 3mu, -mu,
    -3mu, -mu, mu, 2mu, -2mu with mu = sum_k w_k k the mean offset of the normalised
    one-sided Gaussian kernel w_k ~ exp(-k^2 / (2 sigma^2)), k = 0..r."""
    r, H, W, sigma = 3, 20, 26, 1.5
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = xx + 2 * yy
    FH, FW = H + 2 * r, W + 2 * r
    inner = (slice(r, H - r), slice(r, W - r))
    n_inner = (H - 2 * r) * (W - 2 * r)
    w = np.exp(-np.arange(r + 1) ** 2 / (2 * sigma**2))
    mu = float((w * np.arange(r + 1)).sum() / w.sum())

    def hint_of(window):
        h = np.zeros((1, 1, FH, FW), dtype=np.uint8)
        h[0, 0, 2 * r:FH - 2 * r, 2 * r:FW - 2 * r] = window
        return h

    own = oracle.fast_filter(img, r, 1)["out"]
    np.testing.assert_array_equal(own[inner], img[inner] + r / 2)
    for window, thresh, want, counted in ((3, 1e-6, img - r / 2, True), (2, 1e-6, own, False),
                                          (7, float(r), img + r, True), (2, float(r), own, False)):
        res = oracle.fast_filter(img, r, 1, hint=hint_of(window), hint_thresh=thresh)
        np.testing.assert_array_equal(res["out"][inner], want[inner])
        assert res["n_hinted"] == (n_inner if counted else 0)

    own = oracle.gauss_filter(img, r, 1, sigma)["out"]
    for window, thresh, want in ((3, 1e-6, img - mu), (1, 1e-6, img + mu), (7, 1.5 * mu, img + 2 * mu)):
        res = oracle.gauss_filter(img, r, 1, sigma, hint=hint_of(window), hint_thresh=thresh)
        np.testing.assert_allclose(res["out"][inner], want[inner], rtol=0, atol=1e-9)
    for window, thresh in ((2, 1e-6), (8, 1e-6), (2, 1.5 * mu)):  # gaps 2mu, mu, 2mu: outside the band
        res = oracle.gauss_filter(img, r, 1, sigma, hint=hint_of(window), hint_thresh=thresh)
        np.testing.assert_array_equal(res["out"], own)
        assert res["n_hinted"] == 0


def test_storage_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    v = np.concatenate([rng.random(20000), rng.random(2000) * 255, [0.0, 1.0, 0.5, 1 / 3, 2**-20, 2**-25]])
    # exact halfway cases between neighbouring f16 / bf16 values
    v = np.concatenate([v, (np.arange(1, 200) * 2 + 1) * 2.0**-11, (np.arange(1, 200) * 2 + 1) * 2.0**-8])
    # float32-representable values, so that torch's float32 -> 16-bit conversion is one
    # correctly rounded step (its float64 -> 16-bit path rounds through float32 first)
    v = v.astype(np.float32).astype(np.float64)
    for st, tdt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        want = torch.from_numpy(v.astype(np.float32)).to(tdt).to(torch.float64).numpy()
        np.testing.assert_array_equal(oracle.round_storage(v, st), want)
    np.testing.assert_array_equal(oracle.round_storage(v, "f32"), v.astype(np.float32).astype(np.float64))


def test_storage_rounded_filter_stays_on_grid():
    x = synth.round_to_storage(synth.piecewise_plane(20, 20, seed=2), "f16").astype(np.float64)
    out = oracle.filter(x, 2, 3, storage="f16")["out"]
    np.testing.assert_array_equal(oracle.round_storage(out, "f16"), out)


# ---------------------------------------------------------------------------------
# The fast approximation (Sec. "Fast Approximation to One-sided Box Filter",
# Algorithm 3, Eq. (app)).
# ---------------------------------------------------------------------------------
def _fast_brute(img, r, iters, tie="paper"):
    """Pure-Python restatement: replicate pad, per pass the four quadrant means taken
    directly from their pixel sets (not by shifted lookups), the half windows as the mean
    of their two quadrants, first argmin in the tie order, Jacobi update, crop."""
    H, W = len(img), len(img[0])
    FH, FW = H + 2 * r, W + 2 * r
    V = [[img[min(max(y - r, 0), H - 1)][min(max(x - r, 0), W - 1)] for x in range(FW)] for y in range(FH)]
    order = [1, 2, 3, 4, 5, 6, 7, 8] if tie == "paper" else [6, 5, 7, 8, 2, 1, 3, 4]
    quads = {1: (0, r, -r, 0), 2: (0, r, 0, r), 3: (-r, 0, 0, r), 4: (-r, 0, -r, 0)}  # rows, cols
    n = (r + 1) ** 2
    for _ in range(iters):
        nxt = [[0.0] * FW for _ in range(FH)]
        for y in range(FH):
            for x in range(FW):
                a = {}
                for k, (y0, y1, x0, x1) in quads.items():
                    s = 0.0
                    for yy in range(y + y0, y + y1 + 1):
                        for xx in range(x + x0, x + x1 + 1):
                            if 0 <= yy < FH and 0 <= xx < FW:
                                s += V[yy][xx]
                    a[k] = s / n
                a[5] = (a[4] + a[1]) / 2
                a[6] = (a[3] + a[2]) / 2
                a[7] = (a[1] + a[2]) / 2
                a[8] = (a[4] + a[3]) / 2
                u = V[y][x]
                m = order[0]
                for k in order[1:]:
                    if abs(a[k] - u) < abs(a[m] - u):
                        m = k
                nxt[y][x] = a[m]
        V = nxt
    return np.array([[V[y + r][x + r] for x in range(W)] for y in range(H)])


@pytest.mark.parametrize("r,iters,tie", [(1, 1, "paper"), (1, 3, "appendix"), (2, 2, "paper"), (3, 1, "appendix")])
def test_fast_oracle_matches_brute_force(r, iters, tie):
    rng = np.random.default_rng(100 + r * 10 + iters)
    img = rng.random((7, 9))
    got = oracle.fast_filter(img, r, iters, tie=tie)["out"]
    want = _fast_brute(img.tolist(), r, iters, tie)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("r", [1, 3])
@pytest.mark.parametrize("alpha,beta,tie,win", [
    (1, 3, "paper", 5),      # |d| = r/2 * (2, 4, 2, 4, 1, 1, 3, 3): N5 first
    (1, 3, "appendix", 6),   # N6 precedes N5 in the appendix order
    (3, 1, "paper", 7),      # |d| = r/2 * (2, 4, 2, 4, 3, 3, 1, 1): N7 first
    (3, 1, "appendix", 7),
])
def test_fast_linear_ramp_closed_form(alpha, beta, tie, win, r):
    """On U = alpha x + beta y the quadrant means are U + r/2 (-alpha + beta, alpha + beta,
    alpha - beta, -alpha - beta) (N1..N4), and Eq. (app) gives the half windows
    U + r/2 (-alpha, alpha, beta, -beta) (N5..N8) -- which, for a linear image, are also the
    exact half-window means, so the fast and the exact filter agree.  Interior pixels
    (all windows inside the image) move by the first smallest offset in the tie order; a
    wrong shift or a wrong pairing in Eq. (app) changes the offset.  Integer pixels and
    (r+1)^2 a power of two keep every candidate exact in FP64, so the ties are exact."""
    H, W = 24, 26
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = alpha * xx + beta * yy + 100.0
    off = {5: -alpha, 6: alpha, 7: beta, 8: -beta}[win] * r / 2
    for out in (oracle.fast_filter(img, r, 1, tie=tie)["out"], oracle.filter(img, r, 1, tie=tie)["out"]):
        inner = (slice(r, H - r), slice(r, W - r))
        np.testing.assert_array_equal(out[inner], img[inner] + off)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_fast_checkerboard_is_a_fixed_point(r):
    """Every pixel of a checkerboard with cells of 2r has a quadrant inside its own cell
    (|d| = 0, and quadrants precede the half windows in the paper order): corners and
    edges are preserved (the property Sec. 'Fast Approximation' keeps from the exact
    filter)."""
    c = 2 * r
    yy, xx = np.mgrid[0:5 * c, 0:4 * c]
    img = (((yy // c) + (xx // c)) % 2).astype(np.float64)
    np.testing.assert_array_equal(oracle.fast_filter(img, r, 4)["out"], img)


def test_fast_trivial_cases():
    img = np.random.default_rng(3).random((5, 6))
    np.testing.assert_array_equal(oracle.fast_filter(img, 0, 3)["out"], img)   # every window is the pixel
    np.testing.assert_array_equal(oracle.fast_filter(img, 2, 0)["out"], img)   # no pass
    flat = np.full((6, 5), 0.375)
    np.testing.assert_array_equal(oracle.fast_filter(flat, 2, 3)["out"], flat)


# ---------------------------------------------------------------------------------
# The 3D filter (Sec. "Higher Dimension Case"): eight octants, six half windows.
# ---------------------------------------------------------------------------------
def _windows3d(r):
    """Windows as explicit voxel-offset sets: O1..O4 = depth -r..0 with the 2D quadrants
    N1..N4 in (y, x), O5..O8 = depth 0..r with N1..N4, then the halves x-, x+, y+, y-, z-,
    z+ (full span on the other two axes)."""
    neg, pos, full = range(-r, 1), range(0, r + 1), range(-r, r + 1)
    quads = [(pos, neg), (pos, pos), (neg, pos), (neg, neg)]  # (y, x) of N1..N4
    wins = [(zs, ys, xs) for zs in (neg, pos) for (ys, xs) in quads]
    wins += [(full, full, neg), (full, full, pos), (full, pos, full), (full, neg, full), (neg, full, full),
             (pos, full, full)]
    return [[(dz, dy, dx) for dz in zs for dy in ys for dx in xs] for (zs, ys, xs) in wins]


def _filter3d_brute(vol, r, iters):
    D, H, W = vol.shape
    FD, FH, FW = D + 2 * r, H + 2 * r, W + 2 * r
    V = np.empty((FD, FH, FW))
    for z in range(FD):
        for y in range(FH):
            for x in range(FW):
                V[z, y, x] = vol[min(max(z - r, 0), D - 1), min(max(y - r, 0), H - 1), min(max(x - r, 0), W - 1)]
    wins = _windows3d(r)
    for _ in range(iters):
        nxt = np.empty_like(V)
        for z in range(FD):
            for y in range(FH):
                for x in range(FW):
                    best, bm = None, None
                    for offs in wins:
                        s = 0.0
                        for dz, dy, dx in offs:
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if 0 <= zz < FD and 0 <= yy < FH and 0 <= xx < FW:
                                s += V[zz, yy, xx]
                        m = s / len(offs)
                        if best is None or abs(m - V[z, y, x]) < best:
                            best, bm = abs(m - V[z, y, x]), m
                    nxt[z, y, x] = bm
        V = nxt
    return V[r:r + D, r:r + H, r:r + W]


@pytest.mark.parametrize("r,iters", [(1, 1), (1, 2), (2, 1)])
def test_filter3d_matches_brute_force(r, iters):
    vol = np.random.default_rng(7 + r + iters).random((3, 4, 5))
    np.testing.assert_allclose(oracle.filter3d(vol, r, iters)["out"], _filter3d_brute(vol, r, iters), rtol=0,
                               atol=1e-12)


@pytest.mark.parametrize("abc,off", [
    ((1, 2, 4), -1),   # octant offsets r/2 (+-1 +-2 +-4): O2 (z-, y+, x+) is the first with |.| = 1
    ((4, 2, 1), +1),   # O3 (z-, y-, x+): +4 -2 -1
    ((1, 8, 16), -1),  # octants >= 7, halves 1 / 8 / 16: H9 (x-) first
    ((16, 1, 8), +1),  # H11 (y+)
    ((8, 16, 1), -1),  # H13 (z-)
    # exact opposite-sign ties between octants: only the window order decides
    ((3, 1, 3), +1),   # O2 (z-, y+, x+) = +1 before O3 (z-, y-, x+) = -1
    ((3, 3, 1), -1),   # O1 (z-, y+, x-) = -1 before O5 (z+, y+, x-) = +1: the z- octants come first
    ((1, 3, 3), -1),   # O1 (z-, y+, x-) = -1 before O2 (z-, y+, x+) = +1
])
def test_filter3d_linear_ramp_closed_form(abc, off):
    """On U = a x + b y + c z an octant mean is U + r/2 (+-a +-b +-c) and a half window's
    U +- r/2 times one coefficient; interior voxels move by the first smallest offset in
    the window order.  Integers with r = 1 keep every mean exact in FP64 ((r+1)^3 = 8; the
    half-window quotients are correctly rounded), so the ties are exact.  The five cases
    pin the octant signs, the half windows and the order."""
    a, b, c = abc
    r, D, H, W = 1, 6, 7, 8
    zz, yy, xx = np.mgrid[0:D, 0:H, 0:W].astype(np.float64)
    vol = a * xx + b * yy + c * zz + 200.0
    out = oracle.filter3d(vol, r, 1)["out"]
    inner = (slice(r, D - r), slice(r, H - r), slice(r, W - r))
    np.testing.assert_array_equal(out[inner], vol[inner] + off * r / 2)


def test_filter3d_fixed_points():
    flat = np.full((5, 6, 7), 0.625)
    np.testing.assert_array_equal(oracle.filter3d(flat, 2, 3)["out"], flat)
    r, c = 1, 2
    zz, yy, xx = np.mgrid[0:4 * c, 0:3 * c, 0:5 * c]
    cb = (((zz // c) + (yy // c) + (xx // c)) % 2).astype(np.float64)   # every voxel owns an octant of its cell
    np.testing.assert_array_equal(oracle.filter3d(cb, r, 3)["out"], cb)
    vol = np.random.default_rng(1).random((3, 4, 5))
    np.testing.assert_array_equal(oracle.filter3d(vol, 0, 2)["out"], vol)
    np.testing.assert_array_equal(oracle.filter3d(vol, 2, 0)["out"], vol)


# ----------------------------------------------------------------------------------
# one-sided Gaussian filter (Algorithm 1, kernels of Sec. "Separable Kernels")
# ----------------------------------------------------------------------------------
def gauss_brute_force(img, r, iters, sigma):
    """Eq. (6)-(13) windows as set predicates; each window's kernel the product of a 1D
    kernel per axis, one-sided (centre included, normalised over 0..r) on an axis the
    window halves, full (normalised over -r..r) on an axis it spans; zeros outside the
    padded frame; first argmin in window order."""
    import math
    g = [math.exp(-k * k / (2.0 * sigma * sigma)) for k in range(r + 1)]
    half, full = sum(g), g[0] + 2 * sum(g[1:])
    H, W = len(img), len(img[0])
    FH, FW = H + 2 * r, W + 2 * r
    U = [[img[min(max(fy - r, 0), H - 1)][min(max(fx - r, 0), W - 1)] for fx in range(FW)] for fy in range(FH)]
    for _ in range(iters):
        new = [[0.0] * FW for _ in range(FH)]
        for y in range(FH):
            for x in range(FW):
                best, best_ad = None, None
                for i in range(1, 9):
                    # an axis is spanned when the window holds the taps on both sides of the centre
                    xfull = _in_window(i, r, x, y, x - 1, y) and _in_window(i, r, x, y, x + 1, y)
                    yfull = _in_window(i, r, x, y, x, y - 1) and _in_window(i, r, x, y, x, y + 1)
                    s = 0.0
                    for v in range(y - r, y + r + 1):
                        for u in range(x - r, x + r + 1):
                            if 0 <= v < FH and 0 <= u < FW and _in_window(i, r, x, y, u, v):
                                wy = g[abs(v - y)] / (full if yfull else half)
                                wx = g[abs(u - x)] / (full if xfull else half)
                                s += wy * wx * U[v][u]
                    ad = abs(s - U[y][x])
                    if best is None or ad < best_ad:
                        best, best_ad = s, ad
                new[y][x] = best
        U = new
    return np.array([row[r:r + W] for row in U[r:r + H]])


@pytest.mark.parametrize("r,iters,sigma", [(1, 1, 0.8), (1, 2, 3.0), (2, 2, 1.7), (3, 1, 1.0)])
def test_gauss_oracle_matches_brute_force(r, iters, sigma):
    img = np.random.default_rng(40 + r).random((6, 7))
    got = oracle.gauss_filter(img, r, iters, sigma)["out"]
    np.testing.assert_allclose(got, gauss_brute_force(img.tolist(), r, iters, sigma), rtol=0, atol=1e-12)


@pytest.mark.parametrize("r", [1, 2, 5])
def test_gauss_large_sigma_is_the_box_filter(r):
    # sigma = +inf turns every weight flat: the one-sided box filter (Sec. 4 opening)
    img = synth.piecewise_stack(1, 2, 19, 23, seed=7 + r)[0].astype(np.float64)
    a = oracle.gauss_filter(img, r, 3, 1e12, want_maps=True)
    b = oracle.filter(img, r, 3, want_maps=True)
    np.testing.assert_allclose(a["out"], b["out"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(a["maps"], b["maps"])


def _scipy_kernels(r, sigma):
    """Full and one-sided 1D kernels taken from scipy's Gaussian: the impulse response of
    gaussian_filter1d truncated at radius r, and its centre-and-right half renormalised."""
    e = np.zeros(2 * r + 1)
    e[r] = 1.0
    full = ndi.gaussian_filter1d(e, sigma, truncate=r / sigma, mode="constant")   # taps -r..r
    half = full[r:] / full[r:].sum()                                               # taps 0..r
    return full, half


def _one_sided_1d(s, half, side):
    # side -1: sum_k half[k] s(x - k); side +1: sum_k half[k] s(x + k); zeros off the ends
    r = len(half) - 1
    p = np.concatenate([np.zeros(r), s, np.zeros(r)])
    n = len(s)
    return sum(half[k] * p[r + side * k: r + side * k + n] for k in range(r + 1))


@pytest.mark.parametrize("r,sigma", [(2, 1.0), (3, 3.0), (5, 1.6)])
@pytest.mark.parametrize("axis", [0, 1])
def test_gauss_one_axis_signal_against_scipy(r, sigma, axis):
    """An image varying along one axis only: away from the frame's ends on the other axis,
    every window mean is a 1D one-sided (k^-, k^+) or full (k) Gaussian mean of the signal,
    scipy's gaussian_filter1d for the full one (Eq. (oneside))."""
    full, half = _scipy_kernels(r, sigma)
    s = np.random.default_rng(r + 10 * axis).random(17)
    img = np.tile(s, (12, 1)) if axis == 1 else np.tile(s[:, None], (1, 12))
    out = oracle.gauss_filter(img, r, 1, sigma)["out"]
    sp = np.pad(s, r, mode="edge")                     # the frame along the signal's axis
    cand_lo = _one_sided_1d(sp, half, -1)[r:-r]        # x - r..x (or y - r..y)
    cand_hi = _one_sided_1d(sp, half, +1)[r:-r]
    cand_f = ndi.gaussian_filter1d(sp, sigma, truncate=r / sigma, mode="constant")[r:-r]
    # window order 1..8 along x: lo, hi, hi, lo, lo, hi, full, full; along y: hi, hi, lo,
    # lo, full, full, hi, lo -- the first argmin is the first of lo / hi / full to win
    first = [cand_lo, cand_hi, cand_f] if axis == 1 else [cand_hi, cand_lo, cand_f]
    ad = np.stack([np.abs(c - s) for c in first])
    exp1d = np.stack(first)[np.argmin(ad, axis=0), np.arange(len(s))]
    # rows (or columns) whose windows stay inside the frame on the constant axis
    inner = out[r:12 - r, :] if axis == 1 else out[:, r:12 - r].T
    for line in inner:
        np.testing.assert_allclose(line, exp1d, rtol=0, atol=1e-12)


@pytest.mark.parametrize("r,sigma", [(2, 1.2), (4, 3.0)])
def test_gauss_additive_image_products(r, sigma):
    """f(y, x) = a(y) + b(x): with normalised product kernels each window mean splits
    into a y-mean of a plus an x-mean of b, the halves set by Eq. (6)-(13)."""
    full, half = _scipy_kernels(r, sigma)
    rng = np.random.default_rng(5)
    H, W = 14, 15
    a, b = rng.random(H), rng.random(W)
    img = a[:, None] + b[None, :]
    out = oracle.gauss_filter(img, r, 1, sigma)["out"]
    ap, bp = np.pad(a, r, mode="edge"), np.pad(b, r, mode="edge")
    ya = {"lo": _one_sided_1d(ap, half, -1), "hi": _one_sided_1d(ap, half, +1),
          "f": ndi.gaussian_filter1d(ap, sigma, truncate=r / sigma, mode="constant")}
    xb = {"lo": _one_sided_1d(bp, half, -1), "hi": _one_sided_1d(bp, half, +1),
          "f": ndi.gaussian_filter1d(bp, sigma, truncate=r / sigma, mode="constant")}
    # (y part, x part) of N1..N8, y growing downwards
    parts = [("hi", "lo"), ("hi", "hi"), ("lo", "hi"), ("lo", "lo"), ("f", "lo"), ("f", "hi"), ("hi", "f"), ("lo", "f")]
    for y in range(r, H - r):            # frame rows 2r.., windows inside the frame
        for x in range(r, W - r):
            fy, fx = y + r, x + r
            means = [ya[py][fy] + xb[px][fx] for py, px in parts]
            ad = [abs(m - img[y, x]) for m in means]
            assert abs(out[y, x] - means[int(np.argmin(ad))]) < 1e-12


def test_gauss_constant_interior_and_trivial_cases():
    flat = np.full((9, 10), 0.375)
    out = oracle.gauss_filter(flat, 2, 1, 1.3)["out"]
    np.testing.assert_allclose(out[2:-2, 2:-2], flat[2:-2, 2:-2], rtol=0, atol=1e-15)
    img = np.random.default_rng(3).random((5, 6))
    np.testing.assert_array_equal(oracle.gauss_filter(img, 0, 3, 1.0)["out"], img)
    np.testing.assert_array_equal(oracle.gauss_filter(img, 2, 0, 1.0)["out"], img)


def test_gauss_hint_with_own_maps_changes_nothing():
    img = synth.piecewise_stack(1, 2, 23, 31, seed=12)[0].astype(np.float64)
    a = oracle.gauss_filter(img, 3, 3, 1.7, want_maps=True)
    b = oracle.gauss_filter(img, 3, 3, 1.7, hint=a["maps"], hint_thresh=1e-6)
    np.testing.assert_array_equal(a["out"], b["out"])
    assert b["n_hinted"] == 0


@pytest.mark.parametrize("r", [1, 2, 4])
def test_gauss_patch_gives_the_frame_value(r):
    """One pass at a frame pixel depends only on the (2r+1)^2 patch around it, zeros
    outside the frame: the sampled full-size GPU checks rest on this."""
    img = np.random.default_rng(r).random((13, 17))
    frame = np.pad(img, r, mode="edge")
    full = oracle.gauss_iterate_frame(frame, r, 1, 1.3)
    FH, FW = frame.shape
    zf = np.pad(frame, r)  # zeros beyond the frame
    for y in range(FH):
        for x in range(FW):
            patch = zf[y:y + 2 * r + 1, x:x + 2 * r + 1]
            assert oracle.gauss_iterate_frame(patch, r, 1, 1.3)[r, r] == full[y, x]
