"""Pins of the FP64 edge-map oracle (Sec. 2.1) against closed forms, scipy and torch."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import synth
from oracle import edge as oe

DYADIC = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def test_taps_sum_to_one_and_match_scipy_kernel():
    w = oe.blur_taps(1.0)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.array_equal(w, w[::-1])
    delta = np.zeros(11)
    delta[5] = 1.0
    ref = ndi.gaussian_filter1d(delta, 1.0, truncate=2.0, mode="constant")[3:8]
    np.testing.assert_allclose(w, ref, rtol=1e-14, atol=0)


def test_blur_and_sobel_match_scipy_on_the_extended_image():
    rgb = synth.image(37, 53, 1234)
    y = oe.gray(rgb)
    out = oe.edge_map_gray(y)
    # border reading: clamp-extend once, then blur and Sobel without a second clamp
    ext = np.pad(y, 3, mode="edge")
    b = ndi.gaussian_filter(ext, 1.0, truncate=2.0, mode="nearest")
    gx = ndi.sobel(b, axis=1, mode="nearest")[3:-3, 3:-3]
    gy = ndi.sobel(b, axis=0, mode="nearest")[3:-3, 3:-3]
    np.testing.assert_allclose(out["blur"], b[3:-3, 3:-3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["gx"], gx, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["gy"], gy, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["M"], np.hypot(gx, gy), rtol=0, atol=1e-13)


def test_gray_is_luma_over_255():
    rgb = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [10, 20, 30]]], dtype=np.uint8)
    np.testing.assert_allclose(oe.gray(rgb)[0], [0.299, 0.587, 0.114, (2.99 + 11.74 + 3.42) / 255],
                               rtol=1e-14)


def test_constant_image_gives_exactly_zero():
    rgb = np.full((40, 60, 3), 137, dtype=np.uint8)
    out = oe.edge_map(rgb)
    assert out["median"] == 0.0
    assert not out["keep"].any()
    assert np.all(out["E"] == 0.0)
    assert np.all(out["M"] == 0.0)


@pytest.mark.parametrize("dark_left", [True, False])
def test_ideal_step_gives_one_pixel_line_on_the_dark_side(dark_left):
    h, w, c = 20, 24, 11
    lo, hi = 0.25, 0.75
    y = np.where(np.arange(w)[None, :] < c, lo if dark_left else hi, hi if dark_left else lo)
    y = np.repeat(y, h, axis=0).astype(np.float64)
    out = oe.edge_map_gray(y, DYADIC)
    expected_col = c - 1 if dark_left else c
    keep = out["keep"]
    assert keep.sum() == h
    assert np.all(keep[:, expected_col])
    # the two pixels either side of the step tie exactly with dyadic taps
    assert out["M"][0, c - 1] == out["M"][0, c]
    # the same image transposed gives one row
    out_t = oe.edge_map_gray(y.T.copy(), DYADIC)
    assert out_t["keep"].sum() == h and np.all(out_t["keep"][expected_col, :])
    # E is 1 on the line (every kept value equals the median)
    assert np.allclose(out["E"][keep], 1.0)


def test_step_with_gaussian_taps_single_line_and_near_tie():
    h, w, c = 16, 30, 15
    y = np.repeat(np.where(np.arange(w)[None, :] < c, 0.2, 0.9), h, axis=0)
    out = oe.edge_map_gray(y)
    keep = out["keep"]
    assert keep.sum() == h
    cols = np.nonzero(keep[0])[0]
    assert len(cols) == 1 and cols[0] in (c - 1, c)
    assert abs(out["M"][0, c - 1] - out["M"][0, c]) <= 1e-12 * out["M"][0, c]


def test_linear_ramp_interior_magnitude_and_full_suppression():
    # dyadic slope and taps: every value is exact, so the interior ties are exact
    a = 1.0 / 64.0
    h, w = 18, 40
    y = np.repeat((a * np.arange(w))[None, :], h, axis=0)
    out = oe.edge_map_gray(y, DYADIC)
    assert np.all(out["M"][:, 3:-3] == 8.0 * a)
    # pixels whose compared neighbours both sit on the plateau are suppressed;
    # column 3 starts the plateau (its downhill neighbour saw the border:
    # M = 4 (B(3) - B(1)) = 7.75 a) and is the only one kept
    assert out["M"][0, 2] == 7.75 * a
    assert not out["keep"][:, 4:].any() and not out["keep"][:, :3].any()
    assert out["keep"][:, 3].all()
    # sigma = 1 taps: M = 8a up to rounding, and anything kept is a near-tie
    a = 0.013
    y = np.repeat((a * np.arange(w))[None, :], h, axis=0)
    out = oe.edge_map_gray(y)
    np.testing.assert_allclose(out["M"][:, 3:-3], 8.0 * a, rtol=1e-12)
    assert not (out["keep"][:, 4:-3] & ~oe.nms_exempt(out)[:, 4:-3]).any()


def test_rotation_equivariance():
    rgb = synth.image(45, 61, 77)
    out = oe.edge_map(rgb)
    rot = oe.edge_map(np.ascontiguousarray(np.rot90(rgb)))
    np.testing.assert_allclose(rot["M"], np.rot90(out["M"]), rtol=1e-12, atol=1e-14)
    ex = np.rot90(oe.nms_exempt(out)) | oe.nms_exempt(rot)
    diff = (rot["keep"] != np.rot90(out["keep"])) & ~ex
    assert diff.sum() == 0
    np.testing.assert_allclose(rot["median"], out["median"], rtol=1e-12)
    both = rot["keep"] & np.rot90(out["keep"])
    np.testing.assert_allclose(rot["E"][both], np.rot90(out["E"])[both], rtol=1e-12)


def _nms_loop(m, gx, gy):
    """Independent NMS by angle: sector = nearest multiple of 45 degrees."""
    h, w = m.shape
    keep = np.zeros_like(m, dtype=bool)
    boundary = np.zeros_like(keep)
    for yy in range(h):
        for xx in range(w):
            if m[yy, xx] <= 0:
                continue
            ang = math.degrees(math.atan2(gy[yy, xx], gx[yy, xx]))
            k = ang / 45.0
            if abs(abs(k - math.floor(k)) - 0.5) < 1e-9:
                boundary[yy, xx] = True
            s = int(math.floor(k + 0.5)) % 8
            dx, dy = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)][s]

            def mag(x2, y2):
                return m[y2, x2] if 0 <= x2 < w and 0 <= y2 < h else 0.0

            keep[yy, xx] = m[yy, xx] >= mag(xx + dx, yy + dy) and m[yy, xx] > mag(xx - dx, yy - dy)
    return keep, boundary


def test_nms_matches_angle_based_loop():
    rgb = synth.image(33, 29, 4321)
    out = oe.edge_map(rgb)
    keep, boundary = _nms_loop(out["M"], out["gx"], out["gy"])
    diff = (keep != out["keep"]) & ~boundary
    assert diff.sum() == 0
    assert out["keep"].sum() > 50


@pytest.mark.parametrize("n", [1, 2, 7, 8, 1000, 1001])
def test_lower_median_matches_torch_median(n):
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(n).uniform(0.1, 5.0, n)
    assert oe.lower_median(v) == float(torch.median(torch.from_numpy(v)))
    assert oe.lower_median(v) == np.sort(v)[(n - 1) // 2]


def test_median_normalisation():
    rgb = synth.image(64, 80, 1000)
    out = oe.edge_map(rgb)
    kept = out["M"][out["keep"]]
    assert out["median"] == np.sort(kept)[(kept.size - 1) // 2]
    np.testing.assert_allclose(out["E"][out["keep"]], kept / out["median"], rtol=1e-15)
    assert np.all(out["E"][~out["keep"]] == 0.0)
    # half of the kept pixels (rounded up) are <= 1 after normalisation
    assert (out["E"][out["keep"]] <= 1.0).sum() == (kept.size - 1) // 2 + 1 + \
        int((np.sort(kept) == out["median"]).sum() - 1)
