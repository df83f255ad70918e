"""Pins of the oracle's local minimum / maximum (Sec. 3.4: extrema kept
recursively with deques) and of Bernsen's midrange decision built on them.

* The deque route (separable, Theta(HW)) equals the direct definition on
  random tiny images, windows larger than the image and even windows.
* scipy.ndimage's minimum/maximum filters (constant border 255 / 0, which
  cannot win a min / max, with the origin that places Algorithm 1's window)
  give the same extrema.
* Transposing the image and swapping h, w transposes the result.
* Bernsen closed cases: flat images, the 0/255 checkerboard, contrast limits
  0 and 256, and the midrange rule in integers on hand-made 1 x 3 windows.
"""
import numpy as np
import pytest

import oracle
import synth


def tiny_cases(count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        H = int(rng.integers(1, 24))
        W = int(rng.integers(1, 24))
        h = int(rng.integers(1, 2 * max(H, W) + 4))
        w = int(rng.integers(1, 2 * max(H, W) + 4))
        pitch = W + int(rng.integers(0, 5))
        img = rng.integers(0, 256, size=(H, pitch), dtype=np.uint8)
        yield img, H, W, h, w


def test_deque_equals_definition():
    for img, H, W, h, w in tiny_cases(300, 11):
        a = oracle.window_minmax(img, h, w, W=W)
        b = oracle.window_minmax(img, h, w, route="bruteforce", W=W)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("h,w", [(1, 1), (2, 3), (3, 2), (8, 8), (15, 15), (31, 9), (64, 64), (101, 101)])
def test_extrema_match_scipy_filters(h, w):
    ndimage = pytest.importorskip("scipy.ndimage")
    img = synth.document(90, 130, h * 1000 + w, salt_pepper=0.01)
    mn, mx = oracle.window_minmax(img, h, w)
    l, o = (w + 1) // 2, (h + 1) // 2
    # scipy's window starts at -(size // 2) - origin; Algorithm 1's at -(l - 1)
    origin = (o - 1 - h // 2, l - 1 - w // 2)
    np.testing.assert_array_equal(
        mn, ndimage.minimum_filter(img, size=(h, w), mode="constant", cval=255, origin=origin))
    np.testing.assert_array_equal(
        mx, ndimage.maximum_filter(img, size=(h, w), mode="constant", cval=0, origin=origin))


def test_extrema_contain_the_centre_and_are_monotone_in_the_window():
    img = synth.document(60, 70, 3)
    mn3, mx3 = oracle.window_minmax(img, 3, 3)
    mn9, mx9 = oracle.window_minmax(img, 9, 9)  # the 9x9 window holds the 3x3 one (odd sizes)
    assert (mn3 <= img).all() and (img <= mx3).all()
    assert (mn9 <= mn3).all() and (mx9 >= mx3).all()


def test_transpose_swaps_h_and_w():
    img = synth.document(41, 57, 8)
    for h, w in [(5, 9), (12, 3), (33, 60)]:
        mn, mx = oracle.window_minmax(img, h, w)
        tmn, tmx = oracle.window_minmax(np.ascontiguousarray(img.T), w, h)
        np.testing.assert_array_equal(mn, tmn.T)
        np.testing.assert_array_equal(mx, tmx.T)


def test_bernsen_flat_images_are_one_class():
    for val, expect in [(0, 0), (100, 0), (127, 0), (128, 1), (200, 1), (255, 1)]:
        img = np.full((9, 11), val, np.uint8)
        bits, _ = oracle.binarize_bernsen(img, 3, 3, 15)
        assert (bits == expect).all(), val  # mn + mx = 2*val <= 255 is dark


def test_bernsen_checkerboard_and_limits():
    i, j = np.indices((16, 20))
    img = np.where((i + j) % 2 == 0, 0, 255).astype(np.uint8)
    bits, _ = oracle.binarize_bernsen(img, 3, 3, 15)  # contrast 255: midrange 127.5
    np.testing.assert_array_equal(bits, (img == 255).astype(np.uint8))
    # limit 256: no window reaches it, every window is one class
    doc = synth.document(50, 64, 2)
    mn, mx = oracle.window_minmax(doc, 7, 7)
    bits, _ = oracle.binarize_bernsen(doc, 7, 7, 256)
    np.testing.assert_array_equal(bits, (mn.astype(int) + mx > 255).astype(np.uint8))
    # limit 0: the midrange rule everywhere
    bits, _ = oracle.binarize_bernsen(doc, 7, 7, 0)
    np.testing.assert_array_equal(bits, (2 * doc.astype(int) > mn.astype(int) + mx).astype(np.uint8))


def test_bernsen_midrange_ties_in_integers():
    # 1 x 3 windows on one row: centre 10 with extrema 10, 11 -> 2*10 <= 21: dark;
    # centre 11 with extrema 10, 11 -> 22 > 21: bright; the exact tie
    # 2I = mn + mx (centre 20 between 10 and 30) is dark
    img = np.array([[10, 10, 11, 11, 30, 20, 10]], np.uint8)
    bits, _ = oracle.binarize_bernsen(img, 1, 3, 0)
    mn, mx = oracle.window_minmax(img, 1, 3)
    np.testing.assert_array_equal(mn[0], [10, 10, 10, 11, 11, 10, 10])
    np.testing.assert_array_equal(mx[0], [10, 11, 11, 30, 30, 30, 20])
    np.testing.assert_array_equal(bits[0], [0, 0, 1, 0, 1, 0, 0])


def test_minmax_at_matches_full():
    img = synth.document(80, 90, 12)
    mn, mx = oracle.window_minmax(img, 15, 21)
    rng = np.random.default_rng(4)
    ii = rng.integers(0, 80, 200)
    jj = rng.integers(0, 90, 200)
    smn, smx = oracle.window_minmax_at(img, 15, 21, ii, jj)
    np.testing.assert_array_equal(smn, mn[ii, jj])
    np.testing.assert_array_equal(smx, mx[ii, jj])
