"""Pins of the oracle's Haar-like window sums (separable piecewise-constant
weights over Algorithm 1's window; Sec. 3.4's remark that the recursive sums
replace integral images for Haar-like features).

* The integral-image route (Viola and Jones: four lookups per rectangle)
  equals the direct definition on random tiny images, windows larger than
  the image, even sizes and up to four segments per direction.
* One segment of weight 1 in both directions is the window sum S1 of the
  pinned sums oracle.
* Linearity in the image (exact integers), and in the weights.
* Zero-mean profiles give 0 on a constant image away from the border.
* Transposing the image swaps the row and column profiles.
* A hand-computed two-rectangle value on a 4 x 4 image.
"""
import numpy as np
import pytest

import oracle
import synth

FEATURES = {
    "edge_h": ([(6, 1)], [(4, 1), (4, -1)]),
    "edge_v": ([(3, 1), (3, -1)], [(9, 1)]),
    "line_h": ([(5, 1)], [(3, -1), (3, 2), (3, -1)]),
    "line_v": ([(4, -1), (4, 2), (4, -1)], [(7, 1)]),
    "diag": ([(3, 1), (3, -1)], [(5, 1), (5, -1)]),
}


def random_profile(rng, total_max):
    n = int(rng.integers(1, 5))
    return [(int(rng.integers(1, total_max // n + 2)), int(rng.integers(-8, 9))) for _ in range(n)]


def test_integral_equals_definition():
    rng = np.random.default_rng(21)
    for _ in range(200):
        H, W = int(rng.integers(1, 20)), int(rng.integers(1, 20))
        pitch = W + int(rng.integers(0, 4))
        img = rng.integers(0, 256, size=(H, pitch), dtype=np.uint8)
        rows, cols = random_profile(rng, 2 * H + 3), random_profile(rng, 2 * W + 3)
        a = oracle.haar(img, rows, cols, W=W)
        b = oracle.haar(img, rows, cols, route="bruteforce", W=W)
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("h,w", [(1, 1), (7, 5), (8, 8), (31, 31), (64, 3)])
def test_single_box_is_the_window_sum(h, w):
    img = synth.document(50, 70, h * 100 + w)
    S1, _, _ = oracle.window_sums(img, h, w)
    np.testing.assert_array_equal(oracle.haar(img, [(h, 1)], [(w, 1)]), S1.astype(np.int32))


@pytest.mark.parametrize("name", list(FEATURES))
def test_linearity(name):
    rows, cols = FEATURES[name]
    a = synth.document(40, 60, 1) // 2
    b = synth.document(40, 60, 2) // 3
    fa, fb = oracle.haar(a, rows, cols), oracle.haar(b, rows, cols)
    np.testing.assert_array_equal(oracle.haar((a + b).astype(np.uint8), rows, cols), fa + fb)
    rows3 = [(n, 3 * wt) for n, wt in rows]
    np.testing.assert_array_equal(oracle.haar(a, rows3, cols), 3 * fa)


@pytest.mark.parametrize("name", list(FEATURES))
def test_zero_mean_profiles_vanish_on_flat_interior(name):
    rows, cols = FEATURES[name]
    h, w = sum(n for n, _ in rows), sum(n for n, _ in cols)
    img = np.full((60, 70), 173, np.uint8)
    f = oracle.haar(img, rows, cols)
    o, l = (h + 1) // 2, (w + 1) // 2
    inner = f[o: 60 - h, l: 70 - w]
    assert inner.size and (inner == 0).all()


@pytest.mark.parametrize("name", list(FEATURES))
def test_transpose_swaps_profiles(name):
    rows, cols = FEATURES[name]
    img = synth.document(33, 47, 5)
    f = oracle.haar(img, rows, cols)
    ft = oracle.haar(np.ascontiguousarray(img.T), cols, rows)
    np.testing.assert_array_equal(f, ft.T)


def test_hand_computed_two_rectangle():
    img = np.array([[1, 2, 3, 4],
                    [5, 6, 7, 8],
                    [9, 10, 11, 12],
                    [13, 14, 15, 16]], np.uint8)
    # window 2 x 2 at (1, 1): rows (1-1, 1+1] = {1, 2}, columns {1, 2};
    # left column minus right column: (6 + 10) - (7 + 11) = -2
    f = oracle.haar(img, [(2, 1)], [(1, 1), (1, -1)])
    assert f[1, 1] == -2
    # at (0, 0) the window covers rows {0, 1}, columns {0, 1}: (1 + 5) - (2 + 6)
    assert f[0, 0] == -2
    # at (3, 3) it covers row 3 and 4 (outside), columns 3 and 4 (outside): 16 - 0
    assert f[3, 3] == 16
