"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* Sec. 4 (experiment): the definitive, integral-image and recursive
  implementations produce identical results -> three independent sum routes
  must agree bit for bit on random images, windows and borders.
* Closed forms of the Sec. 1 definitions: constant images, 1x1 windows,
  windows covering the whole image (numpy global sums), the all-255 bounds of
  Sec. 3.3, a hand-worked 3x3 example and the 0/255 checkerboard (golden
  files under tests/golden/).
* Sec. 3.3 axis exchange: transposing the image and swapping h, w transposes
  every result.
* Sec. 3.2 square-root-free condition and an exact 128-bit integer decision
  of I <= t for rational k, R; a high-precision (Decimal) evaluation of the
  Sec. 1 formula bounds the FP64 threshold error.
* Sec. 3.4 quantiles: sort, 256-bin count and sliding histogram agree;
  numpy window min/max give the q = 0 and q = 1 ends.
"""
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (x.strip() for x in line.split("=", 1))
            vals[k] = v
    return vals


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


# ---------------------------------------------------------------- window sums
def test_window_params_match_algorithm1():
    # Algorithm 1: l = floor((w+1)/2), r = floor(w/2), o = floor((h+1)/2), u = floor(h/2)
    assert oracle.window_params(31, 31) == (16, 15, 16, 15)
    assert oracle.window_params(32, 32) == (16, 16, 16, 16)
    assert oracle.window_params(1, 1) == (1, 0, 1, 0)
    assert oracle.window_params(2, 5) == (3, 2, 1, 1)


def test_three_routes_agree_random_tiny():
    for img, H, W, h, w in tiny_cases(400, 1):
        a = oracle.window_sums(img, h, w, "bruteforce", W=W)
        b = oracle.window_sums(img, h, w, "integral", W=W)
        c = oracle.window_sums(img, h, w, "recursive", W=W)
        for x, y, z in zip(a, b, c):
            np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(x, z)


def test_three_routes_agree_document():
    img = synth.document(97, 131, 5, stains=2)
    for h, w in [(15, 15), (32, 32), (31, 127), (255, 7), (1, 1), (2, 3)]:
        a = oracle.window_sums(img, h, w, "bruteforce")
        c = oracle.window_sums(img, h, w, "recursive")
        b = oracle.window_sums(img, h, w, "integral")
        for x, y, z in zip(a, b, c):
            np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(x, z)


def test_count_is_sum_of_ones_and_clipped_area():
    for _, H, W, h, w in tiny_cases(100, 2):
        ones = np.ones((H, W), np.uint8)
        S1, S2, n = oracle.window_sums(ones, h, w)
        np.testing.assert_array_equal(S1, n)
        np.testing.assert_array_equal(S2, n)
        # clipped area from interval intersections (Sec. 1 window, clipped)
        l, r, o, u = oracle.window_params(h, w)
        ii = np.arange(H)[:, None]
        jj = np.arange(W)[None, :]
        rows = np.minimum(ii + u, H - 1) - np.maximum(ii - o + 1, 0) + 1
        cols = np.minimum(jj + r, W - 1) - np.maximum(jj - l + 1, 0) + 1
        np.testing.assert_array_equal(n, rows * cols)


def test_constant_image_closed_form():
    for c in (0, 1, 77, 255):
        img = np.full((20, 33), c, np.uint8)
        S1, S2, n = oracle.window_sums(img, 7, 12)
        np.testing.assert_array_equal(S1, c * n.astype(np.uint64))
        np.testing.assert_array_equal(S2, c * c * n.astype(np.uint64))
        bits_s, _ = oracle.sauvola(img, 7, 12, k=0.5)
        bits_n, _ = oracle.niblack(img, 7, 12, k=-0.2)
        # s = 0 -> Sauvola t = m (1-k) = c/2: c <= c/2 only for c = 0
        assert (bits_s == (1 if c > 0 else 0)).all()
        # Niblack t = m = c: I = c <= t everywhere (tie resolves to 0)
        assert (bits_n == 0).all()


def test_unit_window():
    img = synth.uniform(13, 17, 3)
    S1, S2, n = oracle.window_sums(img, 1, 1)
    np.testing.assert_array_equal(S1, img)
    np.testing.assert_array_equal(S2, img.astype(np.uint64) ** 2)
    assert (n == 1).all()
    bits, _ = oracle.sauvola(img, 1, 1, k=0.5)
    np.testing.assert_array_equal(bits, (img != 0).astype(np.uint8))  # t = I(1-k)
    bits, _ = oracle.niblack(img, 1, 1, k=-0.2)
    assert (bits == 0).all()  # t = I


def test_window_covering_image_uses_global_statistics():
    img = synth.uniform(9, 14, 4)
    S1, S2, n = oracle.window_sums(img, 2 * 9 + 1, 2 * 14 + 1)
    assert (S1 == int(img.astype(np.int64).sum())).all()
    assert (S2 == int((img.astype(np.int64) ** 2).sum())).all()
    assert (n == 9 * 14).all()


def test_golden_worked_example():
    g = read_golden("worked_3x3.txt")
    img = np.array([int(x) for x in g["image"].split()], np.uint8).reshape(3, 3)
    h, w = int(g["h"]), int(g["w"])
    S1, S2, n = oracle.window_sums(img, h, w, "recursive")
    t = oracle.threshold(oracle.SAUVOLA, S1, S2, n, 0.5, 128.0)
    bits, _ = oracle.sauvola(img, h, w, k=0.5)
    for name, (i, j) in {"centre": (1, 1), "corner": (0, 0), "edge": (0, 1)}.items():
        assert S1[i, j] == int(g[f"{name}_S1"])
        assert S2[i, j] == int(g[f"{name}_S2"])
        assert n[i, j] == int(g[f"{name}_n"])
        V = int(n[i, j]) * int(S2[i, j]) - int(S1[i, j]) ** 2
        assert V == int(g[f"{name}_V"])
        assert abs(t[i, j] - float(g[f"{name}_t"])) <= 1e-12 * float(g[f"{name}_t"])
        assert bits[i, j] == int(g[f"{name}_bit"])


def test_golden_checkerboard():
    g = read_golden("checkerboard.txt")
    ii, jj = np.indices((10, 12))
    img = (((ii + jj) & 1) * 255).astype(np.uint8)
    S1, S2, n = oracle.window_sums(img, 2, 2)
    inner = (slice(0, 9), slice(0, 11))  # windows fully inside
    assert (S1[inner] == int(g["interior_S1"])).all()
    assert (S2[inner] == int(g["interior_S2"])).all()
    assert (n[inner] == int(g["interior_n"])).all()
    t_s = oracle.threshold(oracle.SAUVOLA, S1, S2, n, 0.5, 128.0)
    t_n = oracle.threshold(oracle.NIBLACK, S1, S2, n, -0.2, 128.0)
    assert (t_s[inner] == float(g["sauvola_t"])).all()
    assert np.allclose(t_n[inner], float(g["niblack_t"]), rtol=0, atol=1e-12)
    bits, _ = oracle.sauvola(img, 2, 2, k=0.5)
    np.testing.assert_array_equal(bits[inner], (img[inner] == 255).astype(np.uint8))


def test_golden_overflow_bounds():
    g = read_golden("bounds.txt")
    img = np.full((300, 300), 255, np.uint8)
    S1, S2, n = oracle.window_sums(img, 255, 255)
    assert S1[150, 150] == int(g["S1_255"])
    assert S2[150, 150] == int(g["S2_255"])
    assert n[150, 150] == int(g["n_255"])
    S1, S2, n = oracle.window_sums(img, 257, 1)
    assert S1[150, 150] == int(g["C_257"]) and S2[150, 150] == int(g["D_257"])
    big = np.full((520, 520), 255, np.uint8)
    a = oracle.window_sums_at(big, 511, 511, [260], [260])
    assert a[1][0] == int(g["S2_511"]) and a[2][0] == int(g["n_511"])


def test_transpose_invariance():
    # Sec. 3.3: the method may run on the transposed image with h and w swapped.
    # Odd windows only: an even window extends down/right of its centre, which
    # transposition maps to down/right again, so odd and even both hold; test both.
    img = synth.document(41, 57, 8, stains=1)
    for h, w in [(7, 19), (8, 5), (31, 31), (1, 60)]:
        a = oracle.window_sums(img, h, w)
        b = oracle.window_sums(np.ascontiguousarray(img.T), w, h)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y.T)
        ba, _ = oracle.sauvola(img, h, w, k=0.5)
        bb, _ = oracle.sauvola(np.ascontiguousarray(img.T), w, h, k=0.5)
        np.testing.assert_array_equal(ba, bb.T)


def test_parallel_oracle_matches_sequential():
    img = synth.document(203, 150, 9, stains=2)
    for h, w in [(15, 15), (64, 9), (255, 255)]:
        _, packed = oracle.sauvola(img, h, w)
        for nt in (1, 3, 7):
            np.testing.assert_array_equal(oracle.binarize_parallel(oracle.SAUVOLA, img, h, w, 0.5, 128.0,
                                                                   threads=nt), packed)


# ---------------------------------------------------------------- thresholds
def test_fp64_threshold_within_rounding_of_exact_formula():
    getcontext().prec = 50
    img = synth.document(60, 70, 10, stains=1)
    S1, S2, n = oracle.window_sums(img, 15, 15)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, S1.size, 300)
    for method, k in ((oracle.SAUVOLA, 0.5), (oracle.NIBLACK, -0.2), (oracle.SAUVOLA, 0.2)):
        t = oracle.threshold(method, S1.ravel()[idx], S2.ravel()[idx], n.ravel()[idx], k, 128.0)
        for q, p in enumerate(idx):
            s1, s2, nn = int(S1.ravel()[p]), int(S2.ravel()[p]), int(n.ravel()[p])
            m = Decimal(s1) / nn
            s = (Decimal(s2) / nn - m * m).sqrt()  # Sec. 1 definition of s
            kk = Decimal(repr(k))
            te = m * (1 + kk * (s / 128 - 1)) if method == oracle.SAUVOLA else m + kk * s
            assert abs(Decimal(float(t[q])) - te) <= Decimal(2.0 ** -44) * (abs(te) + 1)


@pytest.mark.parametrize("h,w", [(15, 15), (31, 31), (63, 63), (8, 40)])
def test_fp64_sauvola_matches_exact_decision(h, w):
    img = synth.document(256, 300, 11, stains=3)
    S1, S2, n = oracle.window_sums(img, h, w)
    bits, _ = oracle.sauvola(img, h, w, k=0.5, R=128.0)
    exact = oracle.sauvola_bits_exact(img, S1, S2, n, 1, 2, 128, 1)
    diff = bits != exact
    # disagreements may only occur where FP64 rounding decides a near-tie
    if diff.any():
        t = oracle.threshold(oracle.SAUVOLA, S1[diff], S2[diff], n[diff], 0.5, 128.0)
        assert np.all(np.abs(img[diff] - t) < 1e-9)
    assert diff.sum() <= 1e-4 * img.size


def test_exact_decision_detects_planted_sign_error():
    # a wrong sign in the threshold formula must show up against the exact rule
    img = synth.document(64, 64, 12)
    S1, S2, n = oracle.window_sums(img, 15, 15)
    exact = oracle.sauvola_bits_exact(img, S1, S2, n, 1, 2, 128, 1)
    m = S1 / n
    s = np.sqrt((n.astype(np.float64) * S2 - S1.astype(np.float64) ** 2)) / n
    wrong = (img > m * (1 + 0.5 * (s / 128 + 1))).astype(np.uint8)  # planted mistake
    assert (wrong != exact).mean() > 0.05


def test_sqrt_free_condition_equivalent():
    # Sec. 3.2: for k >= 0 the square-root-free condition decides I <= t.
    img = synth.document(128, 128, 13, stains=2)
    for k in (0.2, 0.5):
        S1, S2, n = oracle.window_sums(img, 31, 31)
        bits, _ = oracle.sauvola(img, 31, 31, k=k)
        alt = oracle.sauvola_bits_paper_order(img, S1, S2, n, k, 128.0)
        assert (bits != alt).mean() <= 1e-4


def test_pack_bits_layout():
    bits = np.zeros((2, 11), np.uint8)
    bits[0, 0] = 1
    bits[0, 9] = 1
    bits[1, 7] = 1
    bits[1, 10] = 1
    out = oracle.pack_bits(bits, out_pitch=4)
    np.testing.assert_array_equal(out, np.array([[0x01, 0x02, 0, 0], [0x80, 0x04, 0, 0]], np.uint8))


# ---------------------------------------------------------------- quantiles
def test_quantile_routes_agree():
    rng = np.random.default_rng(5)
    for img, H, W, h, w in tiny_cases(120, 6):
        qd = int(rng.integers(1, 11))
        qn = int(rng.integers(0, qd + 1))
        a = oracle.window_quantile(img, h, w, qn, qd, "sort", W=W)
        b = oracle.window_quantile(img, h, w, qn, qd, "count", W=W)
        c = oracle.window_quantile(img, h, w, qn, qd, "sliding", W=W)
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)


def _window_view(img, h, w, fill):
    l, r, o, u = oracle.window_params(h, w)
    pad = np.pad(img.astype(np.int32), ((o - 1, u), (l - 1, r)), constant_values=fill)
    return np.lib.stride_tricks.sliding_window_view(pad, (h, w))


def test_quantile_extremes_are_min_and_max():
    img = synth.document(40, 50, 14, salt_pepper=0.05)
    for h, w in [(5, 5), (6, 9), (31, 31)]:
        v = _window_view(img, h, w, fill=-1)
        mx = v.max(axis=(2, 3))
        mn = np.where(v < 0, 999, v).min(axis=(2, 3))
        np.testing.assert_array_equal(oracle.window_quantile(img, h, w, 1, 1), mx)
        np.testing.assert_array_equal(oracle.window_quantile(img, h, w, 0, 1), mn)


def test_quantile_median_matches_numpy_interior():
    img = synth.uniform(30, 30, 15)
    Q = oracle.window_quantile(img, 5, 5, 1, 2)
    v = _window_view(img, 5, 5, fill=-1)
    # interior: n = 25, rank ceil(12.5) = 13 -> the true median
    med = np.median(v[2:-2, 2:-2].reshape(26, 26, 25), axis=2)
    np.testing.assert_array_equal(Q[2:-2, 2:-2], med.astype(np.uint8))


def test_quantile_constant_and_unit_window():
    img = np.full((12, 9), 93, np.uint8)
    assert (oracle.window_quantile(img, 7, 7, 1, 10) == 93).all()
    img = synth.uniform(12, 9, 16)
    np.testing.assert_array_equal(oracle.window_quantile(img, 1, 1, 1, 2), img)


def test_quantile_binarization_rule():
    img = synth.document(50, 60, 17, salt_pepper=0.02)
    Q = oracle.window_quantile(img, 9, 9, 1, 2)
    bits, packed = oracle.binarize_quantile(img, 9, 9, 1, 2, offset=8)
    np.testing.assert_array_equal(bits, (img.astype(int) > Q.astype(int) - 8).astype(np.uint8))
    np.testing.assert_array_equal(packed, oracle.pack_bits(bits))
