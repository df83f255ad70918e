"""Pins of the oracle's other Table 1 thresholds (Wolf, Feng, Rais, NICK,
Phansalkar) and of the global statistics L, M, S they use.

The formulas are not re-typed here.  Each method is pinned by facts that hold
independently of how the oracle evaluates it:

* global L, M, S against numpy's min, mean and population std;
* special cases that reduce a method to Sauvola or Niblack, whose oracle is
  pinned in test_oracle_pins.py (Wolf with L = 0, Feng with gamma = 0 and
  L = 0, Phansalkar with p = 0 or with exp(-q m) below one ulp);
* other published or closed forms of the same threshold (NICK in the form of
  Khurshid et al., Rais as a two-branch expression, Wolf with k = 1, Feng with
  the integer exponent gamma = 2 written as products);
* invariants: doubling every gray level (with R, L doubled and q halved)
  doubles every threshold, so the binary image cannot change; Rais moves the
  threshold towards m by at most k*s; Wolf stays between L and m.

Local window statistics come from direct numpy slicing (the Sec. 1
definition), not from the oracle's sums.
"""
import numpy as np
import pytest

import oracle
import synth


def brute_stats(img, h, w):
    """S1, S2, n by direct slicing of the clipped window (Sec. 1)."""
    H, W = img.shape
    l, r, o, u = (w + 1) // 2, w // 2, (h + 1) // 2, h // 2
    a = img.astype(np.int64)
    S1 = np.zeros((H, W), np.int64)
    S2 = np.zeros((H, W), np.int64)
    n = np.zeros((H, W), np.int64)
    for i in range(H):
        r0, r1 = max(i - o + 1, 0), min(i + u, H - 1) + 1
        for j in range(W):
            c0, c1 = max(j - l + 1, 0), min(j + r, W - 1) + 1
            blk = a[r0:r1, c0:c1]
            S1[i, j] = blk.sum()
            S2[i, j] = (blk * blk).sum()
            n[i, j] = blk.size
    m = S1 / n
    s = np.sqrt((n * S2 - S1 * S1).astype(np.float64)) / n
    return S1, S2, n, m, s


def case(seed, H=23, W=29, h=7, w=5, lo=0, hi=256):
    rng = np.random.default_rng(seed)
    img = rng.integers(lo, hi, size=(H, W), dtype=np.uint8)
    return img, h, w


def thresholds(method, img, h, w, prm, glob=None):
    S1, S2, n = oracle.window_sums(img, h, w)
    if glob is None:
        glob, _ = oracle.global_stats(img)
    return oracle.threshold_ext(method, S1, S2, n, prm, glob)


# ---------------------------------------------------------------- global stats
@pytest.mark.parametrize("seed", range(6))
def test_global_stats_match_numpy(seed):
    rng = np.random.default_rng(100 + seed)
    H, W = int(rng.integers(1, 80)), int(rng.integers(1, 80))
    img = rng.integers(int(rng.integers(0, 100)), 256, size=(H, W), dtype=np.uint8)
    (L, M, S), (sm, sq, N) = oracle.global_stats(img)
    assert L == img.min()
    assert sm == int(img.astype(np.int64).sum()) and N == H * W
    assert sq == int((img.astype(np.int64) ** 2).sum())
    assert M == img.astype(np.int64).sum() / (H * W)  # one rounding of an exact sum
    assert abs(S - img.astype(np.float64).std()) <= 1e-12 * max(1.0, S)


def test_global_stats_with_row_padding_and_constant_image():
    img = np.full((9, 16), 77, np.uint8)
    img[:, 13:] = 3  # padding columns, outside the W = 13 image
    (L, M, S), (_, _, N) = oracle.global_stats(img, W=13)
    assert (L, M, S, N) == (77.0, 77.0, 0.0, 9 * 13)


def test_global_std_large_page_is_exact_numerator():
    # N * sumsq exceeds 2^64 here: the exact 128-bit numerator must survive
    img = synth.uniform(4400, 4400, 5, lo=235, hi=255)
    (L, M, S), (sm, sq, N) = oracle.global_stats(img)
    assert N * sq > 2**64
    exact = (N * sq - sm * sm) / (N * N)  # Python ints, one final rounding
    assert abs(S * S - exact) <= 4e-16 * exact


# ---------------------------------------------------------------- Wolf
@pytest.mark.parametrize("seed", range(4))
def test_wolf_with_zero_minimum_is_sauvola(seed):
    img, h, w = case(200 + seed)
    img[0, 0] = 0  # global minimum L = 0
    prm = oracle.params(k=0.4, R=110.0)
    S1, S2, n = oracle.window_sums(img, h, w)
    t_wolf = thresholds(oracle.WOLF, img, h, w, prm)
    t_sau = oracle.threshold(oracle.SAUVOLA, S1, S2, n, 0.4, 110.0)
    np.testing.assert_allclose(t_wolf, t_sau, rtol=4e-15, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_wolf_k1_closed_form_and_bounds(seed):
    img, h, w = case(210 + seed, lo=30)
    _, _, _, m, s = brute_stats(img, h, w)
    L = float(img.min())
    R = 130.0
    t1 = thresholds(oracle.WOLF, img, h, w, oracle.params(k=1.0, R=R))
    # k = 1: t = L + (m - L) s / R
    np.testing.assert_allclose(t1, L + (m - L) * s / R, rtol=0, atol=1e-12)
    # 0 <= k <= 1 and s <= R: L <= t <= m
    t = thresholds(oracle.WOLF, img, h, w, oracle.params(k=0.6, R=R))
    assert np.all(t <= m + 1e-12) and np.all(t >= L - 1e-12)
    # k = 0: the local mean
    t0 = thresholds(oracle.WOLF, img, h, w, oracle.params(k=0.0, R=R))
    np.testing.assert_array_equal(t0, m)


# ---------------------------------------------------------------- Feng
@pytest.mark.parametrize("seed", range(3))
def test_feng_gamma0_zero_minimum_is_sauvola(seed):
    img, h, w = case(300 + seed)
    img[5, 5] = 0
    k, R = 0.35, 120.0
    S1, S2, n = oracle.window_sums(img, h, w)
    t_feng = thresholds(oracle.FENG, img, h, w,
                        oracle.params(R=R, alpha1=1.0 - k, k1=k, k2=0.7, gamma=0.0))
    t_sau = oracle.threshold(oracle.SAUVOLA, S1, S2, n, k, R)
    np.testing.assert_allclose(t_feng, t_sau, rtol=4e-15, atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_feng_integer_gamma_as_products(seed):
    img, h, w = case(310 + seed, lo=20)
    _, _, _, m, s = brute_stats(img, h, w)
    L = float(img.min())
    a1, k1, k2, R = 0.88, 0.25, 0.04, 100.0
    x = s / R
    t = thresholds(oracle.FENG, img, h, w, oracle.params(R=R, alpha1=a1, k1=k1, k2=k2, gamma=2.0))
    np.testing.assert_allclose(t, a1 * m + k1 * x * x * x * (m - L) + k2 * x * x * L, rtol=1e-13)
    # gamma = 0: affine in s
    t0 = thresholds(oracle.FENG, img, h, w, oracle.params(R=R, alpha1=a1, k1=k1, k2=k2, gamma=0.0))
    np.testing.assert_allclose(t0, a1 * m + k1 * x * (m - L) + k2 * L, rtol=1e-13)


# ---------------------------------------------------------------- Rais
@pytest.mark.parametrize("seed", range(4))
def test_rais_two_branch_form(seed):
    img, h, w = case(400 + seed)
    img[:, : img.shape[1] // 2] //= 4  # a dark, flat half and a noisy half
    _, _, _, m, s = brute_stats(img, h, w)
    M, S = img.astype(np.float64).mean(), img.astype(np.float64).std()
    k = 0.3
    t = thresholds(oracle.RAIS, img, h, w, oracle.params(k=k))
    ms, MS = m * s, M * S
    frac = np.where(ms >= MS, 1.0 - MS / np.where(ms > 0, ms, 1.0), ms / MS - 1.0)
    np.testing.assert_allclose(t, m + k * frac * s, rtol=0, atol=1e-11)
    # the threshold moves from m by at most k*s, towards the sign of ms - MS
    assert np.all(np.abs(t - m) <= k * s + 1e-12)
    assert np.all(np.sign(np.round(t - m, 9)) * np.sign(np.round(ms - MS, 9)) >= 0)


def test_rais_constant_image_is_mean():
    img = np.full((10, 12), 90, np.uint8)
    t = thresholds(oracle.RAIS, img, 3, 5, oracle.params(k=0.3))
    np.testing.assert_array_equal(t, 90.0)  # m*s = M*S = 0: the 0/0 reading gives f = 0


# ---------------------------------------------------------------- NICK
@pytest.mark.parametrize("seed,h,w", [(0, 7, 5), (1, 19, 19), (2, 1, 1), (3, 40, 3)])
def test_nick_matches_khurshid_form(seed, h, w):
    # Khurshid et al.: T = m + k sqrt((sum p^2 - m^2) / NP), NP = window pixels
    img, _, _ = case(500 + seed)
    S1, S2, n, m, s = brute_stats(img, h, w)
    k = -0.15
    t = thresholds(oracle.NICK, img, h, w, oracle.params(k=k))
    np.testing.assert_allclose(t, m + k * np.sqrt((S2 - m * m) / n), rtol=1e-13)
    t0 = thresholds(oracle.NICK, img, h, w, oracle.params(k=0.0))
    np.testing.assert_array_equal(t0, m)


# ---------------------------------------------------------------- Phansalkar
@pytest.mark.parametrize("seed", range(3))
def test_phansalkar_reduces_to_sauvola(seed):
    img, h, w = case(600 + seed, lo=40)
    S1, S2, n = oracle.window_sums(img, h, w)
    k, R = 0.25, 127.5
    t_sau = oracle.threshold(oracle.SAUVOLA, S1, S2, n, k, R)
    # p = 0 removes the exponential term
    t_p0 = thresholds(oracle.PHANSALKAR, img, h, w, oracle.params(k=k, R=R, p=0.0, q=0.5))
    np.testing.assert_allclose(t_p0, t_sau, rtol=4e-15)
    # m >= 40 and q = 1: p exp(-q m) < 1e-17, below half an ulp of 1
    t_q = thresholds(oracle.PHANSALKAR, img, h, w, oracle.params(k=k, R=R, p=2.0, q=1.0))
    np.testing.assert_allclose(t_q, t_sau, rtol=4e-15)


@pytest.mark.parametrize("seed", range(3))
def test_phansalkar_q0_and_normalised_form(seed):
    img, h, w = case(610 + seed)
    _, _, _, m, s = brute_stats(img, h, w)
    k, R, p = 0.25, 127.5, 2.0
    t = thresholds(oracle.PHANSALKAR, img, h, w, oracle.params(k=k, R=R, p=p, q=0.0))
    np.testing.assert_allclose(t, m * (1 + p) + m * k * (s / R - 1), rtol=1e-13)
    # Phansalkar et al. work on gray levels scaled to [0, 1] (p = 2, q = 10,
    # k = 0.25, R = 0.5); on 0..255 levels that is q = 10/255, R = 127.5
    mn, sn = m / 255.0, s / 255.0
    tn = mn * (1 + p * np.exp(-10.0 * mn) + k * (sn / 0.5 - 1))
    t255 = thresholds(oracle.PHANSALKAR, img, h, w, oracle.params(k=k, R=127.5, p=p, q=10.0 / 255.0))
    np.testing.assert_allclose(t255, 255.0 * tn, rtol=1e-12)


# ---------------------------------------------------------------- invariants
METHODS = [
    (oracle.WOLF, dict(k=0.5, R=96.0), dict(k=0.5, R=192.0)),
    (oracle.FENG, dict(alpha1=0.88, k1=0.25, k2=0.04, gamma=2.0, R=64.0),
     dict(alpha1=0.88, k1=0.25, k2=0.04, gamma=2.0, R=128.0)),
    (oracle.RAIS, dict(k=0.3), dict(k=0.3)),
    (oracle.NICK, dict(k=-0.1), dict(k=-0.1)),
    (oracle.PHANSALKAR, dict(k=0.25, R=64.0, p=2.0, q=20.0 / 255.0),
     dict(k=0.25, R=128.0, p=2.0, q=10.0 / 255.0)),
]


@pytest.mark.parametrize("method,prm1,prm2", METHODS)
def test_doubling_gray_levels_keeps_every_bit(method, prm1, prm2):
    # every threshold is homogeneous of degree 1 in (I, L, M, S, R) with q
    # scaled inversely; doubling is exact in binary floating point, so the
    # binary images are identical bit for bit
    img = synth.document(61, 77, 9)
    half = (img // 2).astype(np.uint8)
    b1, _ = oracle.binarize_ext(method, half, 9, 13, oracle.params(**prm1))
    b2, _ = oracle.binarize_ext(method, (half * 2).astype(np.uint8), 9, 13, oracle.params(**prm2))
    np.testing.assert_array_equal(b1, b2)
    assert 0 < b1.mean() < 1


@pytest.mark.parametrize("method", [oracle.WOLF, oracle.FENG, oracle.RAIS, oracle.NICK, oracle.PHANSALKAR])
def test_binarize_ext_is_the_threshold_decision(method):
    img = synth.document(37, 45, 4, pitch=48)
    prm = oracle.params(k=0.5 if method != oracle.NICK else -0.1)
    bits, packed = oracle.binarize_ext(method, img, 11, 7, prm, W=45)
    t = thresholds(method, img[:, :45], 11, 7, prm)
    np.testing.assert_array_equal(bits, (img[:, :45] > t).astype(np.uint8))
    np.testing.assert_array_equal(packed, oracle.pack_bits(bits))
