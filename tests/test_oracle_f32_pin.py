"""Pin of the oracle's FP32 threshold helper (used only to grade the FP32
fast path): it must equal the pinned FP64 threshold (Sec. 1 Sauvola,
Niblack) within the rounding-error bound of its own FP32 operations.

With u = 2^-24 and exact integer inputs (S1 < 2^24, n <= 65025): m is one
correctly rounded division (u); s = sqrt(V / n^2) takes three roundings under
the root and one for it (<= 5.5 u relative); the Sauvola factor adds four
more and the final product one, Niblack one product and one sum.  A bound of
16 u on the sum of the terms' magnitudes (m, |k| m s / R, |k| m for Sauvola;
m, |k| s for Niblack) covers them with room to spare, while a dropped term,
a wrong sign or a transposed operand moves t by a sizeable fraction of m."""
import numpy as np
import pytest

import oracle

U = 2.0 ** -24


def random_windows(seed, count=20000):
    rng = np.random.default_rng(seed)
    h = rng.integers(1, 256, count)
    w = rng.integers(1, 256, count)
    n = (h * w).astype(np.uint32)
    # window contents: a mean level with a spread, so s covers 0 .. 127.5
    lo = rng.integers(0, 256, count)
    hi = np.minimum(255, lo + rng.integers(0, 256, count))
    frac = rng.random(count)
    n_hi = np.floor(frac * n).astype(np.int64)
    n_lo = n.astype(np.int64) - n_hi
    S1 = (n_lo * lo + n_hi * hi).astype(np.uint32)
    S2 = (n_lo * lo * lo + n_hi * hi * hi).astype(np.uint64)
    return S1, S2, n


@pytest.mark.parametrize("method,k,R", [(oracle.SAUVOLA, 0.5, 128.0), (oracle.SAUVOLA, 0.2, 100.0),
                                        (oracle.SAUVOLA, -0.3, 64.0), (oracle.NIBLACK, -0.2, 128.0),
                                        (oracle.NIBLACK, 0.7, 128.0)])
def test_f32_threshold_within_its_rounding_bound(method, k, R):
    S1, S2, n = random_windows(11 + int(100 * abs(k)) + 7 * method)
    t64 = oracle.threshold(method, S1, S2, n, k, R)
    t32 = oracle.threshold_f32(method, S1, S2, n, k, R).astype(np.float64)
    nd = n.astype(np.float64)
    m = S1 / nd
    s = np.sqrt(np.maximum(0.0, (nd * S2.astype(np.float64) - S1.astype(np.float64) ** 2)) / (nd * nd))
    if method == oracle.SAUVOLA:
        mag = m + abs(k) * m * s / R + abs(k) * m
    else:
        mag = m + abs(k) * s
    err = np.abs(t32 - t64)
    assert (err <= 16 * U * mag + 1e-30).all(), float((err / np.maximum(mag, 1e-30)).max() / U)
    # the bound is not vacuous: FP32 does round somewhere
    assert err.max() > 0


def test_f32_threshold_detects_a_planted_sign_error():
    # the same bound rejects t computed with (s/R + 1) in place of (s/R - 1)
    S1, S2, n = random_windows(5)
    k, R = 0.5, 128.0
    t64 = oracle.threshold(oracle.SAUVOLA, S1, S2, n, k, R)
    nd = n.astype(np.float64)
    m = S1 / nd
    s = np.sqrt(np.maximum(0.0, (nd * S2.astype(np.float64) - S1.astype(np.float64) ** 2)) / (nd * nd))
    wrong = (m * (1.0 + k * (s / R + 1.0))).astype(np.float32).astype(np.float64)
    mag = m + abs(k) * m * s / R + abs(k) * m
    assert (np.abs(wrong - t64) > 16 * U * mag + 1e-30).any()


def test_f32_threshold_bound_detects_sample_variance():
    # dividing V by n (n - 1) instead of n^2 (sample rather than population
    # deviation) leaves the bound on some windows
    S1, S2, n = random_windows(9)
    k, R = 0.5, 128.0
    t64 = oracle.threshold(oracle.SAUVOLA, S1, S2, n, k, R)
    nd = n.astype(np.float64)
    m = S1 / nd
    V = np.maximum(0.0, nd * S2.astype(np.float64) - S1.astype(np.float64) ** 2)
    s = np.sqrt(V / (nd * nd))
    s_sample = np.sqrt(V / (nd * np.maximum(nd - 1.0, 1.0)))
    wrong = m * (1.0 + k * (s_sample / R - 1.0))
    mag = m + abs(k) * m * s / R + abs(k) * m
    assert (np.abs(wrong - t64) > 16 * U * mag + 1e-30).any()
