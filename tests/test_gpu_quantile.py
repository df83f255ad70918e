"""GPU parity of the local-quantile path (Sec. 3.4) against the oracle:
quantile plane and binary output bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_packed, out_buffer, to_device

pytestmark = pytest.mark.gpu

CASES = [
    # H, W, h, w, q_num, q_den
    (70, 300, 9, 9, 1, 2),
    (70, 300, 8, 12, 1, 10),
    (129, 200, 31, 31, 1, 2),
    (40, 33, 2, 3, 3, 4),
    (1, 200, 5, 7, 1, 2),
    (200, 1, 7, 5, 1, 2),
    (15, 19, 60, 50, 1, 2),
    (90, 140, 101, 101, 1, 10),
    (300, 300, 257, 257, 1, 2),  # h*w > 65535: 32-bit histogram counters
    (50, 70, 5, 5, 0, 1),
    (50, 70, 5, 5, 1, 1),
    (160, 230, 36, 36, 1, 2),    # the tallest window with 8-bit own counts (7 h = 252)
    (160, 230, 36, 130, 1, 10),  # ... with a core part and a wide read-ahead
    (160, 230, 37, 37, 1, 2),    # the shortest window with 10-bit own counts
    (200, 230, 146, 40, 1, 2),   # the tallest window with 10-bit own counts (7 h = 1022)
    (200, 230, 147, 147, 1, 10),  # the shortest window with 16-bit own counts
]


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()


@pytest.mark.parametrize("H,W,h,w,qn,qd", CASES)
def test_window_quantile_exact(H, W, h, w, qn, qd):
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 400 + H, stains=1 if min(H, W) > 20 else 0, salt_pepper=0.02,
                         pitch=W + 3)
    t, _ = to_device(img, W, misalign=2)
    Q = bz.window_quantile(t, h, w, qn, qd, W=W).cpu().numpy()
    np.testing.assert_array_equal(Q, oracle.window_quantile(img, h, w, qn, qd, W=W))


@pytest.mark.parametrize("H,W,h,w,qn,qd", CASES)
@pytest.mark.parametrize("offset", [8, 0, -5])
def test_binarize_quantile_exact(H, W, h, w, qn, qd, offset):
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 500 + W, salt_pepper=0.02)
    t, _ = to_device(img)
    out = out_buffer(H, W, extra=1)
    bz.binarize_quantile(t, h, w, qn, qd, offset, out=out)
    _, ref = oracle.binarize_quantile(img, h, w, qn, qd, offset)
    check_packed(out, ref, W)


@pytest.mark.parametrize("h,w,qn,qd", [(31, 31, 1, 2), (31, 31, 1, 10), (101, 101, 1, 2), (101, 101, 1, 10)])
def test_quantile_page_full(h, w, qn, qd):
    """2048 x 2048 page with 2% salt-and-pepper: the full quantile plane and
    binary output against the (parallel) sliding-histogram oracle."""
    import paper_1905_13038_gb300 as bz
    img = synth.quantile_page()
    t, W = to_device(img)
    nt = oracle.max_threads()
    Q = bz.window_quantile(t, h, w, qn, qd).cpu().numpy()
    np.testing.assert_array_equal(Q, oracle.window_quantile(img, h, w, qn, qd, threads=nt))
    out = bz.binarize_quantile(t, h, w, qn, qd, 8)
    _, ref = oracle.binarize_quantile(img, h, w, qn, qd, 8, threads=nt)
    check_packed(out, ref, W)


@pytest.mark.parametrize("h,w", [(36, 36), (36, 9), (37, 37), (146, 20), (147, 147)])
def test_own_counts_at_their_limit(h, w):
    """A flat page puts every pixel of a lane's own part (7 columns x h rows:
    252 at h = 36, 1022 at h = 146) in one gray level, the most an 8-bit
    (10-bit) own count ever holds; a page that is flat except for one bright
    column moves Q across the full count."""
    import paper_1905_13038_gb300 as bz
    H, W = 200, 150
    flat = np.full((H, W), 77, dtype=np.uint8)
    ramp = flat.copy()
    ramp[:, 70] = 250
    for img in (flat, ramp):
        t, _ = to_device(img)
        for qn, qd in ((1, 2), (1, 100), (99, 100)):
            Q = bz.window_quantile(t, h, w, qn, qd).cpu().numpy()
            np.testing.assert_array_equal(Q, oracle.window_quantile(img, h, w, qn, qd))


@pytest.mark.parametrize("h,w,qn,qd", [(31, 31, 1, 20), (31, 31, 19, 20), (45, 77, 1, 8), (101, 101, 7, 8),
                                        (15, 15, 0, 1), (15, 15, 1, 1)])
def test_long_walks_across_empty_gray_levels(h, w, qn, qd):
    """Far-from-median ranks on a page of two levels (30 and 220) in blocks
    with sparse noise: from one row to the next Q crosses the empty gray
    values between the levels, the longest moves its walk makes."""
    import paper_1905_13038_gb300 as bz
    rng = np.random.default_rng(h * 1000 + qn)
    H, W = 260, 330
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.where(((yy // 37) + (xx // 53)) % 2 == 0, 30, 220).astype(np.uint8)
    noise = rng.random((H, W)) < 0.03
    img[noise] = rng.integers(0, 256, int(noise.sum())).astype(np.uint8)
    t, _ = to_device(img)
    Q = bz.window_quantile(t, h, w, qn, qd).cpu().numpy()
    np.testing.assert_array_equal(Q, oracle.window_quantile(img, h, w, qn, qd))
    out = bz.binarize_quantile(t, h, w, qn, qd, 8)
    check_packed(out, oracle.binarize_quantile(img, h, w, qn, qd, 8)[1], W)
