"""GPU parity of the Haar-like window sums (integer work: bit-exact) against
the CPU oracle's integral-image route, through the C ABI.  Shapes span
several 256-column x 32-row tiles with ragged tails, every preset feature,
random profiles of up to four segments with weights up to +-127 (within the
2^31 bound), windows up to 511 x 511 and larger than the image, W = 1,
H = 1, pitch > W and an unaligned base (the byte-load path)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import to_device

pytestmark = pytest.mark.gpu

SHAPES = [(97, 600), (130, 515), (40, 33), (1, 700), (700, 1), (64, 1030)]
WINDOWS = [(24, 24), (6, 9), (2, 2), (63, 129), (300, 257)]


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    return bz


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("hw", WINDOWS)
@pytest.mark.parametrize("name", ["edge_h", "edge_v", "line_h", "line_v", "diag"])
def test_haar_presets_exact(H, W, hw, name):
    import paper_1905_13038_gb300 as bz
    h, w = hw
    if name.startswith("line") and min(h, w) < 3:
        pytest.skip("three segments need h, w >= 3")
    rows, cols = bz.HAAR_FEATURES[name](h, w)
    img = synth.document(H, W, 77 + H + W)
    t, _ = to_device(img)
    got = bz.haar_feature(t, rows, cols).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.haar(img, rows, cols))


@pytest.mark.parametrize("layout", ["pitch+5", "misaligned"])
def test_haar_layouts(layout):
    import paper_1905_13038_gb300 as bz
    H, W = 150, 777
    extra = 5 if layout == "pitch+5" else 0
    img = synth.document(H, W, 4321, pitch=W + extra)
    t, _ = to_device(img, W, misalign=3 if layout == "misaligned" else 0)
    rows, cols = bz.HAAR_FEATURES["diag"](30, 40)
    got = bz.haar_feature(t, rows, cols, W=W).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.haar(img, rows, cols, W=W))


def test_haar_random_profiles():
    import paper_1905_13038_gb300 as bz
    rng = np.random.default_rng(5)
    img = synth.document(120, 650, 99)
    t, _ = to_device(img)
    for _ in range(40):
        rows = [(int(rng.integers(1, 60)), int(rng.integers(-127, 128))) for _ in range(int(rng.integers(1, 5)))]
        cols = [(int(rng.integers(1, 60)), int(rng.integers(-127, 128))) for _ in range(int(rng.integers(1, 5)))]
        h, w = sum(n for n, _ in rows), sum(n for n, _ in cols)
        fm = max(abs(x) for _, x in rows)
        gm = max(abs(x) for _, x in cols)
        if 255 * h * w * fm * gm >= 2**31:
            with pytest.raises(bz.BinarizeError):
                bz.haar_feature(t, rows, cols)
            continue
        got = bz.haar_feature(t, rows, cols).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.haar(img, rows, cols))


def test_haar_full_page():
    import paper_1905_13038_gb300 as bz
    img = synth.document(3072, 4096, 0x19051303800 + 2, stains=3)
    t, _ = to_device(img)
    rows, cols = bz.HAAR_FEATURES["line_h"](24, 24)
    got = bz.haar_feature(t, rows, cols).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.haar(img, rows, cols))


def test_haar_largest_window_and_bounds():
    import paper_1905_13038_gb300 as bz
    img = synth.uniform(90, 600, 3, 200, 255)
    t, _ = to_device(img)
    rows, cols = [(511, 1)], [(255, 1), (256, -1)]
    got = bz.haar_feature(t, rows, cols).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.haar(img, rows, cols))
    with pytest.raises(bz.BinarizeError):
        bz.haar_feature(t, [(511, 40)], [(511, 1)])  # 255 * 511^2 * 40 >= 2^31
    with pytest.raises(bz.BinarizeError):
        bz.haar_feature(t, [(300, 1), (300, 1)], [(5, 1)])  # h > 511
