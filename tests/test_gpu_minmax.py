"""GPU parity of the local minimum / maximum and of Bernsen's decision
(integer work: bit-exact) against the CPU oracle, through the C ABI.

Shapes span several 512-column x 32-row tiles with ragged tails, windows
from 1 x 1 to 511 x 511 (larger than the image too), even windows, W = 1,
H = 1, pitch > W and an unaligned base address (the byte-load path)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_packed, out_buffer, to_device

pytestmark = pytest.mark.gpu

SHAPES = [
    # H, W, h, w
    (97, 600, 15, 15),
    (130, 1100, 31, 127),
    (40, 33, 2, 3),
    (1, 700, 5, 9),
    (700, 1, 9, 5),
    (17, 23, 100, 120),
    (75, 1030, 255, 1),
    (64, 520, 511, 511),
    (66, 515, 1, 1),
    (90, 700, 32, 64),
]


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    return bz


@pytest.mark.parametrize("H,W,h,w", SHAPES)
@pytest.mark.parametrize("layout", ["aligned", "pitch+5", "misaligned"])
def test_window_minmax_exact(H, W, h, w, layout):
    import paper_1905_13038_gb300 as bz
    extra = 5 if layout == "pitch+5" else 0
    img = synth.document(H, W, 500 + H + W, salt_pepper=0.01, pitch=W + extra)
    t, _ = to_device(img, W, misalign=3 if layout == "misaligned" else 0)
    mn, mx = bz.window_minmax(t, h, w, W=W)
    emn, emx = oracle.window_minmax(img, h, w, W=W)
    np.testing.assert_array_equal(mn.cpu().numpy(), emn)
    np.testing.assert_array_equal(mx.cpu().numpy(), emx)


@pytest.mark.parametrize("H,W,h,w", SHAPES)
@pytest.mark.parametrize("limit", [0, 15, 256])
def test_bernsen_exact(H, W, h, w, limit):
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 900 + H * 3 + W, stains=1 if min(H, W) > 20 else 0)
    t, _ = to_device(img, W)
    out = out_buffer(H, W, extra=2)
    bz.binarize_bernsen(t, h, w, limit, out=out, W=W)
    _, packed = oracle.binarize_bernsen(img, h, w, limit, W=W)
    check_packed(out, packed, W)


@pytest.mark.parametrize("layout", ["pitch+5", "misaligned"])
def test_bernsen_layouts(layout):
    import paper_1905_13038_gb300 as bz
    H, W = 150, 777
    extra = 5 if layout == "pitch+5" else 0
    img = synth.document(H, W, 31337, stains=1, pitch=W + extra)
    t, _ = to_device(img, W, misalign=3 if layout == "misaligned" else 0)
    out = out_buffer(H, W, extra=1)
    bz.binarize_bernsen(t, 31, 31, 15, out=out, W=W)
    _, packed = oracle.binarize_bernsen(img, 31, 31, 15, W=W)
    check_packed(out, packed, W)


@pytest.mark.parametrize("h,w", [(15, 15), (31, 31), (255, 255)])
def test_bernsen_full_page(h, w):
    # the bench's page and launch
    import paper_1905_13038_gb300 as bz
    img = synth.document(3072, 4096, 0x19051303800 + 2, stains=3)
    t, _ = to_device(img)
    out = bz.binarize_bernsen(t, h, w, 15)
    _, packed = oracle.binarize_bernsen(img, h, w, 15)
    np.testing.assert_array_equal(out.cpu().numpy(), packed)


def test_minmax_full_page_sampled():
    import paper_1905_13038_gb300 as bz
    img = synth.document(3072, 4096, 0x19051303800 + 2, stains=3)
    t, _ = to_device(img)
    mn, mx = bz.window_minmax(t, 63, 63)
    rng = np.random.default_rng(3)
    ii = np.concatenate([rng.integers(0, 3072, 3000), [0, 3071, 0, 3071]])
    jj = np.concatenate([rng.integers(0, 4096, 3000), [0, 4095, 4095, 0]])
    emn, emx = oracle.window_minmax_at(img, 63, 63, ii, jj)
    np.testing.assert_array_equal(mn.cpu().numpy()[ii, jj], emn)
    np.testing.assert_array_equal(mx.cpu().numpy()[ii, jj], emx)


def test_bernsen_rejects_bad_arguments():
    import paper_1905_13038_gb300 as bz
    img = synth.document(20, 40, 1)
    t, _ = to_device(img)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_bernsen(t, 5, 5, -1)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_bernsen(t, 5, 5, 257)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_bernsen(t, 512, 5, 15)
