"""GPU parity of the window path (Sauvola, Niblack, exact window sums) against
the CPU oracle, element by element, through the C ABI.

Bar: window sums bit-exact; BZ_FP64 and BZ_FP64_DIRECT output bit-exact with
the canonical FP64 threshold; BZ_FP32 output within 1e-5 of the pixels.
Sizes span several 256-column warp tiles and several row bands with ragged
tails; adversarial shapes cover W = 1, H = 1, windows larger than the image,
even windows, pitch > W, unaligned pitch and unaligned base, and the 64-bit
S2 path (h*w > 66051)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_packed, out_buffer, to_device, unpack

pytestmark = pytest.mark.gpu

SHAPES = [
    # H, W, h, w
    (97, 600, 15, 15),
    (97, 600, 31, 127),
    (130, 515, 64, 9),
    (300, 1030, 255, 255),
    (40, 33, 2, 3),
    (1, 700, 5, 9),
    (700, 1, 9, 5),
    (17, 23, 100, 120),
    (270, 290, 260, 257),  # h*w = 66820: 64-bit S2
    (64, 520, 511, 511),
    (33, 257, 32, 32),
]


def image_for(H, W, seed, pitch_extra=0):
    return synth.document(H, W, seed, stains=1 if min(H, W) > 20 else 0, pitch=W + pitch_extra)


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    return bz


@pytest.mark.parametrize("H,W,h,w", SHAPES)
@pytest.mark.parametrize("layout", ["aligned", "pitch+5", "misaligned"])
def test_window_sums_exact(H, W, h, w, layout):
    import paper_1905_13038_gb300 as bz
    extra = 5 if layout == "pitch+5" else 0
    img = image_for(H, W, 100 + H + W, extra)
    t, _ = to_device(img, W, misalign=3 if layout == "misaligned" else 0)
    S1, S2, n = bz.window_sums(t, h, w, W=W)
    e1, e2, en = oracle.window_sums(img, h, w, W=W)
    np.testing.assert_array_equal(S1.cpu().numpy().view(np.uint32), e1)
    np.testing.assert_array_equal(S2.cpu().numpy().view(np.uint64), e2)
    np.testing.assert_array_equal(n.cpu().numpy().view(np.uint32), en)


@pytest.mark.parametrize("H,W,h,w", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp64_direct"])
def test_sauvola_fp64_bit_exact(H, W, h, w, precision):
    import paper_1905_13038_gb300 as bz
    img = image_for(H, W, 200 + H + W, 3)
    t, _ = to_device(img, W)
    out = out_buffer(H, W, extra=2)
    bz.binarize_sauvola(t, h, w, 0.5, 128.0, out=out, precision=precision, W=W)
    _, ref = oracle.sauvola(img, h, w, k=0.5, R=128.0, W=W)
    check_packed(out, ref, W)


@pytest.mark.parametrize("H,W,h,w", SHAPES)
def test_niblack_fp64_bit_exact(H, W, h, w):
    import paper_1905_13038_gb300 as bz
    img = image_for(H, W, 300 + H + W)
    t, _ = to_device(img, W, misalign=1)
    out = out_buffer(H, W, extra=1)
    bz.binarize_niblack(t, h, w, -0.2, out=out, precision="fp64", W=W)
    _, ref = oracle.niblack(img, h, w, k=-0.2, W=W)
    check_packed(out, ref, W)


@pytest.mark.parametrize("k,R", [(0.2, 128.0), (0.34, 100.0), (1.5, 64.0), (0.0, 128.0), (-0.3, 128.0)])
def test_sauvola_other_parameters(k, R):
    import paper_1905_13038_gb300 as bz
    img = image_for(150, 700, 7)
    t, W = to_device(img)
    out = bz.binarize_sauvola(t, 25, 41, k, R, precision="fp64")
    _, ref = oracle.sauvola(img, 25, 41, k=k, R=R)
    check_packed(out, ref, W)


def test_constant_and_checkerboard_ties():
    # Niblack on a constant image puts every pixel exactly on t (tie -> 0);
    # the checkerboard hits s = 127.5.  Ties must follow the FP64 rule.
    import paper_1905_13038_gb300 as bz
    img = np.full((60, 300), 77, np.uint8)
    t, W = to_device(img)
    check_packed(bz.binarize_niblack(t, 9, 9, -0.2), oracle.niblack(img, 9, 9, k=-0.2)[1], W)
    check_packed(bz.binarize_sauvola(t, 9, 9), oracle.sauvola(img, 9, 9)[1], W)
    ii, jj = np.indices((64, 320))
    cb = (((ii + jj) & 1) * 255).astype(np.uint8)
    t, W = to_device(cb)
    check_packed(bz.binarize_sauvola(t, 2, 2), oracle.sauvola(cb, 2, 2)[1], W)
    check_packed(bz.binarize_niblack(t, 4, 4, 0.3), oracle.niblack(cb, 4, 4, k=0.3)[1], W)


@pytest.mark.parametrize("H,W", [(3000, 1000), (60, 300)])
@pytest.mark.parametrize("precision", ["fp64", "fp64_direct"])
def test_flat_and_saturated_regions(H, W, precision):
    """Large constant areas (0, 255 and a mid gray) beside noisy text: windows
    with V = 0 and clusters of near-ties, decided in FP64 (spread over the
    warp in the window kernel); Sauvola with k > 0, k < 0 and a k so small
    that 1 - k rounds to 1, and Niblack."""
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 99 + H, stains=1)
    img[: H // 3, : W // 2] = 0
    img[H // 3: 2 * H // 3, W // 3:] = 255
    img[2 * H // 3:, : W // 4] = 128
    t, _ = to_device(img)
    for k in (0.5, -0.1, 1e-18):
        out = bz.binarize_sauvola(t, 15, 31, k, 128.0, precision=precision)
        check_packed(out, oracle.sauvola(img, 15, 31, k=k)[1], W)
    out = bz.binarize_niblack(t, 15, 31, -0.2, precision=precision)
    check_packed(out, oracle.niblack(img, 15, 31, k=-0.2)[1], W)


def test_fp32_path_and_report_small():
    import paper_1905_13038_gb300 as bz
    img = image_for(400, 900, 9)
    t, W = to_device(img)
    o32 = bz.binarize_sauvola(t, 31, 31, precision="fp32").cpu().numpy()
    _, ref = oracle.sauvola(img, 31, 31)
    flips = int((unpack(o32, W) != unpack(ref, W)).sum())
    rep_flips, maxdt = bz.binarize_precision_report(0, t, 31, 31, 0.5, 128.0)
    assert rep_flips == flips
    assert 0.0 < maxdt < 1e-3  # FP32 and FP64 thresholds differ somewhere, by little
    assert flips <= max(1, 1e-5 * img.size)


def test_invalid_arguments_rejected():
    import torch
    import paper_1905_13038_gb300 as bz
    img = torch.zeros((10, 16), dtype=torch.uint8, device="cuda")
    for h, w in [(0, 3), (3, 0), (512, 3), (3, 600)]:
        with pytest.raises(bz.BinarizeError) as e:
            bz.binarize_sauvola(img, h, w)
        assert e.value.status == 1
    with pytest.raises(bz.BinarizeError) as e:
        bz.binarize_sauvola(img, 3, 3, R=0.0)
    assert e.value.status == 1
    with pytest.raises(bz.BinarizeError) as e:
        bz.binarize_sauvola(img, 3, 3, k=float("nan"))
    assert e.value.status == 1
    # output overlapping the image (Sec. 3.2 forbids it)
    big = torch.zeros((20, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(bz.BinarizeError) as e:
        bz.binarize_sauvola(big[:10], 3, 3, out=big[5:15, :8])
    assert e.value.status == 2
    with pytest.raises(bz.BinarizeError) as e:
        bz.binarize_sauvola(img, 3, 3, out=torch.zeros((10, 1), dtype=torch.uint8, device="cuda"))
    assert e.value.status == 1


# Pages tall enough for the window kernel (not the small-page kernel) whose
# first and last tile columns run the pipelined path with clamped byte
# streams: a partial last tile, a partial last byte, W < 256, W = 8, pitch > W,
# stripe warm-up (h >= 48), the batched warm-up of short tiles and anchors of
# one and two words per lane.
EDGE_SHAPES = [
    # H, W, pitch, h, w
    (3000, 1000, 1000, 15, 15),
    (2800, 1028, 1032, 31, 31),
    (2600, 1100, 1104, 64, 9),
    (2500, 700, 704, 9, 125),
    (5000, 260, 264, 15, 31),
    (20000, 12, 16, 5, 5),
    (20000, 8, 8, 3, 3),
    (600, 777, 784, 31, 127),
    (2500, 1000, 1000, 9, 201),   # two anchor words per lane
    (700, 777, 784, 63, 255),     # two anchor words, stripe warm-up
]


@pytest.mark.parametrize("H,W,pitch,h,w", EDGE_SHAPES)
def test_edge_tiles_fp64_and_fp32(H, W, pitch, h, w):
    import paper_1905_13038_gb300 as bz
    img = image_for(H, W, 5 * H + W + h, pitch_extra=pitch - W)
    t, _ = to_device(img, W)
    for method, k in ((0, 0.5), (1, -0.2)):
        fn = bz.binarize_sauvola if method == 0 else bz.binarize_niblack
        args = (0.5, 128.0) if method == 0 else (-0.2,)
        _, ref = oracle.binarize(method, img, h, w, k, 128.0, W=W)
        out = out_buffer(H, W, extra=1)
        fn(t, h, w, *args, out=out, precision="fp64", W=W)
        check_packed(out, ref, W)
        o32 = fn(t, h, w, *args, precision="fp32", W=W).cpu().numpy()
        flips = int((unpack(o32, W) != unpack(ref, W)).sum())
        assert flips <= max(2, 1e-5 * H * W), flips


# ------------------------------------------------------------ full size ---
LARGE_WINDOWS = [(15, 15), (63, 63), (255, 255), (31, 127)]


@pytest.fixture(scope="module")
def large_page():
    return synth.large_page()


@pytest.mark.parametrize("h,w", LARGE_WINDOWS)
def test_large_page_sauvola_niblack_fp64(large_page, h, w):
    """4096 x 3072 page, the benchmarked launch configuration: full comparison
    with the row-band parallel oracle."""
    import paper_1905_13038_gb300 as bz
    img = large_page
    t, W = to_device(img)
    out = bz.binarize_sauvola(t, h, w, 0.5, 128.0, precision="fp64")
    ref = oracle.binarize_parallel(oracle.SAUVOLA, img, h, w, 0.5, 128.0)
    check_packed(out, ref, W)
    out = bz.binarize_niblack(t, h, w, -0.2, precision="fp64")
    ref = oracle.binarize_parallel(oracle.NIBLACK, img, h, w, -0.2, 128.0)
    check_packed(out, ref, W)


@pytest.mark.parametrize("h,w", LARGE_WINDOWS)
def test_large_page_sums_sampled(large_page, h, w):
    import paper_1905_13038_gb300 as bz
    img = large_page
    t, W = to_device(img)
    S1, S2, n = bz.window_sums(t, h, w)
    rng = np.random.default_rng(h * 1000 + w)
    ii = rng.integers(0, img.shape[0], 10000)
    jj = rng.integers(0, W, 10000)
    # include the four corners and the edges
    ii = np.concatenate([ii, [0, 0, img.shape[0] - 1, img.shape[0] - 1, 0, img.shape[0] // 2]])
    jj = np.concatenate([jj, [0, W - 1, 0, W - 1, W // 2, 0]])
    e1, e2, en = oracle.window_sums_at(img, h, w, ii, jj)
    np.testing.assert_array_equal(S1.cpu().numpy().view(np.uint32)[ii, jj], e1)
    np.testing.assert_array_equal(S2.cpu().numpy().view(np.uint64)[ii, jj], e2)
    np.testing.assert_array_equal(n.cpu().numpy().view(np.uint32)[ii, jj], en)


@pytest.mark.parametrize("method,k", [(0, 0.5), (1, -0.2)])
@pytest.mark.parametrize("h,w", LARGE_WINDOWS)
def test_large_page_fp32_flips(large_page, method, k, h, w):
    """BZ_FP32 flips against the FP64 oracle stay within 1e-5 of the pixels."""
    import paper_1905_13038_gb300 as bz
    img = large_page
    t, W = to_device(img)
    fn = bz.binarize_sauvola if method == 0 else bz.binarize_niblack
    args = (0.5, 128.0) if method == 0 else (-0.2,)
    o32 = fn(t, h, w, *args, precision="fp32").cpu().numpy()
    ref = oracle.binarize_parallel(method, img, h, w, k, 128.0)
    flips = int((unpack(o32, W) != unpack(ref, W)).sum())
    assert flips <= 1e-5 * img.size, flips
    rep, maxdt = bz.binarize_precision_report(method, t, h, w, k, 128.0)
    assert rep == flips
    assert 0.0 < maxdt < 1e-3
