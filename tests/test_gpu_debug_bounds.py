"""The bounds-checked debug build (libbinarize_debug.so, -DBZ_DEBUG).

compute-sanitizer is not available, so the library has a build in which
every global load and store of its kernels is checked against the extent of
the buffer it belongs to; an access outside is recorded in a status word and
skipped, never trapped.  This module runs the small-shape parity cases of the
other test modules (window sums and Sauvola / Niblack in every precision,
edge tiles with clamped byte streams, stripe warm-up, small pages, quantile,
min/max and Bernsen, Haar sums, the batch and the Table 1 kernels) through
the debug library, checks the results against the oracle as those modules
do, and requires the status word to stay 0 after each."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_packed, out_buffer, to_device, unpack
from test_gpu_minmax import SHAPES as MINMAX_SHAPES
from test_gpu_quantile import CASES as QUANTILE_CASES
from test_gpu_window import EDGE_SHAPES, SHAPES as WINDOW_SHAPES, image_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def debug_library(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    bz.use_library(debug=True)
    assert bz.debug_status() is not None, "not the debug build"
    yield bz
    bz.use_library(debug=False)


def clean(bz):
    import torch
    torch.cuda.synchronize()
    st = bz.debug_status(reset=True)
    assert st == (0, 0), f"out-of-extent access: status {st[0]:#x}, first address {st[1]:#x}"


@pytest.mark.parametrize("H,W,h,w", WINDOW_SHAPES)
@pytest.mark.parametrize("layout", ["aligned", "pitch+5", "misaligned"])
def test_window_path(debug_library, H, W, h, w, layout):
    bz = debug_library
    extra = 5 if layout == "pitch+5" else 0
    img = image_for(H, W, 100 + H + W, extra)
    t, _ = to_device(img, W, misalign=3 if layout == "misaligned" else 0)
    S1, S2, n = bz.window_sums(t, h, w, W=W)
    e1, e2, en = oracle.window_sums(img, h, w, W=W)
    np.testing.assert_array_equal(S1.cpu().numpy().view(np.uint32), e1)
    np.testing.assert_array_equal(S2.cpu().numpy().view(np.uint64), e2)
    for precision in ("fp64", "fp64_direct", "fp32"):
        out = out_buffer(H, W, extra=1)
        bz.binarize_sauvola(t, h, w, 0.5, 128.0, out=out, precision=precision, W=W)
        _, ref = oracle.sauvola(img, h, w, W=W)
        if precision == "fp32":
            assert int((unpack(out.cpu().numpy()[:, :(W + 7) // 8], W) != unpack(ref, W)).sum()) <= max(2, 1e-5 * H * W)
        else:
            check_packed(out, ref, W)
    clean(bz)


@pytest.mark.parametrize("H,W,pitch,h,w", EDGE_SHAPES)
def test_window_edge_tiles_and_stripes(debug_library, H, W, pitch, h, w):
    bz = debug_library
    img = image_for(H, W, 5 * H + W + h, pitch_extra=pitch - W)
    t, _ = to_device(img, W)
    _, ref = oracle.binarize(1, img, h, w, -0.2, 128.0, W=W)
    out = out_buffer(H, W, extra=1)
    bz.binarize_niblack(t, h, w, -0.2, out=out, precision="fp64", W=W)
    check_packed(out, ref, W)
    clean(bz)


def test_small_pages_and_large_windows(debug_library):
    bz = debug_library
    for (H, W, h, w) in ((384, 512, 31, 31), (200, 300, 63, 63), (1536, 2048, 255, 255), (1536, 2048, 15, 31)):
        img = synth.document(H, W, H + 7 * W, stains=1)
        t, _ = to_device(img)
        out = bz.binarize_sauvola(t, h, w, 0.5, 128.0, precision="fp64")
        check_packed(out, oracle.sauvola(img, h, w)[1], W)
        clean(bz)


@pytest.mark.parametrize("H,W,h,w,qn,qd", QUANTILE_CASES)
def test_quantile(debug_library, H, W, h, w, qn, qd):
    bz = debug_library
    img = synth.document(H, W, 400 + H, stains=1 if min(H, W) > 20 else 0, salt_pepper=0.02, pitch=W + 3)
    t, _ = to_device(img, W, misalign=2)
    Q = bz.window_quantile(t, h, w, qn, qd, W=W).cpu().numpy()
    np.testing.assert_array_equal(Q, oracle.window_quantile(img, h, w, qn, qd, W=W))
    out = out_buffer(H, W, extra=1)
    bz.binarize_quantile(t, h, w, qn, qd, 8, out=out, W=W)
    check_packed(out, oracle.binarize_quantile(img, h, w, qn, qd, 8, W=W)[1], W)
    clean(bz)


@pytest.mark.parametrize("H,W,h,w", MINMAX_SHAPES)
def test_minmax_and_bernsen(debug_library, H, W, h, w):
    bz = debug_library
    img = synth.document(H, W, 31 * H + W, pitch=W + 5)
    t, _ = to_device(img, W, misalign=1)
    mn, mx = bz.window_minmax(t, h, w, W=W)
    emn, emx = oracle.window_minmax(img, h, w, W=W)
    np.testing.assert_array_equal(mn.cpu().numpy(), emn)
    np.testing.assert_array_equal(mx.cpu().numpy(), emx)
    out = out_buffer(H, W, extra=1)
    bz.binarize_bernsen(t, h, w, 15, out=out, W=W)
    check_packed(out, oracle.binarize_bernsen(img, h, w, 15, W=W)[1], W)
    clean(bz)


@pytest.mark.parametrize("H,W", [(97, 600), (130, 515), (40, 33), (1, 700), (700, 1), (64, 1030)])
def test_haar(debug_library, H, W):
    bz = debug_library
    img = synth.document(H, W, 17 * H + W)
    t, _ = to_device(img)
    for name in bz.HAAR_FEATURES:
        rows, cols = bz.HAAR_FEATURES[name](24, 24)
        got = bz.haar_feature(t, rows, cols).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.haar(img, rows, cols))
    clean(bz)


def test_batch_and_table1(debug_library):
    bz = debug_library
    rng = np.random.default_rng(8)
    jobs, refs = [], []
    for b in range(10):
        H, W = int(rng.integers(1, 300)), int(rng.integers(1, 600))
        h = int(rng.choice([1, 15, 31, 63]))
        method = b % 3
        img = synth.document(H, W, 50 + b, salt_pepper=0.02 if method == 2 else 0.0, pitch=W + int(rng.integers(0, 9)))
        t, _ = to_device(img, W)
        jobs.append(bz.Job(t, method, h, h, k=0.5 if method == 0 else -0.2, R=128.0, q_num=1, q_den=2, offset=8, W=W))
        refs.append((oracle.sauvola(img, h, h, W=W)[1] if method == 0 else
                     oracle.niblack(img, h, h, W=W)[1] if method == 1 else
                     oracle.binarize_quantile(img, h, h, 1, 2, 8, W=W)[1], W))
    bz.binarize_batch(jobs, precision="fp64")
    for j, (ref, W) in zip(jobs, refs):
        check_packed(j.out, ref, W)
    clean(bz)
    img = synth.document(300, 700, 9)
    t, _ = to_device(img)
    out = bz.binarize_wolf(t, 31, 31, k=0.5, R=128.0, precision="fp64")
    check_packed(out, oracle.binarize_ext(oracle.WOLF, img, 31, 31, oracle.params(k=0.5, R=128.0))[1], 700)
    clean(bz)
