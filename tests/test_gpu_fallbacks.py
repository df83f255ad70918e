"""bz_last_fp64_fallbacks counts the pixels the most recent BZ_FP64 call
decided in FP64: on a flat page every Niblack threshold equals the pixel
(t = m + k * 0), so every pixel is a near-tie and goes to the FP64 path; a
following call reports its own count, not a running total (the calls
alternate between two counters, each zeroed by the call before it)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_packed, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()


@pytest.mark.parametrize("H,W", [(300, 700), (1500, 3000)])  # small-page kernel, window kernel
def test_counts_are_per_call(H, W):
    import paper_1905_13038_gb300 as bz
    flat = np.full((H, W), 137, dtype=np.uint8)
    tf, _ = to_device(flat)
    page = synth.document(H, W, 5, stains=1)
    tp, _ = to_device(page)
    for rep in range(3):  # both counters, twice
        out = bz.binarize_niblack(tf, 15, 15, -0.2)
        assert bz.last_fp64_fallbacks() == H * W
        check_packed(out, oracle.niblack(flat, 15, 15, -0.2)[1], W)
        out = bz.binarize_sauvola(tp, 15, 15, 0.5, 128.0)
        n = bz.last_fp64_fallbacks()
        assert 0 <= n < H * W // 100
        check_packed(out, oracle.sauvola(page, 15, 15, 0.5, 128.0)[1], W)
    # an FP32 call leaves the count of the latest BZ_FP64 call
    bz.binarize_niblack(tf, 15, 15, -0.2)
    bz.binarize_niblack(tp, 15, 15, -0.2, precision="fp32")
    assert bz.last_fp64_fallbacks() == H * W


def test_multi_launch_calls_sum_their_launches():
    import paper_1905_13038_gb300 as bz
    H, W = 300, 700
    flat = np.full((H, W), 90, dtype=np.uint8)
    t, _ = to_device(flat)
    bz.binarize_inplace(1, t, 15, 15, k=-0.2, band_rows=40)  # 8 band launches
    assert bz.last_fp64_fallbacks() == H * W
    t, _ = to_device(flat)
    bz.binarize_inplace_cols(1, t, 15, 15, k=-0.2)  # 3 column-band launches
    assert bz.last_fp64_fallbacks() == H * W
