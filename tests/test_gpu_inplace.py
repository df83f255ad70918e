"""In-place binarization (Sec. 3.2: in-place needs the gray levels later
windows still read): the packed output written over the image equals the
oracle's output bit for bit, for several band heights down to the minimum
o = floor((h+1)/2), ragged last bands, one band, pitch > W, and FP64 / FP32;
the bytes after ceil(W/8) in each row keep their gray levels."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    return bz


CASES = [
    # H, W, h, w, band_rows
    (300, 600, 31, 31, 0),
    (300, 600, 31, 31, 16),    # the minimum band o = 16
    (301, 515, 15, 63, 37),    # ragged last band
    (97, 1030, 255, 255, 128),
    (50, 40, 7, 9, 1000),      # one band
    (1, 700, 5, 9, 3),
    (700, 1, 9, 5, 5),
]


@pytest.mark.parametrize("H,W,h,w,band", CASES)
@pytest.mark.parametrize("method", [0, 1])
def test_inplace_matches_oracle(H, W, h, w, band, method):
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 123 + H + W + h, stains=1 if min(H, W) > 20 else 0, pitch=W + 3)
    t, _ = to_device(img, W)
    k = 0.5 if method == 0 else -0.2
    bz.binarize_inplace(method, t, h, w, k=k, R=128.0, band_rows=band, W=W)
    got = t.cpu().numpy()
    _, packed = oracle.binarize(method, img, h, w, k, 128.0, W=W)
    cw = (W + 7) // 8
    np.testing.assert_array_equal(got[:, :cw], packed)
    np.testing.assert_array_equal(got[:, cw:], img[:, cw:])


def test_inplace_fp32_and_scratch_bound():
    import paper_1905_13038_gb300 as bz
    img = synth.document(200, 800, 5, stains=1)
    t, _ = to_device(img)
    ref = bz.binarize_sauvola(t, 31, 31, precision="fp32").cpu().numpy()
    bz.binarize_inplace(0, t, 31, 31, band_rows=40, precision="fp32")
    np.testing.assert_array_equal(t.cpu().numpy()[:, :100], ref)
    assert bz.inplace_scratch_bytes(200, 800, 31, 40) == 2 * 40 * 100
    assert bz.inplace_scratch_bytes(200, 800, 31, 0) == 2 * 200 * 100  # one band of 256 > H rows
    assert bz.inplace_scratch_bytes(200, 800, 31, 15) == -1


def test_inplace_rejects_short_bands():
    import paper_1905_13038_gb300 as bz
    img = synth.document(60, 80, 1)
    t, _ = to_device(img)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_inplace(0, t, 31, 31, band_rows=15)  # o = 16
