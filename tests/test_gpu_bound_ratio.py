"""The certified FP32 threshold, tested against its own bound.

BZ_FP64 output equals the canonical FP64 decision because every pixel whose
FP32 threshold t32 lies within the certified bound E of its gray level is
re-decided in FP64.  That argument needs |t32 - t64| < E at every pixel;
binarize_bound_report measures max |t32 - t64| / E over an image, for every
evaluation form the kernels use, and it must stay below 1 (and above 0: the
two thresholds do differ).  Checked on the full 4096 x 3072 benchmark page at
its four windows for Sauvola and Niblack, on a page with flat and saturated
areas (windows with V = 0, clustered near-ties), and for the other Table 1
methods.  Also: the FP32 path of the Table 1 methods flips at most 1e-5 of
the pixels against the oracle, the bar of the Sauvola and Niblack FP32 tests.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import to_device, unpack

pytestmark = pytest.mark.gpu

WINDOWS = [(15, 15), (63, 63), (255, 255), (31, 127)]
TABLE1 = {
    oracle.WOLF: ("wolf", dict(k=0.5, R=128.0)),
    oracle.FENG: ("feng", dict(alpha1=0.88, k1=0.25, k2=0.04, gamma=2.0, R=128.0)),
    oracle.RAIS: ("rais", dict(k=0.3)),
    oracle.NICK: ("nick", dict(k=-0.1)),
    oracle.PHANSALKAR: ("phansalkar", dict(k=0.25, R=127.5, p=2.0, q=10.0 / 255.0)),
}


@pytest.fixture(scope="module")
def page(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    return to_device(synth.large_page())[0]


@pytest.mark.parametrize("h,w", WINDOWS)
@pytest.mark.parametrize("method,k", [(0, 0.5), (1, -0.2)])
def test_bound_ratio_on_the_benchmark_page(page, method, k, h, w):
    import paper_1905_13038_gb300 as bz
    r = bz.bound_report(method, page, h, w, [k, 128.0])
    assert 0.0 < r < 1.0, r


def test_bound_ratio_on_flat_and_saturated_areas(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    H, W = 700, 1300
    img = synth.document(H, W, 4242, stains=1)
    img[: H // 3, : W // 2] = 0
    img[H // 3: 2 * H // 3, W // 3:] = 255
    img[2 * H // 3:, : W // 4] = 128
    t, _ = to_device(img)
    for (method, k) in ((0, 0.5), (0, -0.1), (0, 1e-18), (1, -0.2)):
        for (h, w) in ((15, 31), (63, 63)):
            r = bz.bound_report(method, t, h, w, [k, 128.0])
            assert 0.0 <= r < 1.0, (method, k, h, w, r)


@pytest.mark.parametrize("method", sorted(TABLE1))
@pytest.mark.parametrize("h,w", [(15, 15), (63, 63), (31, 127)])
def test_bound_ratio_table1(page, method, h, w):
    import paper_1905_13038_gb300 as bz
    prm = list(oracle.params(**TABLE1[method][1]))
    r = bz.bound_report(method, page, h, w, prm)
    assert 0.0 < r < 1.0, r


@pytest.mark.parametrize("method", sorted(TABLE1))
def test_table1_fp32_flips_at_most_1e5(cuda_device, method):
    import paper_1905_13038_gb300 as bz
    bz.build()
    H, W = 1536, 2048
    img = synth.document(H, W, 77, stains=2)
    t, _ = to_device(img)
    name, kw = TABLE1[method]
    got = getattr(bz, f"binarize_{name}")(t, 31, 31, **kw, precision="fp32").cpu().numpy()
    bits, _ = oracle.binarize_ext(method, img, 31, 31, oracle.params(**kw))
    flips = int((unpack(got, W) != bits).sum())
    assert flips <= max(1, 1e-5 * H * W), flips
