"""binarize_host: Sauvola / Niblack straight from host memory (upload,
binarize, download on the caller's stream) equals the oracle bit for bit,
for pinned and pageable images, pitch > W, small and large pages, and a
sequence of calls in flight on one stream (the upload of one call overlapping
the compute of the previous one)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    return bz


@pytest.mark.parametrize("H,W,h,w,method", [(384, 512, 31, 31, 0), (97, 600, 15, 15, 1),
                                            (1, 700, 5, 9, 0), (300, 1030, 255, 255, 0),
                                            (3072, 4096, 63, 63, 0)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_matches_oracle(H, W, h, w, method, pinned):
    import torch
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 17 + H + W, stains=1 if min(H, W) > 20 else 0, pitch=W + 3)
    t = torch.from_numpy(img)
    if pinned:
        t = t.pin_memory()
    k = 0.5 if method == 0 else -0.2
    got = bz.binarize_host(method, t, h, w, k=k, W=W).numpy()
    _, ref = oracle.binarize(method, img, h, w, k, 128.0, W=W)
    np.testing.assert_array_equal(got, ref)


def test_host_calls_in_flight_on_one_stream():
    import torch
    import paper_1905_13038_gb300 as bz
    s = torch.cuda.Stream()
    pages = [torch.from_numpy(synth.document(700, 900, 40 + q, stains=1)).pin_memory() for q in range(4)]
    outs = [bz.binarize_host(0, p, 31, 31, stream=s, sync=False) for p in pages]
    s.synchronize()
    for p, o in zip(pages, outs):
        _, ref = oracle.sauvola(p.numpy(), 31, 31)
        np.testing.assert_array_equal(o.numpy(), ref)


def test_host_growing_pages_in_flight():
    # the library's device staging buffers grow while earlier calls are
    # still in flight; every call must still see its own page
    import torch
    import paper_1905_13038_gb300 as bz
    s = torch.cuda.Stream()
    shapes = [(100, 200), (700, 900), (50, 3000), (1200, 1100), (300, 64), (1200, 1100)]
    pages = [torch.from_numpy(synth.document(H, W, 90 + q, stains=1)).pin_memory()
             for q, (H, W) in enumerate(shapes)]
    outs = [bz.binarize_host(0, p, 15, 31, stream=s, sync=False) for p in pages]
    s.synchronize()
    for p, o in zip(pages, outs):
        _, ref = oracle.sauvola(p.numpy(), 15, 31)
        np.testing.assert_array_equal(o.numpy(), ref)


@pytest.mark.parametrize("H,W,pitch", [(3072, 4096, 4096), (500, 777, 784), (97, 600, 603)])
def test_host_multi_windows(H, W, pitch):
    """One upload, several windows: each output equals the oracle's."""
    import torch
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 7 + H + W, stains=1, pitch=pitch)
    t = torch.from_numpy(img).pin_memory()
    windows = [(15, 15), (63, 63), (31, 127), (5, 9)]
    if H >= 3000:
        windows.append((255, 255))
    outs = bz.binarize_host_multi(0, t, windows, k=0.5, W=W)
    for (h, w), o in zip(windows, outs):
        _, ref = oracle.binarize(0, img, h, w, 0.5, 128.0, W=W)
        np.testing.assert_array_equal(o.numpy(), ref)


def test_host_multi_in_flight():
    import torch
    import paper_1905_13038_gb300 as bz
    s = torch.cuda.Stream()
    pages = [torch.from_numpy(synth.document(600 + 50 * q, 700, 60 + q, stains=1)).pin_memory()
             for q in range(4)]
    windows = [(15, 15), (31, 31)]
    res = [bz.binarize_host_multi(1, p, windows, k=-0.2, stream=s, sync=False) for p in pages]
    s.synchronize()
    for p, outs in zip(pages, res):
        for (h, w), o in zip(windows, outs):
            _, ref = oracle.niblack(p.numpy(), h, w, k=-0.2)
            np.testing.assert_array_equal(o.numpy(), ref)


def test_host_multi_rejects_bad_arguments():
    import torch
    import paper_1905_13038_gb300 as bz
    t = torch.zeros((10, 16), dtype=torch.uint8)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_host_multi(0, t, [(3, 3), (0, 3)])  # an invalid window
    out = torch.zeros((10, 2), dtype=torch.uint8)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_host_multi(0, t, [(3, 3), (5, 5)], outs=[out, out])  # outputs overlap


def test_host_rejects_bad_arguments():
    import torch
    import paper_1905_13038_gb300 as bz
    t = torch.zeros((10, 16), dtype=torch.uint8)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_host(2, t, 3, 3)  # quantile is not a host method
    with pytest.raises(bz.BinarizeError):
        bz.binarize_host(0, t, 0, 3)
