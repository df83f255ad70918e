"""binarize_batch_noalloc: the batched entry point for callers that cannot
allocate device memory when they call the library (all of their GPU memory is
pre-reserved by their own arena or caching allocator, or the call sits in a
latency-critical loop that must not wait on the driver's allocator).  Its
output must equal binarize_batch's, here bit for bit (the tolerance of every
binarization parity test), on two calls in a row: the second call is smaller
than the first and reuses the static work list the first one left behind.  In
the exact precisions a few jobs are also checked against the oracle, and a
call after the first must leave the device's free memory unchanged.

This file is collected last on purpose (test_zz_*), so that a run stopping at
the first failure has run every other test before it; it also passes alone.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import to_device

pytestmark = pytest.mark.gpu


def _jobs(seed, count):
    """`count` random jobs plus a Sauvola and a quantile job with h = w = 511 on
    small pages (window sums past 32 bits, windows far larger than the page).
    Returns (jobs, host images, job parameters)."""
    import paper_1905_13038_gb300 as bz
    rng = np.random.default_rng(seed)
    jobs, imgs, prm = [], [], []
    specs = []
    for b in range(count):
        H = int(rng.integers(1, 300))
        W = int(rng.integers(1, 600))
        h = int(rng.choice([1, 2, 15, 31, 63, 127]))
        w = int(rng.choice([1, 3, 15, 31, 64]))
        specs.append((H, W, h, w, int(rng.integers(0, 3))))
    specs.append((37, 45, 511, 511, 0))
    specs.append((29, 53, 511, 511, 2))
    for b, (H, W, h, w, method) in enumerate(specs):
        img = synth.document(H, W, seed * 7919 + b, salt_pepper=0.02 if method == 2 else 0.0,
                             pitch=W + int(rng.integers(0, 9)))
        t, _ = to_device(img, W, misalign=int(rng.integers(0, 2)))
        if method == 0:
            jobs.append(bz.Job(t, bz.SAUVOLA, h, w, k=0.5, R=128.0, W=W))
        elif method == 1:
            jobs.append(bz.Job(t, bz.NIBLACK, h, w, k=-0.2, W=W))
        else:
            jobs.append(bz.Job(t, bz.QUANTILE, h, w, q_num=1, q_den=10, offset=8, W=W))
        imgs.append(img)
        prm.append((W, h, w, method))
    return jobs, imgs, prm


def _call_noalloc_cabi(jobs, precision, stream=None):
    """Through the C ABI directly: binarize_batch_noalloc(jobs, n, precision, stream)."""
    import torch
    import paper_1905_13038_gb300 as bz
    lib = bz._load()
    arr = (bz._JobC * len(jobs))(*[j.c for j in jobs])
    s = torch.cuda.current_stream() if stream is None else stream
    return lib.binarize_batch_noalloc(arr, len(jobs), precision, ctypes.c_void_p(s.cuda_stream))


def _oracle_packed(img, W, h, w, method):
    if method == 0:
        return oracle.sauvola(img, h, w, k=0.5, R=128.0, W=W)[1]
    if method == 1:
        return oracle.niblack(img, h, w, k=-0.2, W=W)[1]
    return oracle.binarize_quantile(img, h, w, 1, 10, 8, W=W)[1]


@pytest.mark.parametrize("precision", [0, 1, 2])  # BZ_FP64, BZ_FP32, BZ_FP64_DIRECT
def test_noalloc_batch_matches_batch_twice_in_a_row(cuda_device, precision):
    import torch
    import paper_1905_13038_gb300 as bz
    bz.build()
    for call, (seed, count) in enumerate(((11, 37), (12, 23))):  # the second call is smaller
        jobs, imgs, prm = _jobs(seed, count)
        ref, _, _ = _jobs(seed, count)  # same images and parameters, own outputs
        bz.binarize_batch(ref, precision=precision)
        for j in jobs:
            j.out.fill_(0xAB)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call_noalloc_cabi(jobs, precision)
        torch.cuda.synchronize()
        assert st == 0, bz.status_string(st)
        if call > 0:  # the first call on a device may load the library's module
            assert torch.cuda.mem_get_info()[0] == free0, "a call after the first changed free memory"
        for a, b in zip(jobs, ref):
            wb = (a.c.W + 7) // 8
            np.testing.assert_array_equal(a.out.cpu().numpy()[:, :wb], b.out.cpu().numpy()[:, :wb])
        # the exact precisions decide every pixel as the oracle does: check the
        # two h = w = 511 jobs and the first three others directly
        for idx in [0, 1, 2, len(jobs) - 2, len(jobs) - 1]:
            W, h, w, method = prm[idx]
            if precision == 1 and method != 2:
                continue  # FP32 Sauvola/Niblack are graded by flip counts elsewhere
            wb = (W + 7) // 8
            got = jobs[idx].out.cpu().numpy()[:, :wb]
            np.testing.assert_array_equal(got, _oracle_packed(imgs[idx], W, h, w, method)[:, :wb])


def test_noalloc_rejects_more_jobs_than_the_static_list(cuda_device):
    import paper_1905_13038_gb300 as bz
    bz.build()
    lib = bz._load()
    arr = (bz._JobC * 513)()
    st = lib.binarize_batch_noalloc(arr, 513, 0, None)
    assert st == 1  # BZ_EINVAL, nothing launched


def test_noalloc_refuses_stream_capture(cuda_device):
    """A captured call would replay whatever work list the latest call staged
    in the static host buffer, so a capturing stream is refused (BZ_EINVAL)
    and nothing is enqueued."""
    import torch
    import paper_1905_13038_gb300 as bz
    bz.build()
    jobs, _, _ = _jobs(21, 3)
    _call_noalloc_cabi(jobs, 0)  # first call outside capture
    torch.cuda.synchronize()
    x = torch.zeros(16, device="cuda")
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            x += 1  # something to capture
            st = _call_noalloc_cabi(jobs, 0, stream)
    assert st == 1  # BZ_EINVAL
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
