"""In-place binarization (Sec. 3.2: in-place needs the gray levels later
windows still read): the packed output written over the image equals the
oracle's output bit for bit, for several band heights down to the minimum
o = floor((h+1)/2), ragged last bands, one band, pitch > W, and FP64 / FP32;
the bytes after ceil(W/8) in each row keep their gray levels.  The same for
the column-band version (Sec. 3.3's exchanged axes), including the widest
window a 256-column band allows (w = 450: the first band's output bytes end
exactly where the second band's windows begin) and served in-place requests
mixed with separate-output ones."""
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


COL_CASES = [
    # H, W, h, w, band_cols
    (300, 600, 31, 31, 0),      # three bands, the last one ragged
    (301, 1030, 15, 450, 0),    # 256-column bands at their widest window
    (120, 1100, 9, 451, 0),     # 512-column bands
    (97, 1030, 255, 511, 0),
    (64, 1500, 31, 31, 768),    # explicit band width
    (50, 40, 7, 9, 0),          # one band narrower than 256
    (1, 700, 5, 9, 0),
    (700, 1, 9, 5, 0),
]


@pytest.mark.parametrize("H,W,h,w,band", COL_CASES)
@pytest.mark.parametrize("method", [0, 1])
def test_inplace_cols_matches_oracle(H, W, h, w, band, method):
    import paper_1905_13038_gb300 as bz
    img = synth.document(H, W, 321 + H + W + w, stains=1 if min(H, W) > 20 else 0, pitch=W + 5)
    t, _ = to_device(img, W, misalign=(H + W) % 2)
    k = 0.5 if method == 0 else -0.2
    bz.binarize_inplace_cols(method, t, h, w, k=k, R=128.0, band_cols=band, W=W)
    got = t.cpu().numpy()
    _, packed = oracle.binarize(method, img, h, w, k, 128.0, W=W)
    cw = (W + 7) // 8
    np.testing.assert_array_equal(got[:, :cw], packed)
    np.testing.assert_array_equal(got[:, cw:], img[:, cw:])


def test_inplace_cols_fp32_and_band_checks():
    import paper_1905_13038_gb300 as bz
    img = synth.document(200, 800, 6, stains=1)
    t, _ = to_device(img)
    ref = bz.binarize_sauvola(t, 31, 31, precision="fp32").cpu().numpy()
    bz.binarize_inplace_cols(0, t, 31, 31, precision="fp32")
    np.testing.assert_array_equal(t.cpu().numpy()[:, :100], ref)
    t2, _ = to_device(img)
    for bad in (128, 300):  # not a multiple of 256
        with pytest.raises(bz.BinarizeError):
            bz.binarize_inplace_cols(0, t2, 31, 31, band_cols=bad)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_inplace_cols(0, t2, 31, 451, band_cols=256)  # l = 226 needs 512
    np.testing.assert_array_equal(t2.cpu().numpy(), img)  # nothing written


def test_server_mixes_inplace_and_separate_output_jobs():
    """Served in-place requests (out == image) under a budget that admits some
    only with column bands, mixed with separate-output Sauvola, Niblack and
    quantile requests: every result equals the oracle's."""
    import torch
    rng = np.random.default_rng(77)
    imgs, jobs, refs = [], [], []
    import paper_1905_13038_gb300 as bz
    for b in range(24):
        kind = b % 4  # 0, 1: in-place Sauvola / Niblack; 2: Sauvola; 3: quantile
        H = int(rng.integers(1, 320))
        W = int(rng.integers(1, 2100 if kind < 2 else 700))
        h = int(rng.choice([1, 15, 31, 63, 255]))
        w = int(rng.choice([1, 15, 31, 64, 255, 449]))
        img = synth.document(H, W, 900 + b, stains=1 if min(H, W) > 30 else 0,
                             salt_pepper=0.02 if kind == 3 else 0.0, pitch=W + int(rng.integers(0, 9)))
        t, _ = to_device(img, W, misalign=int(rng.integers(0, 2)))
        if kind in (0, 1):
            k = 0.5 if kind == 0 else -0.2
            jobs.append(bz.Job(t, bz.SAUVOLA if kind == 0 else bz.NIBLACK, h, w, k=k, R=128.0, W=W,
                               inplace=True))
            refs.append(("inplace", oracle.binarize(kind, img, h, w, k, 128.0, W=W)[1], W, img))
        elif kind == 2:
            jobs.append(bz.Job(t, bz.SAUVOLA, h, w, k=0.5, R=128.0, W=W))
            refs.append(("out", oracle.sauvola(img, h, w, 0.5, 128.0, W=W)[1], W, img))
        else:
            jobs.append(bz.Job(t, bz.QUANTILE, h, w, q_num=1, q_den=2, offset=8, W=W))
            refs.append(("out", oracle.binarize_quantile(img, h, w, 1, 2, 8, W=W)[1], W, img))
    # the largest in-place request fits only with column bands
    ip = [j for j in jobs if j.out is j.image]
    need_rows = [j.c.H * j.c.in_pitch + bz.inplace_scratch_bytes(j.c.H, j.c.W, j.c.h) for j in ip]
    need_cols = [j.c.H * j.c.in_pitch + bz.inplace_cols_scratch_bytes(j.c.H, j.c.W, j.c.w) for j in ip]
    big = int(np.argmax(need_rows))
    assert need_cols[big] < need_rows[big]
    budget = need_cols[big]
    others = [j.c.H * (j.c.in_pitch + j.c.out_pitch) for j in jobs if j.out is not j.image]
    assert max(others) <= budget
    srv = bz.Server(hbm_budget_bytes=budget, max_slots=8)
    try:
        tickets = [srv.submit(j) for j in jobs]
        for t in tickets:
            assert srv.wait(t, 60000) == 0
    finally:
        srv.close()
    torch.cuda.synchronize()
    for job, (kind, ref, W, img) in zip(jobs, refs):
        cw = (W + 7) // 8
        if kind == "inplace":
            got = job.image.cpu().numpy()
            np.testing.assert_array_equal(got[:, :cw], ref)
            np.testing.assert_array_equal(got[:, cw:W], img[:, cw:W])
        else:
            np.testing.assert_array_equal(job.out.cpu().numpy()[:, :cw], ref)


def test_server_rejects_inplace_job_over_budget_and_batch_rejects_inplace():
    import paper_1905_13038_gb300 as bz
    img = synth.document(100, 900, 8)
    t, _ = to_device(img)
    job = bz.Job(t, bz.SAUVOLA, 15, 15, inplace=True)
    least = 100 * 900 + bz.inplace_cols_scratch_bytes(100, 900, 15)
    srv = bz.Server(hbm_budget_bytes=least - 1, max_slots=2)
    try:
        with pytest.raises(bz.BinarizeError) as e:
            srv.submit(job)
        assert e.value.status == 4  # BZ_EBUDGET
    finally:
        srv.close()
    q = bz.Job(t, bz.QUANTILE, 15, 15, inplace=True)
    srv = bz.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    try:
        with pytest.raises(bz.BinarizeError) as e:
            srv.submit(q)  # in place only for Sauvola / Niblack
        assert e.value.status == 1
    finally:
        srv.close()
    with pytest.raises(bz.BinarizeError) as e:
        bz.binarize_batch([job])
    assert e.value.status == 2  # BZ_EOVERLAP
