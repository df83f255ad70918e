"""Autotuner on the GPU: every launch configuration the tuner may choose for
a page gives the oracle's bits (the configurations only split the work
differently), the explicit tuning calls return the stored winner, and the
cache they write reads back."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import check_packed, out_buffer, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def tmp_cache(cuda_device, tmp_path):
    import paper_1905_13038_gb300 as bz
    bz.build()
    path = tmp_path / "tune.json"
    bz.tune_load(str(path))  # empty cache; tuning saves here
    yield path
    bz.tune_clear()


def _gpu_tag():
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name}/{p.multi_processor_count}"


@pytest.mark.parametrize("h,w", [(15, 31), (63, 63)])
def test_every_window_configuration_matches_the_oracle(h, w, tmp_cache):
    import paper_1905_13038_gb300 as bz
    H, W = 1536, 2048
    img = synth.document(H, W, 20261205, stains=2)
    t, _ = to_device(img)
    _, ref = oracle.sauvola(img, h, w, k=0.5, R=128.0)
    out, cfg = bz.autotune_window(bz.SAUVOLA, t, h, w, k=0.5, R=128.0, precision="fp64")
    check_packed(out, ref, W)
    assert cfg["tile_h"] >= 1 and cfg["us"] > 0.0
    key = bz.tune_key(_gpu_tag(), "window", 0, h, w, H, W)
    assert bz.tune_get(key)["tile_h"] == cfg["tile_h"]
    # the candidates of the search, forced one by one through the cache
    _, plan = bz.tune_window_plan(_gpu_tag(), "fp64", H, W, h, w, 1)  # any SM count: tile_h is cached
    th0 = cfg["tile_h"]
    for tile_h in sorted({max(1, th0 // 2), th0, th0 + 1, 2 * th0, 7}):
        for edge in (0.5, 0.82, 1.0):
            for stripes in ((0, 1) if h >= 48 else (0,)):
                bz.tune_set(key, tile_h, edge, stripes, 1.0)
                o = out_buffer(H, W, extra=1)
                bz.binarize_sauvola(t, h, w, k=0.5, R=128.0, out=o, precision="fp64")
                check_packed(o, ref, W)


def test_quantile_configurations_match_the_oracle(tmp_cache):
    import paper_1905_13038_gb300 as bz
    H, W = 600, 700
    img = synth.document(H, W, 777, salt_pepper=0.02)
    t, _ = to_device(img)
    _, ref = oracle.binarize_quantile(img, 31, 31, 1, 10, 8)
    out, cfg = bz.autotune_quantile(t, 31, 31, 1, 10, 8)
    check_packed(out, ref, W)
    key = bz.tune_key(_gpu_tag(), "quantile", 0, 31, 31, H, W)
    assert bz.tune_get(key)["tile_h"] == cfg["tile_h"] >= 1
    for tile_h in (1, 5, 64, 600):
        bz.tune_set(key, tile_h, 1.0, -1, 1.0)
        o = out_buffer(H, W, extra=1)
        bz.binarize_quantile(t, 31, 31, 1, 10, 8, out=o)
        check_packed(o, ref, W)


def test_batch_tuning_keeps_the_bits(tmp_cache):
    import paper_1905_13038_gb300 as bz
    rng = np.random.default_rng(3)
    specs, imgs, jobs = [], [], []
    for b in range(12):
        H, W = int(rng.integers(50, 400)), int(rng.integers(50, 500))
        h = int(rng.choice([15, 31, 63]))
        method = int(rng.integers(0, 3))
        img = synth.document(H, W, 900 + b, salt_pepper=0.02 if method == 2 else 0.0)
        t, _ = to_device(img)
        jobs.append(bz.Job(t, method, h, h, k=0.5 if method == 0 else -0.2, R=128.0, q_num=1, q_den=2, offset=8))
        specs.append((H, W, h, method))
        imgs.append(img)
    cfg = bz.autotune_batch(jobs, precision="fp64")
    assert 1 <= cfg["win_mult"] <= 16 and 1 <= cfg["quant_mult"] <= 16
    for j, img, (H, W, h, method) in zip(jobs, imgs, specs):
        if method == 0:
            ref = oracle.sauvola(img, h, h, k=0.5, R=128.0)[1]
        elif method == 1:
            ref = oracle.niblack(img, h, h, k=-0.2)[1]
        else:
            ref = oracle.binarize_quantile(img, h, h, 1, 2, 8)[1]
        check_packed(j.out, ref, W)


def test_tuned_cache_file_reads_back(tmp_cache):
    import paper_1905_13038_gb300 as bz
    img = synth.document(2048, 2048, 5)  # large enough for the window kernel (not the small-page one)
    t, _ = to_device(img)
    bz.autotune_window(bz.NIBLACK, t, 15, 15, k=-0.2, precision="fp32")
    assert tmp_cache.exists()
    assert bz.tune_load(str(tmp_cache)) >= 1
