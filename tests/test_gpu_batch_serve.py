"""Batched (one persistent graph launch) and served (continuous batching)
execution: every result equals the single-image call and the oracle, alone
and in the mix."""
import os

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


def make_jobs(count, seed, with_quantile=True):
    import paper_1905_13038_gb300 as bz
    rng = np.random.default_rng(seed)
    jobs, refs = [], []
    for b in range(count):
        H = int(rng.integers(1, 400))
        W = int(rng.integers(1, 700))
        h = int(rng.choice([1, 2, 15, 31, 63, 127, 255]))
        w = int(rng.choice([1, 3, 15, 31, 64, 127]))
        method = int(rng.integers(0, 3 if with_quantile else 2))
        img = synth.document(H, W, seed * 1000 + b, stains=1 if min(H, W) > 30 else 0,
                             salt_pepper=0.02 if method == 2 else 0.0, pitch=W + int(rng.integers(0, 9)))
        t, _ = to_device(img, W, misalign=int(rng.integers(0, 2)))
        if method == 0:
            job = bz.Job(t, bz.SAUVOLA, h, w, k=0.5, R=128.0, W=W)
            ref = oracle.sauvola(img, h, w, 0.5, 128.0, W=W)[1]
        elif method == 1:
            job = bz.Job(t, bz.NIBLACK, h, w, k=-0.2, W=W)
            ref = oracle.niblack(img, h, w, -0.2, W=W)[1]
        else:
            job = bz.Job(t, bz.QUANTILE, h, w, q_num=1, q_den=2, offset=8, W=W)
            ref = oracle.binarize_quantile(img, h, w, 1, 2, 8, W=W)[1]
        jobs.append(job)
        refs.append((ref, W, img, method, h, w))
    return jobs, refs


def test_batch_matches_oracle_and_single_calls():
    import torch
    import paper_1905_13038_gb300 as bz
    jobs, refs = make_jobs(40, 1)
    bz.binarize_batch(jobs, precision="fp64")
    torch.cuda.synchronize()
    for job, (ref, W, img, method, h, w) in zip(jobs, refs):
        check_packed(job.out, ref, W)
        # the single-image call gives the same bytes
        single = (bz.binarize_sauvola(job.image, h, w, 0.5, 128.0, W=W) if method == 0 else
                  bz.binarize_niblack(job.image, h, w, -0.2, W=W) if method == 1 else
                  bz.binarize_quantile(job.image, h, w, 1, 2, 8, W=W))
        np.testing.assert_array_equal(single.cpu().numpy(), job.out.cpu().numpy()[:, :single.shape[1]])


def test_batch_repeated_launches_and_precisions():
    import torch
    import paper_1905_13038_gb300 as bz
    jobs, refs = make_jobs(12, 2, with_quantile=False)
    for prec in ("fp64", "fp32", "fp64_direct", "fp64"):
        for j in jobs:
            j.out.fill_(0xAB)
        bz.binarize_batch(jobs, precision=prec)
        torch.cuda.synchronize()
        if prec != "fp32":
            for job, (ref, W, *_r) in zip(jobs, refs):
                check_packed(job.out, ref, W)


def test_batch_rejects_invalid_job_without_launching():
    import torch
    import paper_1905_13038_gb300 as bz
    jobs, _ = make_jobs(3, 3, with_quantile=False)
    bad = bz.Job(jobs[0].image, bz.SAUVOLA, 3, 3, R=-1.0)
    for j in jobs:
        j.out.fill_(0xAB)
    with pytest.raises(bz.BinarizeError):
        bz.binarize_batch(jobs + [bad])
    torch.cuda.synchronize()
    for j in jobs:
        assert (j.out.cpu().numpy() == 0xAB).all()


def test_server_results_same_alone_and_in_mix():
    import torch
    import paper_1905_13038_gb300 as bz
    jobs, refs = make_jobs(60, 4)
    srv = bz.Server(hbm_budget_bytes=2_000_000, max_slots=16)
    try:
        tickets = [srv.submit(j) for j in jobs]
        for t in tickets:
            assert srv.wait(t, 60000) == 0
    finally:
        srv.close()
    torch.cuda.synchronize()
    for job, (ref, W, *_r) in zip(jobs, refs):
        check_packed(job.out, ref, W)


def test_server_budget_cancel_timeout_and_faults(monkeypatch):
    import paper_1905_13038_gb300 as bz
    jobs, _ = make_jobs(6, 5, with_quantile=False)
    srv = bz.Server(hbm_budget_bytes=1_000, max_slots=2)
    try:
        big = [j for j in jobs if j.c.H * (j.c.in_pitch + j.c.out_pitch) > 1_000]
        if big:
            with pytest.raises(bz.BinarizeError) as e:
                srv.submit(big[0])
            assert e.value.status == 4  # BZ_EBUDGET
    finally:
        srv.close()
    # cancellation: a cancelled ticket reports BZ_ECANCELLED (queued or running)
    srv = bz.Server(hbm_budget_bytes=1 << 30, max_slots=1)
    try:
        ts = [srv.submit(j) for j in jobs]
        assert srv.cancel(ts[-1]) == 0
        assert srv.wait(ts[-1], 60000) == 8
        for t in ts[:-1]:
            assert srv.wait(t, 60000) == 0
    finally:
        srv.close()
    # host-side fault injection: a failing launch and a late completion
    monkeypatch.setenv("BZ_FAULT", "launch")
    srv = bz.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    try:
        t = srv.submit(jobs[0])
        assert srv.wait(t, 60000) == 5  # BZ_ECUDA
    finally:
        srv.close()
    # late completions: a wait on a running request times out without
    # waiting for the GPU; the request is cancelled and keeps its ticket until
    # a later wait reports BZ_ECANCELLED.  A request still queued when its wait
    # times out is dropped (its ticket is then unknown).
    monkeypatch.setenv("BZ_FAULT", "slow:1500")
    srv = bz.Server(hbm_budget_bytes=1 << 30, max_slots=1)
    try:
        t0 = srv.submit(jobs[0])
        t1 = srv.submit(jobs[1])
        import time
        time.sleep(0.2)  # t0 is running (slowly), t1 waits for the one slot
        start = time.perf_counter()
        assert srv.wait(t0, 50) == 6  # BZ_ETIMEOUT
        assert srv.wait(t1, 50) == 6  # BZ_ETIMEOUT, dropped while queued
        assert time.perf_counter() - start < 1.0  # neither waited for the GPU
        assert srv.wait(t1, 0) == 1  # BZ_EINVAL: no such ticket any more
        assert srv.wait(t0, 60000) == 8  # BZ_ECANCELLED once the GPU is done
    finally:
        srv.close()
    monkeypatch.delenv("BZ_FAULT")
