"""Serving loop: continuous batching with admission by device footprint.

Checks that a job gives the same result alone and in a mix of jobs that
arrive while others run (bitwise: the tile arithmetic never depends on the
batch), that host and device outputs agree, that cancellation, bounded waits
and admission refusal report their status codes, and that several jobs were
in flight at once."""
import time

import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = scff.Context(0)
    yield c
    c.close()


def small_jobs(n, seed=0):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        h = int(rng.integers(2, 7))
        m = W.molecule_dz_d(7000 + seed * 100 + i, h)
        S = int(rng.integers(1, 9))
        na = int(rng.integers(12, 40))
        jobs.append(W.Job(m, W.transition_matrices(7000 + i, S, m.nbf), W.axis(na, 20.0), W.axis(na + 3, 18.0),
                          W.axis(na + 5, 16.0)))
    return jobs


def alone(ctx, job, prec):
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    g = ctx.qgrid_product(job.qx, job.qy, job.qz)
    f, f2 = ctx.form_factor(b, t, g, precision=prec, f_out="cuda")
    ctx.sync()
    out = (f.clone(), f2.clone())
    ctx.release(g)
    ctx.release(b)
    return out


@pytest.mark.parametrize("prec", [scff.TF32X3, scff.FP16X2, scff.FP32])
def test_mixed_stream_equals_alone(ctx, prec):
    import torch
    jobs = small_jobs(14, seed=1)
    ref = [alone(ctx, j, prec) for j in jobs]
    srv = scff.Server(ctx, precision=prec, slots=2, max_batch_jobs=4)
    handles, outs, ids = [], [], []
    for k, job in enumerate(jobs):
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        handles.append((b, t))
        if k % 2 == 0:
            f = torch.full((job.n_states, job.nq, 2), float("nan"), device="cuda")
            f2 = torch.full((job.n_states, job.nq), float("nan"), device="cuda")
        else:
            f = torch.full((job.n_states, job.nq, 2), float("nan")).pin_memory()
            f2 = torch.full((job.n_states, job.nq), float("nan")).pin_memory()
        outs.append((f, f2))
        ids.append(srv.submit(b, t, job.qx, job.qy, job.qz, f, f2))
        if k % 5 == 4:
            time.sleep(0.002)          # arrivals while earlier batches run
    for i in ids:
        srv.wait(i, timeout_s=120)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["batches"] >= 2
    for (f, f2), (fr, f2r) in zip(outs, ref):
        assert torch.equal(f.cuda(), fr) and torch.equal(f2.cuda(), f2r)
    for b, t in handles:
        ctx.release(b)


def test_server_parity_cancel_timeout_admission(ctx):
    import torch
    job = W.scaled_job(W.config2(), 48)
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    srv = scff.Server(ctx, precision=scff.TF32X3, slots=1, max_batch_jobs=1, arena_bytes=256 << 20)
    f = torch.empty((job.n_states, job.nq, 2), device="cuda")
    i1 = srv.submit(b, t, job.qx, job.qy, job.qz, f)
    # queued behind i1 on the single slot: can be cancelled before admission
    g = torch.empty((job.n_states, job.nq, 2), device="cuda")
    i2 = srv.submit(b, t, job.qx, job.qy, job.qz, g)
    try:
        srv.cancel(i2)
        cancelled = True
    except scff.ScffError:
        cancelled = False            # already admitted: allowed, just not cancellable
    # bounded wait: a zero timeout on a job that may still run returns TIMEOUT or OK
    try:
        srv.wait(i1, timeout_s=0.0)
    except scff.ScffError as e:
        assert e.code == 6
    srv.wait(i1, timeout_s=120)
    if cancelled:
        with pytest.raises(scff.ScffError) as e:
            srv.wait(i2, timeout_s=1)
        assert e.value.code == 7
    else:
        srv.wait(i2, timeout_s=120)
    idx = W.subset_indices(job.nq, 400, 3)
    ref = oracle.grid_form_factor(job, idx)
    fc = f.cpu().numpy()
    fc = fc[..., 0] + 1j * fc[..., 1]
    assert np.max(np.abs(fc[:, idx] - ref)) / np.max(np.abs(ref)) < 1e-5
    # a job larger than the whole arena is refused
    big = W.config3()
    bb = ctx.basis(big.mol)
    tb = ctx.transitions(bb, big.T)
    fb = torch.empty((big.n_states, big.nq, 2), device="cuda")
    ib = srv.submit(bb, tb, big.qx, big.qy, big.qz, fb)
    with pytest.raises(scff.ScffError) as e:
        srv.wait(ib, timeout_s=30)
    assert e.value.code == 4
    st = srv.stats()
    srv.close()
    assert st["failed"] == 1
    ctx.release(b)
    ctx.release(bb)


@pytest.mark.parametrize("ratio", [16.0, 0.0])
def test_batch_cost_ratio_separates_large_and_small_jobs(ctx, ratio):
    # With a ratio of 16 a job ~100x more work than the first of a batch waits for the next
    # batch; with no limit (0, the default) all of them may share one.  Results equal the jobs alone.
    import torch
    small = small_jobs(3, seed=4)
    big = W.scaled_job(W.config3(), 40)
    jobs = small + [big]
    ref = [alone(ctx, j, scff.FP16X2) for j in jobs]
    srv = scff.Server(ctx, precision=scff.FP16X2, slots=1, max_batch_jobs=8, batch_cost_ratio=ratio)
    handles, outs, ids = [], [], []
    for job in jobs:
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        handles.append((b, t))
        f = torch.full((job.n_states, job.nq, 2), float("nan"), device="cuda")
        f2 = torch.full((job.n_states, job.nq), float("nan"), device="cuda")
        outs.append((f, f2))
    # hold the slot with a first batch so that the rest queue up together
    ids.append(srv.submit(*handles[0], jobs[0].qx, jobs[0].qy, jobs[0].qz, *outs[0]))
    for k in range(1, len(jobs)):
        ids.append(srv.submit(*handles[k], jobs[k].qx, jobs[k].qy, jobs[k].qz, *outs[k]))
    for i in ids:
        srv.wait(i, timeout_s=120)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs)
    if ratio <= 0:
        assert st["batches"] <= 2
    else:
        assert st["batches"] >= 2
    for (f, f2), (fr, f2r) in zip(outs, ref):
        assert torch.equal(f, fr) and torch.equal(f2, f2r)
    for b, _ in handles:
        ctx.release(b)
