"""Batched persistent launches (plans): each job's result in a batch must be
identical to the same job run alone (the tile arithmetic never depends on
the rest of the batch), with one or several workspace groups, direct and
CUDA-graph replay, and within the parity tolerance of the oracle."""
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


def mixed_jobs():
    j1 = W.config1()
    j2 = W.scaled_job(W.config2(), 40)
    j3 = W.Job(j1.mol, W.transition_matrices(55, 5, j1.mol.nbf), W.axis(9, 7.0), W.axis(33, 8.0), W.axis(70, 9.0))
    m4 = W.molecule_dz_d(4077, 6)
    j4 = W.Job(m4, W.transition_matrices(4077, 4, m4.nbf), W.axis(30, 20.0), W.axis(30, 20.0), W.axis(30, 20.0))
    # pure d and f shells (pair classes up to degree 6, T expanded to Cartesian components)
    m5 = W.molecule_pol_f(4099, 2, pure=W.PURE_D | W.PURE_F)
    j5 = W.Job(m5, W.transition_matrices(4099, 3, m5.nbf), W.axis(20, 12.0), W.axis(26, 12.0), W.axis(17, 12.0))
    return [j1, j2, j3, j4, j5]


def make_batch(ctx, jobs, prec):
    import torch
    tdt = torch.float64 if prec == scff.FP64 else torch.float32
    specs, handles = [], []
    for k, job in enumerate(jobs):
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        g = ctx.qgrid_product(job.qx, job.qy, job.qz)
        f = torch.full((job.n_states, job.nq, 2), float("nan"), dtype=tdt, device="cuda")
        f2 = torch.full((job.n_states, job.nq), float("nan"), dtype=tdt, device="cuda")
        specs.append((b, t, g, f, f2, 1.0 + 0.25 * k))
        handles.append((b, t, g))
    return specs, handles


@pytest.mark.parametrize("prec", [scff.TF32X3, scff.BF16X3, scff.FP16X2, scff.FP32, scff.FP64])
@pytest.mark.parametrize("split", [False, True])
def test_batch_equals_alone(ctx, prec, split):
    import torch
    if split and prec in (scff.FP32, scff.FP64):
        pytest.skip("direct-path jobs are not grouped")
    jobs = mixed_jobs()
    specs, handles = make_batch(ctx, jobs, prec)
    plan = ctx.plan(specs, precision=prec)
    info = plan.info()
    if split:
        # a workspace below the batch's total but above its largest job: several groups
        total = info["device_bytes"]
        plan.release()
        plan = ctx.plan(specs, precision=prec, workspace_bytes=int(0.85 * total))
        info = plan.info()
    if prec not in (scff.FP32, scff.FP64):
        assert info["tc_jobs"] == len(jobs)
        assert (info["groups"] > 1) == split
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.run(stream)
    stream.synchronize()
    ctx.sync(stream)
    batched = [(s[3].clone(), s[4].clone()) for s in specs]
    # replay through a captured graph: same numbers
    for s in specs:
        s[3].fill_(float("nan"))
    plan.run_graph(stream)
    plan.run_graph(stream)
    stream.synchronize()
    for s, (f, f2) in zip(specs, batched):
        assert torch.equal(s[3], f) and torch.equal(s[4], f2)
    # each job alone through the single-job entry point: bitwise the same
    for (b, t, g), s, (f, f2), job in zip(handles, specs, batched, jobs):
        fa, f2a = ctx.form_factor(b, t, g, precision=prec, scale=s[5], f_out="cuda")
        ctx.sync()
        assert torch.equal(fa, f) and torch.equal(f2a, f2)
        idx = W.subset_indices(job.nq, 300, 9)
        ref = oracle.grid_form_factor(job, idx, scale=s[5])
        fc = f.cpu().numpy()
        fc = fc[..., 0] + 1j * fc[..., 1]
        err = np.max(np.abs(fc[:, idx] - ref)) / np.max(np.abs(ref))
        assert err < (1e-10 if prec == scff.FP64 else 1e-5)
    plan.release()


@pytest.mark.parametrize("prec", [scff.FP16X2, scff.TF32X3, scff.BF16X2])
def test_zstaged_batch_equals_alone(ctx, prec):
    # every job's z axis is a multiple of 128, so the group runs the variant whose generators
    # read Z and Y staged in shared memory; odd and even x, ny not a multiple of anything
    import torch
    m1 = W.molecule_dz_d(4101, 3)
    m2 = W.molecule_pol_f(4102, 2)
    jobs = [W.Job(m1, W.transition_matrices(4101, 5, m1.nbf), W.axis(7, 12.0), W.axis(5, 9.0), W.axis(128, 14.0)),
            W.Job(m2, W.transition_matrices(4102, 3, m2.nbf), W.axis(10, 8.0), W.axis(3, 11.0), W.axis(256, 16.0)),
            W.Job(m1, W.transition_matrices(4103, 9, m1.nbf), W.axis(4, 20.0), W.axis(9, 20.0), W.axis(128, 20.0))]
    specs, handles = make_batch(ctx, jobs, prec)
    plan = ctx.plan(specs, precision=prec)
    stream = torch.cuda.Stream()
    plan.run_graph(stream)
    stream.synchronize()
    ctx.sync(stream)
    tol = 5e-5 if prec == scff.BF16X2 else 1e-5
    for (b, t, g), s, job in zip(handles, specs, jobs):
        fa, f2a = ctx.form_factor(b, t, g, precision=prec, scale=s[5], f_out="cuda")
        ctx.sync()
        assert torch.equal(fa, s[3]) and torch.equal(f2a, s[4])
        idx = W.subset_indices(job.nq, 400, 11)
        ref = oracle.grid_form_factor(job, idx, scale=s[5])
        fc = s[3].cpu().numpy()
        fc = fc[..., 0] + 1j * fc[..., 1]
        assert np.max(np.abs(fc[:, idx] - ref)) / np.max(np.abs(ref)) < tol
    plan.release()


def test_admission_rejects_oversize_job(ctx):
    import torch
    job = W.config3()
    specs, _ = make_batch(ctx, [job], scff.TF32X3)
    with pytest.raises(scff.ScffError) as e:
        ctx.plan(specs, precision=scff.TF32X3, workspace_bytes=64 << 20)
    assert e.value.code == 4  # ADMISSION
