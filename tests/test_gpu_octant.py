"""Octant form (scff_set_tc_variant mode 4): CTA pairs for FP16 hi/lo and BF16 hi/lo, single CTAs
for BF16 hi/mid/lo.

On a grid whose three axes are antisymmetric, the y and z factors of every
pair term at -q are the complex conjugates of those at +q, so one real
contraction per octant point gives f at (qx, +-qy, +-qz) and the mirrored
points.  The results are compared with the FP64 oracle element by element,
with the plain CTA-pair launch (mode 3, within the split's bar), and for the
symmetry f(-q) = conj(f(q)) that the writes must reproduce exactly."""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def tol_of(prec):
    return 5e-5 if prec == scff.BF16X2 else 1e-5


def f_job(nx, ny, nz, seed, n_heavy=1, n_states=3, a=(10.0, 8.0, 12.0)):
    base = W.config_f(n_heavy=n_heavy, n_states=n_states)
    return W.Job(base.mol, base.T, W.axis(nx, a[0]), W.axis(ny, a[1]), W.axis(nz, a[2]), seed)


# grids: odd axes (points that are their own mirror on every axis), a z axis whose octant half is a
# whole number of 32-point tiles (banded download in y rows), ragged column tiles, one-point axes
GRIDS = [(7, 5, 9), (4, 33, 20), (6, 8, 128), (9, 1, 64), (1, 3, 1), (16, 16, 16)]


@pytest.mark.parametrize("prec", [scff.FP16X2, scff.BF16X2, scff.BF16X3])
@pytest.mark.parametrize("grid", GRIDS)
def test_octant_matches_oracle_and_pair_form(prec, grid):
    # mode 4 against the oracle and against mode 3 (CTA pairs in the Re/Im form for the two-piece
    # splits; BF16 hi/mid/lo has no pairs and runs the single-CTA gather variant in both forms)
    job = f_job(*grid, seed=3600 + sum(grid))
    ctx = scff.Context(0)
    try:
        ctx.set_tc_variant(4)
        f4, f24 = scff.evaluate_job(ctx, job, precision=prec)
        assert ctx.last_path()["variant"] == "octant"
        ctx.set_tc_variant(3)
        f3, _ = scff.evaluate_job(ctx, job, precision=prec)
        assert ctx.last_path()["variant"] == ("gather" if prec == scff.BF16X3 else "pair")
    finally:
        ctx.close()
    idx = W.subset_indices(job.nq, 400, 17)
    ref = oracle.grid_form_factor(job, idx)
    assert rel(f4[:, idx], ref) < tol_of(prec)
    assert rel(f4, f3) < tol_of(prec)
    assert np.allclose(f24, np.abs(f4) ** 2, rtol=1e-5, atol=1e-30)
    n = (job.qx.size, job.qy.size, job.qz.size)
    h = f4.reshape(-1, *n)
    assert np.array_equal(h, np.conj(h[:, ::-1, ::-1, ::-1]))  # every mirrored point written


@pytest.mark.parametrize("prec", [scff.FP16X2, scff.BF16X3])
@pytest.mark.parametrize("drain", [2, 3, 8])
def test_octant_regimes(drain, prec):
    # drains of 2 and 3 chunks, tail-split parts (few tiles on the z = 128 grid), an odd m-tile
    # count (the pair's second half all padding), overlapped download off / automatic / two bands
    jobs = [f_job(7, 5, 128, 3611), f_job(4, 33, 20, 3612), W.config1()]
    ctx = scff.Context(0)
    try:
        ctx.set_tc_drain(drain)
        ctx.set_tc_variant(4)
        for job, bands in zip(jobs, (0, 1, 2)):
            ctx.set_download_bands(bands)
            f, _ = scff.evaluate_job(ctx, job, precision=prec)
            idx = W.subset_indices(job.nq, 300, 19)
            assert rel(f[:, idx], oracle.grid_form_factor(job, idx)) < 1e-5
    finally:
        ctx.close()


@pytest.mark.parametrize("bands", [0, 2, 3])
def test_octant_banded_download_is_the_device_result(bands):
    # 8 x 12 x 64: octant y rows of 32 points, one tile each; the host copy of each band equals the
    # device output bitwise
    job = f_job(8, 12, 64, 3620, n_states=5)
    ctx = scff.Context(0)
    try:
        ctx.set_tc_variant(4)
        ctx.set_download_bands(bands)
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        g = ctx.qgrid_product(job.qx, job.qy, job.qz)
        fd, f2d = ctx.form_factor(b, t, g, precision=scff.FP16X2, f_out="cuda")
        ctx.sync()
        fd = fd.cpu().numpy()
        fd = fd[..., 0] + 1j * fd[..., 1]
        fh, f2h = ctx.form_factor(b, t, g, precision=scff.FP16X2)
        assert np.array_equal(fh, fd) and np.array_equal(f2h, f2d.cpu().numpy())
    finally:
        ctx.close()


def test_octant_on_a_shifted_grid_runs_the_pair_form():
    # an axis that is not antisymmetric: mode 4 runs as mode 3, bitwise
    job = f_job(6, 5, 20, 3630)
    job = W.Job(job.mol, job.T, job.qx + 0.25, job.qy, job.qz, 3630)
    ctx = scff.Context(0)
    try:
        ctx.set_tc_variant(4)
        f4, _ = scff.evaluate_job(ctx, job, precision=scff.FP16X2)
        assert ctx.last_path()["variant"] == "pair"
        ctx.set_tc_variant(3)
        f3, _ = scff.evaluate_job(ctx, job, precision=scff.FP16X2)
    finally:
        ctx.close()
    assert np.array_equal(f4, f3)
    idx = W.subset_indices(job.nq, 300, 23)
    assert rel(f4[:, idx], oracle.grid_form_factor(job, idx)) < 1e-5


def test_octant_full_size_job():
    # the 10-heavy-atom job (170 functions, 12 states, 128^3) in the default mode, which is the
    # octant form for FP16 hi/lo: sampled points against the oracle
    job = W.config3()
    ctx = scff.Context(0)
    try:
        f, _ = scff.evaluate_job(ctx, job, precision=scff.FP16X2)
        assert ctx.last_path()["variant"] == "octant"
    finally:
        ctx.close()
    idx = W.subset_indices(job.nq, 256, 29)
    assert rel(f[:, idx], oracle.grid_form_factor(job, idx)) < 1e-5


def test_mixed_plan_equals_alone():
    # one plan holding a shifted grid (CTA pairs in the Re/Im form) and antisymmetric grids (octant
    # form): the launch takes the form per job; alone, the antisymmetric jobs run the five-stage
    # octant build.  Each job's result is bitwise the same in the batch and alone.
    import torch
    j1 = f_job(7, 5, 9, 3640)
    j2 = f_job(6, 5, 20, 3641)
    j2 = W.Job(j2.mol, j2.T, j2.qx + 0.25, j2.qy, j2.qz, 3641)
    j3 = W.config1()
    jobs = [j1, j2, j3]
    ctx = scff.Context(0)
    try:
        ctx.set_tc_variant(4)
        specs = []
        for k, job in enumerate(jobs):
            b = ctx.basis(job.mol)
            t = ctx.transitions(b, job.T)
            g = ctx.qgrid_product(job.qx, job.qy, job.qz)
            specs.append((b, t, g, torch.full((job.n_states, job.nq, 2), float("nan"), device="cuda"),
                          torch.full((job.n_states, job.nq), float("nan"), device="cuda"), 1.0 + 0.5 * k))
        plan = ctx.plan(specs, precision=scff.FP16X2)
        stream = torch.cuda.Stream()
        plan.run_graph(stream)
        stream.synchronize()
        ctx.sync(stream)
        for s, job in zip(specs, jobs):
            fa, f2a = ctx.form_factor(s[0], s[1], s[2], precision=scff.FP16X2, scale=s[5], f_out="cuda")
            ctx.sync()
            assert torch.equal(fa, s[3]) and torch.equal(f2a, s[4])
            idx = W.subset_indices(job.nq, 300, 31)
            fc = s[3].cpu().numpy()
            fc = fc[..., 0] + 1j * fc[..., 1]
            assert rel(fc[:, idx], oracle.grid_form_factor(job, idx, scale=s[5])) < 1e-5
        plan.release()
    finally:
        ctx.close()
