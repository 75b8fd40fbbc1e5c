"""Autotuner: the first call of a job shape times the candidate
configurations and keeps the fastest; the result meets the precision's bar
and later calls of the shape reuse the choice."""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [scff.TF32X3, scff.BF16X3, scff.FP16X2])
def test_autotune_choice_and_parity(prec):
    ctx = scff.Context(0)
    try:
        ctx.set_autotune(True)
        for job in (W.config2(), W.config1()):
            b = ctx.basis(job.mol)
            t = ctx.transitions(b, job.T)
            g = ctx.qgrid_product(job.qx, job.qy, job.qz)
            with pytest.raises(scff.ScffError):
                ctx.autotune_choice(b, t, g, prec)
            f1, _ = ctx.form_factor(b, t, g, precision=prec)
            ch = ctx.autotune_choice(b, t, g, prec)
            assert ch["best_us"] > 0 and ch["state_block"] in (8, 12, 16)
            n0 = ctx.kernel_launches()
            f2, _ = ctx.form_factor(b, t, g, precision=prec)
            assert ctx.kernel_launches() - n0 <= 12        # no re-tuning on the second call
            assert np.array_equal(f1, f2)
            idx = W.subset_indices(job.nq, 500, 8)
            ref = oracle.grid_form_factor(job, idx)
            assert np.max(np.abs(f1[:, idx] - ref)) / np.max(np.abs(ref)) < 1e-5
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", [scff.FP16X2, scff.TF32X3, scff.BF16X2])
def test_generator_variants_agree_bitwise(prec):
    # On a grid whose z axis is a multiple of 128 every W generator variant the split allows can run
    # (gathered from global memory, Z and Y staged in shared memory, or gathered one chunk ahead with
    # the running sums in TMEM); they form the same W and add the same partial sums in the same order,
    # so the results are bitwise equal, and scff_last_path reports which one ran.
    base = W.config_f(n_heavy=2, n_states=5)
    job = W.Job(base.mol, base.T, W.axis(9, 12.0), W.axis(6, 9.0), W.axis(128, 14.0), 3520)
    variants = (0, 1, 2, 3) if prec in (scff.FP16X2, scff.BF16X2) else (0, 1)
    ctx = scff.Context(0)
    try:
        out = {}
        for z in variants:
            ctx.set_tc_variant(z)
            f, f2 = scff.evaluate_job(ctx, job, precision=prec)
            p = ctx.last_path()
            assert p["path"] == "tensor_cores" and p["variant"] == scff.GEN_VARIANTS[z]
            out[z] = (f, f2)
        for z in variants[1:]:
            assert np.array_equal(out[0][0], out[z][0]) and np.array_equal(out[0][1], out[z][1])
        idx = W.subset_indices(job.nq, 600, 12)
        ref = oracle.grid_form_factor(job, idx)
        tol = 5e-5 if prec == scff.BF16X2 else 1e-5
        assert np.max(np.abs(out[0][0][:, idx] - ref)) / np.max(np.abs(ref)) < tol
        # with the autotuner on, the variants are candidates and the choice is reported
        ctx.set_tc_zstage(-1)
        ctx.set_autotune(True)
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        g = ctx.qgrid_product(job.qx, job.qy, job.qz)
        fa, _ = ctx.form_factor(b, t, g, precision=prec)
        ch = ctx.autotune_choice(b, t, g, prec)
        octant = prec in (scff.FP16X2, scff.BF16X2)
        assert ch["zstage"] in variants + ((4,) if octant else ())
        if ch["tensor_cores"] and ch["zstage"] != 4:
            assert np.array_equal(fa, out[0][0])
        # the octant form (a candidate for the kinds with CTA pairs) rounds differently
        assert np.max(np.abs(fa[:, idx] - ref)) / np.max(np.abs(ref)) < tol
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", [scff.FP16X2, scff.BF16X2])
@pytest.mark.parametrize("drain", [2, 3, 8, 0])
@pytest.mark.parametrize("variant", [2, 3])
def test_variant_regimes(prec, drain, variant):
    # The prefetching and CTA-pair variants against the gather variant, bitwise, where their
    # bookkeeping differs: drains of 2 and 3 chunks (odd groups, a last group shorter than the rest),
    # the whole K in one TMEM run (0), items of a single k-chunk and tail-split parts (the small
    # z = 128 grid has few tiles, so its last tiles run as parts), an odd number of m-tiles (the
    # pair's second half all padding), ragged column tiles, and the mirrored half on antisymmetric
    # axes.
    base = W.config_f(n_heavy=1, n_states=3)
    jobs = [W.Job(base.mol, base.T, W.axis(7, 10.0), W.axis(5, 8.0), W.axis(128, 12.0), 3521),
            W.Job(base.mol, base.T, W.axis(4, 10.0), W.axis(33, 8.0), W.axis(20, 12.0), 3522),
            W.config1()]
    ctx = scff.Context(0)
    try:
        ctx.set_tc_drain(drain)
        for job, bands in zip(jobs, (0, 1, 2)):
            ctx.set_download_bands(bands)   # overlapped download (automatic, off, two bands)
            out = {}
            for z in (0, variant):
                ctx.set_tc_variant(z)
                out[z] = scff.evaluate_job(ctx, job, precision=prec)
                assert ctx.last_path()["variant"] == scff.GEN_VARIANTS[z]
            assert np.array_equal(out[0][0], out[variant][0]) and np.array_equal(out[0][1], out[variant][1])
            idx = W.subset_indices(job.nq, 300, 13)
            ref = oracle.grid_form_factor(job, idx)
            tol = 5e-5 if prec == scff.BF16X2 else 1e-5
            if drain != 0:
                assert np.max(np.abs(out[variant][0][:, idx] - ref)) / np.max(np.abs(ref)) < tol
    finally:
        ctx.close()


def test_last_path_reports_the_path_taken():
    job = W.config1()
    ctx = scff.Context(0)
    try:
        assert ctx.last_path()["path"] is None
        scff.evaluate_job(ctx, job, precision=scff.FP16X2)
        # the default for FP16 hi/lo on an antisymmetric grid: CTA pairs in the octant form
        assert ctx.last_path() == {"path": "tensor_cores", "precision": "fp16x2", "variant": "octant"}
        # a tensor-core precision on an explicit q list runs the FP32 direct path
        scff.evaluate_job(ctx, job, precision=scff.BF16X3, q_list=np.array([[0.1, 0.2, 0.3], [1.0, 0.0, 0.0]]))
        assert ctx.last_path() == {"path": "direct_fp32", "precision": "fp32", "variant": None}
        scff.evaluate_job(ctx, job, precision=scff.FP64)
        assert ctx.last_path()["path"] == "direct_fp64"
    finally:
        ctx.close()
