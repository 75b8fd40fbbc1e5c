"""GPU parity at the largest sizes of the workloads: the serving stream's large
job (40 heavy atoms + 40 H, 680 functions, 32 states, 128^3, about 67 M
(q-point x state) values) and the largest molecules of the batched
distribution, each through the single-job entry point in the launch
configuration the bench uses (host outputs, so the banded download runs too),
checked against the FP64 oracle on seeded sampled points.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {scff.FP64: 1e-10, scff.FP32: 1e-6, scff.BF16X3: 1e-5, scff.TF32X3: 1e-5, scff.FP16X2: 1e-5}


@pytest.fixture(scope="module")
def ctx():
    c = scff.Context(0)
    yield c
    c.close()


def rel_err(f, g):
    num = np.max(np.abs(np.asarray(f) - np.asarray(g)), axis=-1)
    return np.max(num / np.max(np.abs(np.asarray(g)), axis=-1))


@pytest.fixture(scope="module")
def large():
    job = W.config5_large()
    idx = W.subset_indices(job.nq, 192, 5991)
    return job, idx, oracle.grid_form_factor(job, idx)


@pytest.mark.parametrize("prec", [scff.BF16X3, scff.TF32X3, scff.FP16X2])
def test_large_job_tensor_cores(ctx, large, prec):
    job, idx, ref = large
    assert job.mol.nbf == 680 and job.n_states == 32
    f, f2 = scff.evaluate_job(ctx, job, precision=prec)
    assert rel_err(f[:, idx], ref) < TOL[prec]
    assert np.allclose(f2[:, idx], np.abs(f[:, idx]) ** 2, rtol=1e-5, atol=1e-30)
    # f(-q) = conj f(q) on the mirrored half, written by the same launch
    assert np.array_equal(f[:, job.nq - 1 - idx], np.conj(f[:, idx]))


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32])
def test_large_job_direct_list_path(ctx, large, prec):
    job, idx, ref = large
    f, _ = scff.evaluate_job(ctx, job, precision=prec, q_list=job.q_points(idx))
    assert rel_err(f, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.BF16X3, scff.FP16X2])
def test_largest_batched_molecules(ctx, prec):
    # the three largest molecules among the first 64 of the batched distribution
    jobs = sorted((W.config4_job(i) for i in range(64)), key=lambda j: -j.mol.nbf)[:3]
    for k, job in enumerate(jobs):
        idx = W.subset_indices(job.nq, 128, 5995 + k)
        ref = oracle.grid_form_factor(job, idx)
        f, _ = scff.evaluate_job(ctx, job, precision=prec)
        assert rel_err(f[:, idx], ref) < TOL[prec], (job.mol.nbf, job.n_states, len(job.qx))
