"""Error-bounded pair screening: the screened result stays within
eps * max_q|f_s(q)| of the exact one for every state (FP64 path, so the
difference is the screening error alone), removes pairs, and keeps the
tensor-core modes within their oracle bar."""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps", [1e-7, 1e-4, 1e-2])
def test_screening_error_bound_fp64(eps):
    job = W.scaled_job(W.config3(), 24)
    ctx = scff.Context(0)
    try:
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        g = ctx.qgrid_product(job.qx, job.qy, job.qz)
        exact, _ = ctx.form_factor(b, t, g, precision=scff.FP64)
        ctx.set_screening(eps)
        scr, _ = ctx.form_factor(b, t, g, precision=scff.FP64)
        info = ctx.screening_info(t, g)
        assert 0 < info["kept_pairs"] < info["pairs"]
        err = np.max(np.abs(scr - exact), axis=1)
        bound = eps * np.max(np.abs(exact), axis=1)
        assert np.all(err <= bound)
    finally:
        ctx.close()


def test_screening_with_tensor_cores_meets_bar():
    job = W.config3()
    ctx = scff.Context(0)
    try:
        ctx.set_screening(1e-7)
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        g = ctx.qgrid_product(job.qx, job.qy, job.qz)
        f, _ = ctx.form_factor(b, t, g, precision=scff.BF16X3)
        info = ctx.screening_info(t, g)
        assert info["kept_rows"] < info["rows"]
        idx = W.subset_indices(job.nq, 2048, 31)
        ref = oracle.grid_form_factor(job, idx)
        assert np.max(np.max(np.abs(f[:, idx] - ref), axis=1) / np.max(np.abs(ref), axis=1)) < 1e-5
    finally:
        ctx.close()
