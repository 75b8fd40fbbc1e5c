"""Autotuner: the first call of a job shape times the candidate
configurations and keeps the fastest; the result meets the precision's bar
and later calls of the shape reuse the choice."""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [scff.TF32X3, scff.BF16X3])
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
