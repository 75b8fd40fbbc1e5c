"""GPU checks of the tensor-core tail split in its three regimes.

A persistent launch of T equal tiles on P SMs leaves R = T mod P tiles for a
last, partial wave; those run as s parts over disjoint k ranges with s chosen
to minimise ceil(R s / P) / s (at most 2P parts).  The shapes below give (on
148 SMs) R = 20 (s = 7, fewer parts than SMs), R = 80 (s = 3, more parts than
SMs, so some CTAs run two parts) and R = 120 (no split).  Every point of the
split-BF16 result is compared with the FP32 direct path and sampled points
with the oracle.
"""
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


def rel_err(f, g):
    num = np.max(np.abs(np.asarray(f) - np.asarray(g)), axis=-1)
    return np.max(num / np.max(np.abs(np.asarray(g)), axis=-1))


@pytest.mark.parametrize("nx, ny, seed", [(64, 84, 4201), (128, 76, 4203), (64, 134, 4205)])
def test_tail_split_regimes(ctx, nx, ny, seed):
    base = W.config2()
    T = W.transition_matrices(seed, 3, base.mol.nbf)
    # shifted x axis: not antisymmetric, so every row is computed (3 nx / 128 m-tiles, ny n-tiles)
    job = W.Job(base.mol, T, W.axis(nx, 10.0) + 0.03, W.axis(ny, 11.0), W.axis(128, 12.0), seed)
    f_tc, _ = scff.evaluate_job(ctx, job, precision=scff.BF16X3)
    f_32, _ = scff.evaluate_job(ctx, job, precision=scff.FP32)
    assert rel_err(f_tc, f_32) < 1e-5
    idx = W.subset_indices(job.nq, 500, seed + 1)
    assert rel_err(f_tc[:, idx], oracle.grid_form_factor(job, idx)) < 1e-5
