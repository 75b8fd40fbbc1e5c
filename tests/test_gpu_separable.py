"""Separable integrals (scff_separable_integral) against the oracle's full
3-D grid summed with the same weights, and against the library's own FP64
grid evaluation; the axes differ in length and spacing."""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu


def weights(q, kind):
    dq = q[1] - q[0] if len(q) > 1 else 1.0
    if kind == 0:
        return dq * np.exp(-0.1 * q * q)
    if kind == 1:
        return dq * np.cos(0.3 * q) / (1 + q * q)
    return dq * np.ones_like(q)


def test_separable_matches_oracle_and_grid():
    base = W.config1()
    job = W.Job(base.mol, W.transition_matrices(31, 3, base.mol.nbf), W.axis(11, 6.0), W.axis(14, 9.0),
                W.axis(17, 7.5))
    wx, wy, wz = weights(job.qx, 0), weights(job.qy, 1), weights(job.qz, 2)
    ctx = scff.Context(0)
    try:
        b = ctx.basis(job.mol)
        t = ctx.transitions(b, job.T)
        I = ctx.separable_integral(b, t, job.qx, wx, job.qy, wy, job.qz, wz)
        ref = oracle.grid_form_factor(job).reshape(job.n_states, len(job.qx), len(job.qy), len(job.qz))
        Iref = np.einsum("sijk,i,j,k->s", ref, wx, wy, wz)
        mag = np.einsum("sijk,i,j,k->s", np.abs(ref), np.abs(wx), np.abs(wy), np.abs(wz))
        assert np.max(np.abs(I - Iref) / mag) < 1e-11
        g = ctx.qgrid_product(job.qx, job.qy, job.qz)
        f, _ = ctx.form_factor(b, t, g, precision=scff.FP64)
        Ig = np.einsum("sijk,i,j,k->s", f.reshape(ref.shape), wx, wy, wz)
        assert np.max(np.abs(I - Ig) / mag) < 1e-12
        # larger molecule, q = 0 only on every axis: the integral is f_s(0) = tr(T S)
        job3 = W.config3()
        b3 = ctx.basis(job3.mol)
        t3 = ctx.transitions(b3, job3.T)
        one, zero = np.ones(1), np.zeros(1)
        I0 = ctx.separable_integral(b3, t3, zero, one, zero, one, zero, one)
        f0 = oracle.form_factor(job3.mol, job3.T, np.zeros((1, 3)))[:, 0]
        assert np.max(np.abs(I0 - f0)) < 1e-10 * np.max(np.abs(f0))
    finally:
        ctx.close()
