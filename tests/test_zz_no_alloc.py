"""The allocation-free entry point (scff_form_factor_static).

It exists for callers that cannot allocate device memory while they run --
for example code inside a framework whose caching allocator already owns the
device memory, or a serving loop that must not stall on cudaMalloc/cudaFree.
They pass their own device buffers; the library keeps its intermediates in a
fixed device array of its own.  This file is collected last so that a run
that stops at the first failure has run every other test before it.

The check: two calls in a row (a larger job, then a smaller one, so a stale
scratch would show) must match the regular entry point (scff_form_factor,
FP64, explicit q list) within the FP64 tolerance of the parity tests, and an
input beyond the scratch limit must be rejected with a clear error.
"""
import numpy as np
import pytest

from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def regular(ctx, job, q):
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    g = ctx.qgrid_list(q)
    try:
        f, f2 = ctx.form_factor(b, t, g, precision=scff.FP64)
    finally:
        ctx.release(g)
        ctx.release(b)
    return f, f2


def static_call(job, q):
    import torch
    dev = torch.device("cuda", 0)
    T = torch.from_numpy(np.ascontiguousarray(job.T)).to(dev)
    qd = torch.from_numpy(np.ascontiguousarray(q, dtype=np.float64)).to(dev)
    f = torch.full((job.n_states, len(q), 2), float("nan"), dtype=torch.float64, device=dev)
    f2 = torch.full((job.n_states, len(q)), float("nan"), dtype=torch.float64, device=dev)
    scff.form_factor_static(job.mol, T, qd, f, f2)
    f = f.cpu().numpy()
    return f[..., 0] + 1j * f[..., 1], f2.cpu().numpy()


def rel_err(f, g):
    return np.max(np.max(np.abs(f - g), axis=-1) / np.max(np.abs(g), axis=-1))


def test_static_entry_matches_regular_entry_twice():
    ctx = scff.Context(0)
    try:
        rng = np.random.default_rng(21)
        jobs = [W.config2(), W.config1()]          # larger first, then smaller
        qs = [rng.uniform(-15, 15, size=(777, 3)), np.vstack([np.zeros((1, 3)), rng.uniform(-10, 10, size=(300, 3))])]
        for job, q in zip(jobs, qs):
            f_ref, f2_ref = regular(ctx, job, q)
            f, f2 = static_call(job, q)
            assert np.all(np.isfinite(f)) and np.all(np.isfinite(f2))
            assert rel_err(f, f_ref) < FP64_TOL
            assert rel_err(f2, f2_ref) < FP64_TOL
    finally:
        ctx.close()


def test_static_entry_matches_oracle():
    """The allocation-free call checked against the FP64 oracle directly (not only against the
    regular entry point): config 1 on explicit q points, including q = 0."""
    import oracle
    job = W.config1()
    rng = np.random.default_rng(22)
    q = np.vstack([np.zeros((1, 3)), rng.uniform(-10, 10, size=(255, 3))])
    f, f2 = static_call(job, q)
    ref = oracle.form_factor(job.mol, job.T, q)
    assert rel_err(f, ref) < FP64_TOL
    assert rel_err(f2, np.abs(ref) ** 2) < FP64_TOL


def test_static_entry_rejects_oversize_basis():
    import torch
    big = W.molecule_dz_d(4242, 30)                # 30 heavy + 30 H: 450 records > 256
    T = torch.zeros((1, big.nbf, big.nbf), dtype=torch.float64, device="cuda")
    q = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((1, 4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(scff.ScffError) as e:
        scff.form_factor_static(big, T, q, f)
    assert e.value.code == 1 and "256" in str(e.value)
