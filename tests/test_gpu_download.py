"""Overlapped download of host outputs on the tensor-core path
(scff_set_download_bands).

A host-output call runs the output tiles band by band (bands of output
columns) in one launch that reports its progress, and copies each finished
band while later bands compute.  Checks: the host result matches a
device-output call of the same job within the split-precision bound (the band
order hands the tail split to other tiles), one band reproduces the device
result bitwise, the banded result matches the oracle on sampled points, and
every band layout (mirrored pairs of column runs, contiguous runs, a ragged
last tile, f2 omitted) lands every column.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture()
def ctx():
    c = scff.Context(0)
    yield c
    c.close()


def rel_err(f, g):
    num = np.max(np.abs(np.asarray(f) - np.asarray(g)), axis=-1)
    return np.max(num / np.max(np.abs(np.asarray(g)), axis=-1))


def both(ctx, job, prec=scff.BF16X3, with_f2=True):
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    g = ctx.qgrid_product(job.qx, job.qy, job.qz)
    try:
        fd, f2d = ctx.form_factor(b, t, g, precision=prec, f_out="cuda", with_f2=with_f2)
        ctx.sync()
        fd = fd.cpu().numpy()
        fd = fd[..., 0] + 1j * fd[..., 1]
        f2d = f2d.cpu().numpy() if f2d is not None else None
        fh, f2h = ctx.form_factor(b, t, g, precision=prec, with_f2=with_f2)
        return fh, f2h, fd, f2d
    finally:
        ctx.release(g)
        ctx.release(b)


def grid_job(seed, n_states, nx, ny, nz, a=12.0, shift=0.0):
    base = W.config2()
    T = W.transition_matrices(seed, n_states, base.mol.nbf)
    return W.Job(base.mol, T, W.axis(nx, a) + shift, W.axis(ny, a), W.axis(nz, a), seed)


@pytest.mark.parametrize("bands", [2, 3, 5, 8])
def test_mirrored_bands_match_device_output(ctx, bands):
    # antisymmetric 48 x 32 x 64 grid: half rows, N = 2048 = 16 column tiles
    job = grid_job(4101, 7, 48, 32, 64)
    ctx.set_download_bands(bands)
    fh, f2h, fd, f2d = both(ctx, job)
    assert rel_err(fh, fd) < TOL
    assert np.allclose(f2h, np.abs(fh) ** 2, rtol=1e-5, atol=1e-30)
    n = (48, 32, 64)
    h = fh.reshape(7, *n)
    assert np.array_equal(h, np.conj(h[:, ::-1, ::-1, ::-1]))  # every mirrored column landed
    idx = W.subset_indices(job.nq, 600, 4102)
    assert rel_err(fh[:, idx], oracle.grid_form_factor(job, idx)) < TOL


def test_one_band_is_the_device_result_bitwise(ctx):
    job = grid_job(4103, 5, 32, 32, 64)
    ctx.set_download_bands(1)
    fh, f2h, fd, f2d = both(ctx, job)
    assert np.array_equal(fh, fd) and np.array_equal(f2h, f2d)


@pytest.mark.parametrize("bands", [3, 4])
def test_contiguous_bands_with_ragged_last_tile(ctx, bands):
    # not antisymmetric (shifted x axis): every row is computed, bands are
    # contiguous column runs; N = 20 * 30 = 600 leaves a ragged last tile
    job = grid_job(4105, 6, 40, 20, 30, shift=0.05)
    ctx.set_download_bands(bands)
    fh, f2h, fd, f2d = both(ctx, job)
    assert rel_err(fh, fd) < TOL
    assert rel_err(f2h, f2d) < 2 * TOL
    idx = W.subset_indices(job.nq, 500, 4106)
    assert rel_err(fh[:, idx], oracle.grid_form_factor(job, idx)) < TOL


def test_mirror_with_ragged_columns_runs_unbanded(ctx):
    # antisymmetric grid with N = 20 * 30 not a multiple of the tile width:
    # banding is skipped, so the host result is the device result bitwise
    job = grid_job(4107, 4, 40, 20, 30)
    ctx.set_download_bands(4)
    fh, f2h, fd, f2d = both(ctx, job)
    assert np.array_equal(fh, fd) and np.array_equal(f2h, f2d)


@pytest.mark.parametrize("prec", [scff.TF32X3, scff.BF16X2, scff.FP16X2])
def test_bands_without_f2_and_other_kinds(ctx, prec):
    job = grid_job(4109, 3, 64, 32, 32)
    ctx.set_download_bands(3)
    fh, f2h, fd, f2d = both(ctx, job, prec=prec, with_f2=False)
    assert f2h is None and f2d is None
    assert rel_err(fh, fd) < (5e-5 if prec == scff.BF16X2 else TOL)


def test_invalid_band_count(ctx):
    for n in (-1, 9):
        with pytest.raises(scff.ScffError) as e:
            ctx.set_download_bands(n)
        assert e.value.code == 1


def test_bands_with_autotune_and_screening(ctx):
    # the autotuner's choice and the screened pair set both feed the banded path
    job = grid_job(4111, 6, 64, 32, 64)
    ctx.set_download_bands(3)
    ctx.set_autotune(True)
    ctx.set_screening(1e-9)
    fh, f2h, fd, f2d = both(ctx, job)
    assert rel_err(fh, fd) < TOL
    idx = W.subset_indices(job.nq, 400, 4112)
    assert rel_err(fh[:, idx], oracle.grid_form_factor(job, idx)) < TOL
