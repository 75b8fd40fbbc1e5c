"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Error metric (per state): max_q |f_gpu - f_oracle| / max_q |f_oracle| over
the compared points.  Bars: FP64 1e-10, FP32 1e-6, the 1e-5-grade tensor-core
splits (BF16 hi/mid/lo, TF32 hi/lo, FP16 hi/lo) 1e-5.  The fast BF16 hi/lo
split keeps three products of two 8-bit pieces, so its per-product error is
~2^-16; it is held to its own documented 5e-5 bar.
"""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {scff.FP64: 1e-10, scff.FP32: 1e-6, scff.BF16X3: 1e-5, scff.TF32X3: 1e-5, scff.BF16X2: 5e-5,
       scff.FP16X2: 1e-5}
TC = [scff.BF16X3, scff.TF32X3, scff.BF16X2, scff.FP16X2]


@pytest.fixture(scope="module")
def ctx():
    c = scff.Context(0)
    yield c
    c.close()


def rel_err(f, g):
    f = np.asarray(f)
    g = np.asarray(g)
    num = np.max(np.abs(f - g), axis=-1)
    den = np.max(np.abs(g), axis=-1)
    return np.max(num / den)


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32] + TC)
def test_config1_full_grid(ctx, prec):
    job = W.config1()
    f, f2 = scff.evaluate_job(ctx, job, precision=prec)
    ref = oracle.grid_form_factor(job)
    assert rel_err(f, ref) < TOL[prec]
    assert np.allclose(f2, np.abs(f) ** 2, rtol=1e-5 if prec else 1e-12, atol=1e-30)


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32])
def test_config1_list_path(ctx, prec):
    job = W.config1()
    rng = np.random.default_rng(0)
    q = np.vstack([np.zeros((1, 3)), rng.uniform(-12, 12, size=(300, 3))])
    f, _ = scff.evaluate_job(ctx, job, precision=prec, q_list=q)
    ref = oracle.form_factor(job.mol, job.T, q)
    assert rel_err(f, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32] + TC)
def test_config2_grid_sampled(ctx, prec):
    job = W.config2()
    idx = W.subset_indices(job.nq, 1500, 2002)
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32] + TC)
def test_config3_full_size_sampled(ctx, prec):
    # Full 128^3 grid, 12 states; the oracle checks a seeded 4096-point subset.
    job = W.config3()
    idx = W.subset_indices(job.nq, 4096 if prec != scff.FP64 else 1024, 3003)
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


def test_hermiticity_on_gpu(ctx):
    job = W.config2()
    f, _ = scff.evaluate_job(ctx, job, precision=scff.FP64)
    n = len(job.qx)
    g = f.reshape(f.shape[0], n, n, n)
    mirror = np.conj(g[:, ::-1, ::-1, ::-1])
    assert np.max(np.abs(g - mirror)) < 1e-12 * np.max(np.abs(g))


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32] + TC)
def test_ragged_grid_and_odd_state_count(ctx, prec):
    # Non-power-of-two axes (ragged tiles) and 13 states (not a multiple of the state block).
    base = W.config1()
    T = W.transition_matrices(77, 13, base.mol.nbf)
    job = W.Job(base.mol, T, W.axis(5, 6.0), W.axis(7, 9.0), W.axis(131, 11.0))
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 600, 5)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP16X2, scff.BF16X3])
def test_many_states_on_few_rows(ctx, prec):
    # 60 states on a 3-point x axis (2 computed rows per state): a 128-row tile then spans 65
    # states, more than the tiled A-image build stages in shared memory, so the image comes from the
    # one-thread-per-vector build; the result must meet the same bar.
    base = W.config1()
    T = W.transition_matrices(78, 60, base.mol.nbf)
    job = W.Job(base.mol, T, W.axis(3, 6.0), W.axis(5, 8.0), W.axis(24, 10.0))
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 200, 6)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32])
def test_block_shared_rows_with_padded_states(ctx, prec):
    # z axis a multiple of the 128-point block (every block's points share (ix, iy), the FP32
    # path's shared-row variant), 10 states padded to a block of 12, odd x axis (Hermitian half
    # ends inside a block)
    base = W.config1()
    T = W.transition_matrices(78, 10, base.mol.nbf)
    job = W.Job(base.mol, T, W.axis(5, 6.0), W.axis(3, 9.0), W.axis(256, 11.0))
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 600, 6)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


@pytest.mark.parametrize("S", [5, 16])
def test_fp32_state_blocks_on_block_shared_rows(ctx, S):
    # FP32 state blocks of 8 and 16 states on a grid whose z axis is a multiple of 128: the
    # variant that collapses each pair's x and y powers once per block and evaluates polynomials
    # in q_z alone; d shells (pair degree up to 4) and an odd x axis
    base = W.config2()
    T = W.transition_matrices(79, S, base.mol.nbf)
    job = W.Job(base.mol, T, W.axis(7, 12.0), W.axis(4, 9.0), W.axis(128, 15.0), 79)
    f, _ = scff.evaluate_job(ctx, job, precision=scff.FP32)
    idx = W.subset_indices(job.nq, 700, 7)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[scff.FP32]


def test_degenerate_inputs(ctx):
    job = W.config1()
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    # empty explicit list
    g = ctx.qgrid_list(np.zeros((0, 3)))
    f, f2 = ctx.form_factor(b, t, g, precision=scff.FP64)
    assert f.shape == (1, 0)
    # single point grid at q = 0: f(0) = tr(T S) is real
    g1 = ctx.qgrid_product([0.0], [0.0], [0.0])
    f, _ = ctx.form_factor(b, t, g1, precision=scff.FP64)
    ref = oracle.form_factor(job.mol, job.T, np.zeros((1, 3)))
    assert abs(f[0, 0] - ref[0, 0]) < 1e-12 * abs(ref[0, 0])
    # zero transition matrix gives exactly zero
    tz = ctx.transitions(b, np.zeros_like(job.T))
    fz, _ = ctx.form_factor(b, tz, g1, precision=scff.FP32)
    assert np.all(fz == 0)
    # antisymmetric T gives zero to rounding
    ta = ctx.transitions(b, job.T - np.transpose(job.T, (0, 2, 1)))
    fa, _ = ctx.form_factor(b, ta, ctx.qgrid_product(job.qx, job.qy, job.qz), precision=scff.FP64)
    fs, _ = ctx.form_factor(b, t, ctx.qgrid_product(job.qx, job.qy, job.qz), precision=scff.FP64)
    assert np.max(np.abs(fa)) < 1e-13 * np.max(np.abs(fs)) * 10


def test_scale_and_device_outputs(ctx):
    import torch
    job = W.config1()
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    g = ctx.qgrid_product(job.qx, job.qy, job.qz)
    f_host, _ = ctx.form_factor(b, t, g, precision=scff.FP64, scale=np.sqrt(2.0))
    fd, f2d = ctx.form_factor(b, t, g, precision=scff.FP64, scale=np.sqrt(2.0), f_out="cuda")
    ctx.sync()
    fd = fd.cpu().numpy()
    assert np.array_equal(fd[..., 0] + 1j * fd[..., 1], f_host)
    ref = oracle.grid_form_factor(job, scale=np.sqrt(2.0))
    assert rel_err(f_host, ref) < 1e-10


def test_invalid_inputs_are_rejected(ctx):
    job = W.config1()
    m = job.mol
    bad = W.Molecule(**{**m.__dict__, "shell_l": np.where(m.shell_l == 2, 4, m.shell_l).astype(np.int32)})
    with pytest.raises(scff.ScffError) as e:
        ctx.basis(bad)
    assert e.value.code == 2  # UNSUPPORTED_L
    neg = W.Molecule(**{**m.__dict__, "exponents": -m.exponents})
    with pytest.raises(scff.ScffError) as e:
        ctx.basis(neg)
    assert e.value.code == 1
    b = ctx.basis(m)
    with pytest.raises(ValueError):
        ctx.transitions(b, np.zeros((1, 3, 3)))
    with pytest.raises(scff.ScffError):
        ctx.qgrid_product([], [0.0], [0.0])


# ---------------------------------------------------------------- Cartesian f shells

@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32] + TC)
def test_f_shells_grid_sampled(ctx, prec):
    # d and f polarisation on heavy atoms, p on H: pair classes up to degree 6.
    job = W.config_f()
    f, f2 = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 1500, 3501)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]
    assert np.allclose(f2, np.abs(f) ** 2, rtol=1e-5 if prec else 1e-12, atol=1e-30)


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32, scff.FP16X2])
def test_f_shells_on_block_shared_rows(ctx, prec):
    # f-pair classes (degree 5 and 6) on a z axis of 128 points: every 128-point block of the
    # direct kernels shares (ix, iy), so the f classes run the block-shared-row variant and merge
    # with the low classes' partial result; an odd x axis ends the Hermitian half inside a block.
    base = W.config_f(n_heavy=2, n_states=5)
    job = W.Job(base.mol, base.T, W.axis(7, 12.0), W.axis(5, 9.0), W.axis(128, 14.0), 3510)
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 900, 3511)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32])
def test_f_shells_list_path(ctx, prec):
    job = W.config_f(n_heavy=2, n_states=5)
    rng = np.random.default_rng(35)
    q = np.vstack([np.zeros((1, 3)), rng.uniform(-10, 10, size=(257, 3))])
    f, _ = scff.evaluate_job(ctx, job, precision=prec, q_list=q)
    ref = oracle.form_factor(job.mol, job.T, q)
    assert rel_err(f, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32, scff.BF16X3, scff.FP16X2])
def test_f_only_basis(ctx, prec):
    # Every pair has degree 6: only the f-pair classes run.
    rng = np.random.default_rng(36)
    xyz = rng.uniform(-1.2, 1.2, size=(2, 3))
    mol = W.Molecule(name="f-only", xyz=xyz, shell_atom=np.array([0, 1], np.int32),
                     shell_l=np.array([3, 3], np.int32), shell_nprim=np.array([2, 1], np.int32),
                     exponents=np.array([1.3, 0.45, 0.8]), coefficients=rng.standard_normal(3), heavy=2)
    T = W.transition_matrices(36, 3, mol.nbf)
    ax = W.axis(24, 9.0)
    job = W.Job(mol, T, ax, W.axis(19, 7.0), W.axis(33, 10.0), 36)
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 800, 37)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


# ---------------------------------------------------------------- pure (spherical-harmonic) d and f shells

@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32, scff.BF16X3, scff.TF32X3, scff.FP16X2])
def test_pure_shells_grid_sampled(ctx, prec):
    job = W.config_f(pure=W.PURE_D | W.PURE_F)
    assert job.mol.nbf == 104
    f, _ = scff.evaluate_job(ctx, job, precision=prec)
    idx = W.subset_indices(job.nq, 1500, 3502)
    ref = oracle.grid_form_factor(job, idx)
    assert rel_err(f[:, idx], ref) < TOL[prec]


def test_pure_transitions_from_device_match_host(ctx):
    import torch
    job = W.config_f(n_heavy=2, n_states=4, n=20, pure=W.PURE_D)
    b = ctx.basis(job.mol)
    assert b.nbf == job.mol.nbf
    g = ctx.qgrid_product(job.qx, job.qy, job.qz)
    fh, _ = ctx.form_factor(b, ctx.transitions(b, job.T), g, precision=scff.FP64)
    td = torch.tensor(job.T, dtype=torch.float64, device="cuda")
    fd, _ = ctx.form_factor(b, ctx.transitions(b, td), g, precision=scff.FP64)
    assert np.array_equal(fh, fd)
    ref = oracle.grid_form_factor(job, W.subset_indices(job.nq, 400, 7))
    assert rel_err(fh[:, W.subset_indices(job.nq, 400, 7)], ref) < TOL[scff.FP64]
    with pytest.raises(ValueError):
        ctx.transitions(b, torch.zeros((1, 105, 105), dtype=torch.float64, device="cuda"))


def test_static_entry_rejects_pure_shells(ctx):
    import torch
    job = W.config_f(n_heavy=1, n_states=2, n=4, pure=W.PURE_F)
    T = torch.tensor(job.T, dtype=torch.float64, device="cuda")
    q = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((2, 3, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(scff.ScffError) as e:
        scff.form_factor_static(job.mol, T, q, f)
    assert e.value.code == 1


def test_bounded_wait_reports_timeout_and_context_survives(ctx):
    # A device-side wait on an mbarrier nothing arrives at gives up after its
    # limit and raises the context's TIMEOUT status instead of hanging; the
    # context keeps working afterwards.
    with pytest.raises(scff.ScffError) as e:
        ctx.wait_selftest(4096)
    assert e.value.code == 6
    job = W.config1()
    f, _ = scff.evaluate_job(ctx, job, precision=scff.FP64)
    assert rel_err(f, oracle.grid_form_factor(job)) < TOL[scff.FP64]


@pytest.mark.parametrize("prec", [scff.FP64, scff.FP32, scff.BF16X3, scff.FP16X2])
def test_hermitian_half_is_exact_mirror(prec):
    # On an antisymmetric grid the half-evaluated result (default) mirrors
    # f(-q) = conj(f(q)) exactly and agrees with the full evaluation within the
    # tolerance; a grid that is not antisymmetric is evaluated in full.
    c = scff.Context(0)
    try:
        base = W.config1()
        T = W.transition_matrices(91, 5, base.mol.nbf)
        job = W.Job(base.mol, T, W.axis(9, 7.0), W.axis(12, 8.0), W.axis(33, 9.0), 91)
        f_half, f2_half = scff.evaluate_job(c, job, precision=prec)
        n = (9, 12, 33)
        g = f_half.reshape(5, *n)
        assert np.array_equal(g, np.conj(g[:, ::-1, ::-1, ::-1]))
        assert np.array_equal(f2_half.reshape(5, *n), f2_half.reshape(5, *n)[:, ::-1, ::-1, ::-1])
        c.set_hermitian(False)
        f_full, _ = scff.evaluate_job(c, job, precision=prec)
        ref = oracle.grid_form_factor(job)
        assert rel_err(f_half, ref) < TOL[prec]
        assert rel_err(f_full, ref) < TOL[prec]
        c.set_hermitian(True)
        shifted = W.Job(base.mol, T, W.axis(9, 7.0) + 0.1, W.axis(12, 8.0), W.axis(33, 9.0), 91)
        f_s, _ = scff.evaluate_job(c, shifted, precision=prec)
        assert rel_err(f_s, oracle.grid_form_factor(shifted)) < TOL[prec]
    finally:
        c.close()


def test_alu_peak_microbenchmark(ctx):
    # FMA-chain rates of this GPU: positive, FP32 well above FP64, and not above
    # the lanes x 2 flop x clock ceiling (148 SMs x 128 lanes x 2 x 2.1 GHz).
    p32, ms32 = ctx.alu_peak(False, 16384)
    p64, ms64 = ctx.alu_peak(True, 1024)
    assert 5.0 < p32 < 148 * 128 * 2 * 2.1e9 / 1e12
    assert 0.05 < p64 < p32
    assert ms32 > 0 and ms64 > 0
    # packed f32x2 chains: at least the scalar rate's order, at most two FMAs per lane and clock
    p32x2, ms32x2 = ctx.alu_peak(False, 16384, packed=True)
    assert 0.5 * p32 < p32x2 < 2 * 148 * 128 * 2 * 2.1e9 / 1e12 and ms32x2 > 0
    for bad in (0, -5, 1 << 25):
        with pytest.raises(scff.ScffError) as e:
            ctx.alu_peak(False, bad)
        assert e.value.code == 1
