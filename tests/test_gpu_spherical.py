"""GPU parity of the spherical method (scff_spherical) against the oracle's
spherical-harmonic projection of the FP64 Cartesian oracle.

Error metric per state: max over (q, l, m) of |R - R_oracle| / max |R_oracle|
(and likewise for f on the angular grid and for the isotropic average).
Bars as for the Cartesian path: FP64 1e-10, the split tensor-core modes 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import spherical as SPH
from paper_2512_18010_b300 import scff
from paper_2512_18010_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {scff.FP64: 1e-10, scff.BF16X3: 1e-5, scff.TF32X3: 1e-5}
PRECS = [scff.FP64, scff.BF16X3, scff.TF32X3]


@pytest.fixture(scope="module")
def ctx():
    c = scff.Context(0)
    yield c
    c.close()


def rel_err(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.max(np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1))


def angular_grid(nt, np_):
    theta = np.pi * (np.arange(nt) + 0.5) / nt
    phi = 2 * np.pi * np.arange(np_) / np_
    return theta, phi


_REF = {}


def reference(name, job, q, lmax, n_gl):
    key = (name, tuple(q), lmax)
    if key not in _REF:
        _REF[key] = SPH.project(job.mol, job.T, q, lmax, n_gl=n_gl)
    return _REF[key]


@pytest.mark.parametrize("prec", PRECS)
def test_config1_R_f_iso(ctx, prec):
    job = W.config1()
    q = np.array([0.0, 0.7, 2.0, 4.5, 7.5])
    lmax = 10
    Rref = reference("cfg1", job, q, lmax, 48)
    theta, phi = angular_grid(9, 14)
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    out = ctx.spherical(b, t, q, lmax, theta, phi, precision=prec)
    assert rel_err(out["R"], Rref) < TOL[prec]
    fref = SPH.reconstruct(Rref, lmax, theta, phi)
    assert rel_err(out["f"], fref) < TOL[prec]
    assert np.allclose(out["f2"], np.abs(out["f"]) ** 2, rtol=1e-5 if prec else 1e-12, atol=1e-30)
    iso_ref = SPH.isotropic_average(Rref, lmax)
    assert rel_err(out["iso"], iso_ref) < 4 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_f_and_pure_shells(ctx, prec):
    # pair degree 6 (f with f), pure d and f: every (lambda, mu) up to 6
    job = W.config_f(seed=3600, n_heavy=1, n_states=3, n=8, pure=W.PURE_D | W.PURE_F)
    q = np.array([0.3, 1.8, 3.9])
    lmax = 8
    Rref = reference("pure-f", job, q, lmax, 44)
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    out = ctx.spherical(b, t, q, lmax, precision=prec, want=("R", "iso"))
    assert rel_err(out["R"], Rref) < TOL[prec]


@pytest.mark.parametrize("prec", [scff.FP64, scff.BF16X3])
def test_benzene_ring_twelve_states(ctx, prec):
    job = W.config2()
    q = np.array([0.5, 2.2, 4.0])
    lmax = 12
    Rref = reference("cfg2", job, q, lmax, 48)
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    out = ctx.spherical(b, t, q, lmax, precision=prec, scale=np.sqrt(2.0), want=("R",))
    assert rel_err(out["R"], np.sqrt(2.0) * Rref) < TOL[prec]


def test_expansion_converges_to_the_cartesian_path(ctx):
    # With l_max high enough the truncated expansion is the form factor itself:
    # compare with the Cartesian FP64 path at the same q vectors.
    job = W.config1()
    q = np.array([1.2, 3.0])
    theta, phi = angular_grid(5, 7)
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    out = ctx.spherical(b, t, q, 32, theta, phi, precision=scff.FP64, want=("f",))
    u = SPH.directions(theta, phi).reshape(-1, 3)
    pts = np.concatenate([qn * u for qn in q])
    g = ctx.qgrid_list(pts)
    fc, _ = ctx.form_factor(b, t, g, precision=scff.FP64)
    fs = out["f"].reshape(out["f"].shape[0], -1)
    assert np.max(np.abs(fs - fc)) < 1e-10 * np.max(np.abs(fc))


def test_isotropic_average_of_an_s_gaussian(ctx):
    # <|f|^2> of exp(-q^2/8a) e^{iq.P} is exp(-q^2/4a) at every q and origin.
    mol = W.Molecule(name="s", xyz=np.array([[0.8, -0.5, 1.1]]), shell_atom=np.array([0], np.int32),
                     shell_l=np.array([0], np.int32), shell_nprim=np.array([1], np.int32),
                     exponents=np.array([0.9]), coefficients=np.array([1.0]))
    b = ctx.basis(mol)
    t = ctx.transitions(b, np.ones((1, 1, 1)))
    q = np.array([0.0, 0.5, 1.5, 3.0])
    out = ctx.spherical(b, t, q, 36, precision=scff.FP64, want=("iso",))
    assert np.allclose(out["iso"][0], np.exp(-q * q / (4 * 0.9)), rtol=1e-11, atol=0)


def test_invalid_spherical_arguments(ctx):
    job = W.config1()
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    with pytest.raises(scff.ScffError) as e:
        ctx.spherical(b, t, [1.0], 41)
    assert e.value.code == 1
    with pytest.raises(scff.ScffError) as e:
        ctx.spherical(b, t, [1.0], 4, precision=scff.FP32)
    assert e.value.code == 1
    with pytest.raises(scff.ScffError) as e:
        ctx.spherical(b, t, [-1.0], 4)
    assert e.value.code == 1
    # |f|^2 alone (without f) is allowed
    theta, phi = angular_grid(3, 4)
    out = ctx.spherical(b, t, [1.0], 4, theta, phi, precision=scff.FP64, want=("f2",))
    ref = ctx.spherical(b, t, [1.0], 4, theta, phi, precision=scff.FP64, want=("f",))
    assert np.allclose(out["f2"], np.abs(ref["f"]) ** 2, rtol=1e-13)
