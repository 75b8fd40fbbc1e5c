"""Pins of the FFT-method oracle (oracle/fft.py) and of the oracle's
real-space density: the direct discrete Fourier sum, the analytic transform
of an s Gaussian, convergence to the exact Cartesian oracle, discrete
Parseval, and the density against the quadrature reference's functions."""
import numpy as np
import pytest

import oracle
from oracle import fft as FFT
from paper_2512_18010_b300 import workloads as W
from tests import quadrature_ref as Q
from tests.test_oracle_pins import mol_of


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_density_matches_independent_function_values():
    # Phi at random points from the quadrature reference's own (numerically
    # normalised) functions, Cartesian and pure.
    rng = np.random.default_rng(70)
    base = mol_of(rng.uniform(-1, 1, size=(2, 3)), [(0, 2, [1.3, 0.4], rng.standard_normal(2)),
                                                     (1, -1, [0.9, 0.3], rng.standard_normal(4)),
                                                     (1, 3, [0.7], [1.0])])
    for pure in (0, W.PURE_D | W.PURE_F):
        mol = W.Molecule(**{**base.__dict__, "pure": pure})
        T = rng.standard_normal((2, mol.nbf, mol.nbf))
        r = rng.uniform(-2.5, 2.5, size=(25, 3))
        qb = Q.QuadBasis(mol)
        vals = np.zeros((mol.nbf, len(r)))
        for i, (A, terms, al, w) in enumerate(qb.fn):
            d = r - A[None, :]
            ang = sum(k * d[:, 0] ** a * d[:, 1] ** b * d[:, 2] ** c for k, (a, b, c) in terms)
            vals[i] = ang * sum(wk * np.exp(-ak * np.sum(d * d, 1)) for ak, wk in zip(al, w))
        ref = np.einsum("smn,mr,nr->sr", T, vals, vals)
        assert rel(oracle.density(mol, T, r), ref) < 1e-11


def test_fft_route_equals_the_direct_sum():
    job = W.config1()
    n, dq, c = (16, 8, 12), (0.6, 0.9, 0.5), (0.1, -0.2, 0.05)
    f, phi = FFT.form_factor(job.mol, job.T, n, dq, c)
    ax = FFT.axes(n, dq, c)
    rng = np.random.default_rng(71)
    picks = [tuple(rng.integers(0, n[i]) for i in range(3)) for _ in range(6)] + [(0, 0, 0), (8, 4, 6)]
    q = np.array([[ax[0][1][i], ax[1][1][j], ax[2][1][k]] for i, j, k in picks])
    d = FFT.direct_sum(phi, n, dq, c, q)
    got = np.array([f[:, i, j, k] for i, j, k in picks]).T
    assert rel(got, d) < 1e-12


def test_s_gaussian_matches_its_analytic_transform():
    # Normalised s primitive: Phi = phi^2, whose transform is exp(-q^2/(8a)) e^{iq.P};
    # the spacing puts the aliased copies (2 pi / dx = 16 away) below exp(-8^2/2.4)
    # ~ 3e-12 and the box edge (12.6 Bohr) makes tiling negligible.
    P = np.array([0.4, -0.3, 0.6])
    a = 0.3
    mol = mol_of(P[None, :], [(0, 0, [a], [1.0])])
    n, dq, c = (64, 64, 64), (0.25, 0.25, 0.25), (0.0, 0.0, 0.0)
    f, _ = FFT.form_factor(mol, np.ones((1, 1, 1)), n, dq, c)
    ax = FFT.axes(n, dq, c)
    qx, qy, qz = np.meshgrid(ax[0][1], ax[1][1], ax[2][1], indexing="ij")
    exact = np.exp(-(qx ** 2 + qy ** 2 + qz ** 2) / (8 * a)) * np.exp(1j * (qx * P[0] + qy * P[1] + qz * P[2]))
    assert np.max(np.abs(f[0] - exact)) < 1e-11


def test_converges_to_the_cartesian_oracle():
    rng = np.random.default_rng(72)
    mol = mol_of(rng.uniform(-0.8, 0.8, size=(2, 3)), [(0, 1, [1.6, 0.5], rng.standard_normal(2)),
                                                       (1, 0, [1.1, 0.35], rng.standard_normal(2)),
                                                       (1, 2, [0.9], [1.0])])
    T = rng.standard_normal((1, mol.nbf, mol.nbf))
    n, dq, c = (64, 64, 64), (0.3, 0.3, 0.3), (0.0, 0.0, 0.0)
    f, _ = FFT.form_factor(mol, T, n, dq, c)
    ax = FFT.axes(n, dq, c)
    picks = [(32, 32, 32), (40, 30, 33), (20, 41, 28), (35, 35, 18)]
    q = np.array([[ax[0][1][i], ax[1][1][j], ax[2][1][k]] for i, j, k in picks])
    exact = oracle.form_factor(mol, T, q)
    got = np.array([f[:, i, j, k] for i, j, k in picks]).T
    assert rel(got, exact) < 1e-6


def test_discrete_parseval():
    job = W.config1()
    n, dq, c = (16, 16, 16), (0.7, 0.7, 0.7), (0.0, 0.0, 0.0)
    f, phi = FFT.form_factor(job.mol, job.T, n, dq, c)
    a, b = FFT.parseval(phi, f, n, dq)
    assert a == pytest.approx(b, rel=1e-12)
