"""Pins of the spherical-harmonic oracle (oracle/spherical.py) against what
the mathematics fixes: the plane-wave (Rayleigh) expansion of an s Gaussian,
reconstruction of the exact Cartesian f, convergence of the sphere rule,
the q = 0 limit, and Parseval against an independent sphere rule."""
import numpy as np
import pytest
from scipy.special import spherical_jn, sph_harm_y

import oracle
from oracle import spherical as SPH
from paper_2512_18010_b300 import workloads as W
from tests.test_oracle_pins import mol_of


def test_s_gaussian_off_origin_is_the_rayleigh_expansion():
    # One normalised s primitive at P: f(q) = exp(-q^2/(8a)) e^{i q.P}, whose
    # expansion is R_lm(q) = 4 pi i^l j_l(q|P|) conj(Y_l^m(P^)) exp(-q^2/(8a)).
    P = np.array([0.9, -0.4, 1.3])
    a = 0.7
    mol = mol_of(P[None, :], [(0, 0, [a], [1.0])])
    T = np.ones((1, 1, 1))
    q = np.array([0.0, 0.6, 2.1, 4.0])
    lmax = 10
    R = SPH.project(mol, T, q, lmax, n_gl=48)[0]
    r = np.linalg.norm(P)
    th, ph = np.arccos(P[2] / r), np.arctan2(P[1], P[0])
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            exp = (4 * np.pi * (1j ** l) * spherical_jn(l, q * r) * np.conj(sph_harm_y(l, m, th, ph))
                   * np.exp(-q * q / (8 * a)))
            got = R[:, SPH.lm_index(l, m)]
            assert np.max(np.abs(got - exp)) < 1e-12, (l, m)


def test_reconstruction_converges_to_the_cartesian_oracle():
    job = W.config1()
    q = np.array([1.5, 3.0])
    lmax = 30
    R = SPH.project(job.mol, job.T, q, lmax, n_gl=56)
    rng = np.random.default_rng(60)
    theta = np.arccos(rng.uniform(-1, 1, 5))
    phi = rng.uniform(0, 2 * np.pi, 4)
    f_sph = SPH.reconstruct(R, lmax, theta, phi)                      # [S, q, theta, phi]
    u = SPH.directions(theta, phi).reshape(-1, 3)
    for iq, qn in enumerate(q):
        f = oracle.form_factor(job.mol, job.T, qn * u).reshape(1, len(theta), len(phi))
        assert np.max(np.abs(f_sph[:, iq] - f)) < 1e-10 * np.max(np.abs(f))
    # a low l_max visibly truncates (the test above is not vacuous)
    f_low = SPH.reconstruct(R, 2, theta, phi)
    f3 = oracle.form_factor(job.mol, job.T, q[1] * u).reshape(1, len(theta), len(phi))
    assert np.max(np.abs(f_low[:, 1] - f3)) > 1e-3 * np.max(np.abs(f3))


def test_sphere_rule_converged():
    job = W.config1()
    q = np.array([2.5])
    a = SPH.project(job.mol, job.T, q, 12, n_gl=40)
    b = SPH.project(job.mol, job.T, q, 12, n_gl=64)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def test_q_zero_has_only_the_monopole():
    job = W.config1()
    R = SPH.project(job.mol, job.T, np.array([0.0]), 6, n_gl=16)[0, 0]
    f0 = oracle.form_factor(job.mol, job.T, np.zeros((1, 3)))[0, 0]
    assert abs(R[0] - np.sqrt(4 * np.pi) * f0) < 1e-13 * abs(f0)
    assert np.max(np.abs(R[1:])) < 1e-13 * abs(f0)


def test_parseval_against_an_independent_rule():
    # (1/4pi) sum |R_lm|^2 (all significant l) equals the sphere average of
    # |f|^2 taken with a randomly rotated product rule of another size.
    job = W.config1()
    q = np.array([2.0])
    lmax = 30
    R = SPH.project(job.mol, job.T, q, lmax, n_gl=48)
    iso = SPH.isotropic_average(R, lmax)[0, 0]
    theta, phi, w = SPH.sphere_rule(37)
    u = SPH.directions(theta, phi + 0.3).reshape(-1, 3)
    Rot = W.random_rotation(np.random.default_rng(61))
    f = oracle.form_factor(job.mol, job.T, q[0] * u @ Rot.T)[0]
    avg = np.sum(w.reshape(-1) * np.abs(f) ** 2) / (4 * np.pi)
    assert iso == pytest.approx(avg, rel=1e-11)
