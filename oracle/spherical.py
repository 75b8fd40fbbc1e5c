"""Spherical-harmonic expansion of the form factor -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product path never does.

What it computes (Sec. "Analytic Method", Eqs. SphericalMethod and RTensor,
and the isotropic average that follows them): the form factor on a sphere of
radius q is expanded in complex spherical harmonics with the Condon-Shortley
phase,

    f_s(q q^) = sum_{l, m} Y_l^m(q^) R^s_{lm}(q),

so R^s_{lm}(q) is the projection

    R^s_{lm}(q) = Int dOmega conj(Y_l^m(q^)) f_s(q q^),

which is what this module evaluates: f_s from the FP64 Cartesian oracle on a
product rule of Gauss-Legendre nodes in cos(theta) and equally spaced phi, and
the projection by that rule (exact for every spherical harmonic of degree
below 2 n_gl, so the only error is the aliasing of f's components above that
degree, which decay faster than exponentially once l exceeds q times the
largest distance of a pair centre from the origin).  The truncated expansion
up to l_max and the isotropic average <|f_s|^2>_Omega = (1/4pi) sum |R|^2
follow from R.  scipy's sph_harm_y (a library routine) supplies Y_l^m.
The paper's own route (Theta and Gaunt coefficients, W tensor, spherical
Bessel functions) reaches the same R; this definition does not use it.

Parity status: pinned in tests/test_oracle_spherical.py (the plane-wave
expansion of an s Gaussian, reconstruction of the exact f, quadrature
convergence, q = 0, Parseval against an independent sphere rule).
"""
from __future__ import annotations

import numpy as np
from scipy.special import sph_harm_y

from . import form_factor


def lm_index(l: int, m: int) -> int:
    """Position of (l, m) in the flattened order l = 0.., m = -l..l."""
    return l * l + l + m


def sph_harm(lmax: int, theta, phi) -> np.ndarray:
    """Y[lm, ...] for all l <= lmax at the given angles (broadcast together)."""
    theta, phi = np.broadcast_arrays(np.asarray(theta, float), np.asarray(phi, float))
    out = np.zeros(((lmax + 1) ** 2,) + theta.shape, dtype=np.complex128)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            out[lm_index(l, m)] = sph_harm_y(l, m, theta, phi)
    return out


def sphere_rule(n_gl: int):
    """Nodes (theta[n_gl], phi[2 n_gl]) and weights w[n_gl, 2 n_gl] summing to 4 pi."""
    x, wx = np.polynomial.legendre.leggauss(n_gl)
    n_phi = 2 * n_gl
    theta = np.arccos(x)
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    w = wx[:, None] * np.full((1, n_phi), 2.0 * np.pi / n_phi)
    return theta, phi, w


def directions(theta, phi) -> np.ndarray:
    """Unit vectors [n_theta, n_phi, 3] of a product angular grid."""
    th, ph = np.meshgrid(np.asarray(theta, float), np.asarray(phi, float), indexing="ij")
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1)


def project(mol, T, q_radial, lmax: int, n_gl: int, scale: float = 1.0, renorm: bool = True,
            threads: int = 0) -> np.ndarray:
    """R[s, iq, lm] by projection of the oracle's f onto Y_l^m (l <= lmax)."""
    q_radial = np.asarray(q_radial, dtype=np.float64)
    theta, phi, w = sphere_rule(n_gl)
    u = directions(theta, phi).reshape(-1, 3)
    Yc = np.conj(sph_harm(lmax, theta[:, None], phi[None, :])).reshape((lmax + 1) ** 2, -1)
    T = np.asarray(T, dtype=np.float64)
    if T.ndim == 2:
        T = T[None]
    R = np.zeros((T.shape[0], len(q_radial), (lmax + 1) ** 2), dtype=np.complex128)
    wf = w.reshape(-1)
    for iq, qn in enumerate(q_radial):
        f = form_factor(mol, T, qn * u, scale=scale, renorm=renorm, threads=threads)  # [S, n_dir]
        R[:, iq, :] = np.einsum("sd,ld->sl", f * wf[None, :], Yc)
    return R


def reconstruct(R: np.ndarray, lmax: int, theta, phi) -> np.ndarray:
    """f[s, iq, itheta, iphi] = sum_{l <= lmax} Y_l^m R_lm on a product angular grid."""
    Y = sph_harm(lmax, np.asarray(theta, float)[:, None], np.asarray(phi, float)[None, :])
    n = (lmax + 1) ** 2
    return np.einsum("sql,ltp->sqtp", R[..., :n], Y[:n])


def isotropic_average(R: np.ndarray, lmax: int) -> np.ndarray:
    """<|f_s|^2>_Omega(q) = (1/4pi) sum_{l <= lmax, m} |R_lm(q)|^2."""
    n = (lmax + 1) ** 2
    return np.sum(np.abs(R[..., :n]) ** 2, axis=-1) / (4.0 * np.pi)
