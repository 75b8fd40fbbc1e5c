"""Brute-force reference for the form factor by numerical quadrature.

Independent of both the oracle and the CUDA library: it builds the basis
functions from the raw shell definitions itself, normalises primitives and
contractions numerically, and integrates each primitive pair's Fourier
integral per axis with the trapezoid rule (exponentially convergent for
Gaussian integrands).  The 3-D integral of a product of two Cartesian
Gaussian primitives factorises exactly into three 1-D integrals, so this is
the definition f_s(q) = sum T^s_{mu nu} Int phi_mu phi_nu e^{iq.r} d^3r
written out with quadrature in place of algebra.
"""
from __future__ import annotations

import numpy as np

_COMP = {
    0: [(0, 0, 0)],
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)],
    3: [(3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2),
        (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)],
    -1: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
}

# Pure (spherical-harmonic) shells: the real solid harmonics r^l Z_lm as
# Cartesian polynomials [(k, (a, b, c)), ...], m = -l..l.  Their harmonicity
# and their match with sympy's real spherical harmonics are tested separately.
PURE = {
    2: [[(1, (1, 1, 0))],
        [(1, (0, 1, 1))],
        [(2, (0, 0, 2)), (-1, (2, 0, 0)), (-1, (0, 2, 0))],
        [(1, (1, 0, 1))],
        [(1, (2, 0, 0)), (-1, (0, 2, 0))]],
    3: [[(3, (2, 1, 0)), (-1, (0, 3, 0))],
        [(1, (1, 1, 1))],
        [(4, (0, 1, 2)), (-1, (2, 1, 0)), (-1, (0, 3, 0))],
        [(2, (0, 0, 3)), (-3, (2, 0, 1)), (-3, (0, 2, 1))],
        [(4, (1, 0, 2)), (-1, (3, 0, 0)), (-1, (1, 2, 0))],
        [(1, (2, 0, 1)), (-1, (0, 2, 1))],
        [(1, (3, 0, 0)), (-3, (1, 2, 0))]],
}
PURE_FLAG = {2: 2, 3: 4}


def _trap_axis(a, A, alpha, b, B, beta, q):
    """Int (x-A)^a (x-B)^b exp(-alpha (x-A)^2 - beta (x-B)^2 + i q x) dx by trapezoid."""
    p = alpha + beta
    P = (alpha * A + beta * B) / p
    half = np.sqrt(80.0 / p) + 1.0 / np.sqrt(p)
    h = 2 * np.pi / (abs(q) + np.sqrt(300.0 * p)) / 1.5
    n = int(np.ceil(2 * half / h)) + 1
    x = P + np.linspace(-half, half, n)
    dx = x[1] - x[0]
    g = (x - A) ** a * (x - B) ** b * np.exp(-alpha * (x - A) ** 2 - beta * (x - B) ** 2)
    return np.sum(g * np.exp(1j * q * x)) * dx


class QuadBasis:
    """Contracted Gaussians (Cartesian or pure) normalised by quadrature."""

    def __init__(self, mol, renorm=True):
        self.fn = []   # (center[3], terms [(k, powers)], alphas[k], weights[k])
        pure_bits = int(getattr(mol, "pure", 0))
        eo = co = 0
        for s in range(mol.n_shells):
            l = int(mol.shell_l[s])
            np_ = int(mol.shell_nprim[s])
            A = np.asarray(mol.xyz[int(mol.shell_atom[s])], dtype=np.float64)
            al = np.asarray(mol.exponents[eo:eo + np_], dtype=np.float64)
            if l in PURE and pure_bits & PURE_FLAG[l]:
                funcs = PURE[l]
            else:
                funcs = [[(1, pw)] for pw in _COMP[l]]
            for i, terms in enumerate(funcs):
                off = co + (np_ if (l == -1 and i > 0) else 0)
                c = np.asarray(mol.coefficients[off:off + np_], dtype=np.float64)
                # primitive normalisation by quadrature: Int chi^2 = 1
                nrm = np.array([self._self_overlap(terms, a_) for a_ in al])
                w = c / np.sqrt(nrm)
                self.fn.append([A, terms, al, w])
            eo += np_
            co += np_ * (2 if l == -1 else 1)
        if renorm:
            for f in self.fn:
                s = self._pair(f, f, np.zeros(3)).real
                f[3] = f[3] / np.sqrt(s)

    @staticmethod
    def _self_overlap(terms, alpha):
        tot = 0.0
        for ka, pa in terms:
            for kb, pb in terms:
                v = ka * kb
                for i in range(3):
                    v *= _trap_axis(pa[i], 0.0, alpha, pb[i], 0.0, alpha, 0.0).real
                tot += v
        return tot

    def _pair(self, f, g, q):
        A, ta, aa, wa = f
        B, tb, ab, wb = g
        tot = 0j
        for k in range(len(aa)):
            for kk in range(len(ab)):
                for ka, pa in ta:
                    for kb, pb in tb:
                        v = ka * kb + 0j
                        for i in range(3):
                            v *= _trap_axis(pa[i], A[i], aa[k], pb[i], B[i], ab[kk], q[i])
                        tot += wa[k] * wb[kk] * v
        return tot

    @property
    def nbf(self):
        return len(self.fn)

    def matrix(self, q):
        """M[mu, nu] = Int phi_mu phi_nu e^{i q.r} d^3r."""
        n = self.nbf
        M = np.zeros((n, n), dtype=np.complex128)
        for i in range(n):
            for j in range(i, n):
                M[i, j] = self._pair(self.fn[i], self.fn[j], q)
                M[j, i] = M[i, j]
        return M

    def dipole_matrices(self):
        """D_k[mu, nu] = Int phi_mu r_k phi_nu d^3r by quadrature (k = x, y, z)."""
        n = self.nbf
        D = np.zeros((3, n, n))
        for i in range(n):
            for j in range(n):
                A, ta, aa, wa = self.fn[i]
                B, tb, ab, wb = self.fn[j]
                assert len(ta) == 1 and len(tb) == 1, "dipole_matrices: Cartesian functions only"
                pa, pb = ta[0][1], tb[0][1]
                for k in range(3):
                    tot = 0.0
                    for u in range(len(aa)):
                        for v in range(len(ab)):
                            val = 1.0
                            for ax in range(3):
                                if ax == k:
                                    # r_k = (x - B) + B
                                    m1 = _trap_axis(pa[ax], A[ax], aa[u], pb[ax] + 1, B[ax], ab[v], 0.0).real
                                    m0 = _trap_axis(pa[ax], A[ax], aa[u], pb[ax], B[ax], ab[v], 0.0).real
                                    val *= m1 + B[ax] * m0
                                else:
                                    val *= _trap_axis(pa[ax], A[ax], aa[u], pb[ax], B[ax], ab[v], 0.0).real
                            tot += wa[u] * wb[v] * val
                    D[k, i, j] = tot
        return D


def form_factor(mol, T, qs, renorm=True):
    """f[s, iq] by quadrature for q vectors qs[n, 3]."""
    qb = QuadBasis(mol, renorm=renorm)
    T = np.asarray(T)
    if T.ndim == 2:
        T = T[None]
    out = np.zeros((T.shape[0], len(qs)), dtype=np.complex128)
    for iq, q in enumerate(np.asarray(qs, dtype=np.float64)):
        M = qb.matrix(q)
        out[:, iq] = np.einsum("smn,mn->s", T, M)
    return out
