"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
closed forms, the paper's printed p_z normalisation (Appendix A), brute-force
quadrature of the definition (tests/quadrature_ref.py), and identities the
exact result must satisfy (Hermiticity, translation phase law, rotation
covariance, inversion parity, antisymmetric-T null, small-q dipole limit).
"""
import numpy as np
import pytest

import oracle
from paper_2512_18010_b300 import workloads as W
from tests import quadrature_ref as Q


def mol_of(xyz, shells):
    """shells: list of (atom, l, exps, coefs)."""
    return W.Molecule(
        name="hand",
        xyz=np.asarray(xyz, dtype=np.float64).reshape(-1, 3),
        shell_atom=np.array([s[0] for s in shells], np.int32),
        shell_l=np.array([s[1] for s in shells], np.int32),
        shell_nprim=np.array([len(s[2]) for s in shells], np.int32),
        exponents=np.concatenate([np.asarray(s[2], float) for s in shells]),
        coefficients=np.concatenate([np.asarray(s[3], float) for s in shells]),
    )


def dfact(n):
    return 1.0 if n <= 0 else float(np.prod(np.arange(n, 0, -2)))


def prim_norm_textbook(alpha, a, b, c):
    """N^2 = (2a/pi)^{3/2} (4a)^{a+b+c} / ((2a-1)!! (2b-1)!! (2c-1)!!)."""
    return np.sqrt((2 * alpha / np.pi) ** 1.5 * (4 * alpha) ** (a + b + c)
                   / (dfact(2 * a - 1) * dfact(2 * b - 1) * dfact(2 * c - 1)))


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------- normalisation

@pytest.mark.parametrize("alpha", [0.08, 0.8, 13.0, 2900.0])
def test_pz_normalisation_matches_paper(alpha):
    # Appendix A prints N^{p_z} = (pi^{3/2} sigma^5 / 2)^{-1/2} for exp(-r^2/(2 sigma^2)).
    sigma = 1.0 / np.sqrt(2 * alpha)
    expected = (0.5 * np.pi ** 1.5 * sigma ** 5) ** -0.5
    assert oracle.prim_norm(alpha, 0, 0, 1) == pytest.approx(expected, rel=1e-14)


@pytest.mark.parametrize("pw", [(0, 0, 0), (1, 0, 0), (2, 0, 0), (1, 1, 0), (0, 1, 1),
                                (3, 0, 0), (2, 0, 1), (1, 1, 1)])
def test_primitive_normalisation_textbook(pw):
    for alpha in (0.1, 1.7, 250.0):
        assert oracle.prim_norm(alpha, *pw) == pytest.approx(prim_norm_textbook(alpha, *pw), rel=1e-13)


def test_contracted_functions_unit_norm_by_quadrature():
    job = W.config1()
    atom, pw, prims = oracle.functions(job.mol)
    for f in range(len(atom)):
        al, w = prims[f]
        s = 0.0
        for k in range(len(al)):
            for kk in range(len(al)):
                v = 1.0
                for i in range(3):
                    v *= Q._trap_axis(pw[f, i], 0.0, al[k], pw[f, i], 0.0, al[kk], 0.0).real
                s += w[k] * w[kk] * v
        assert s == pytest.approx(1.0, abs=1e-12)


# ---------------------------------------------------------------- closed forms

def test_single_s_closed_form():
    # Normalised s primitive, T = 1: f(q) = exp(i q.A) exp(-q^2 / (8 alpha)).
    A = np.array([0.3, -1.1, 0.7])
    alpha = 0.65
    mol = mol_of(A, [(0, 0, [alpha], [1.0])])
    rng = np.random.default_rng(0)
    q = rng.uniform(-9, 9, size=(50, 3))
    f = oracle.form_factor(mol, np.ones((1, 1, 1)), q)[0]
    exp = np.exp(1j * q @ A) * np.exp(-np.sum(q * q, 1) / (8 * alpha))
    assert rel_err(f, exp) < 1e-14


def _gpt(alpha, A, beta, B, q):
    p = alpha + beta
    P = (alpha * A + beta * B) / p
    K = np.exp(-alpha * beta * np.sum((A - B) ** 2) / p)
    return (np.pi / p) ** 1.5 * K * np.exp(1j * q @ P) * np.exp(-np.sum(q * q, 1) / (4 * p)), p


def test_s_s_two_centre_closed_form():
    A, B = np.array([0.0, 0.2, -0.4]), np.array([1.3, -0.5, 0.9])
    a, b = 1.4, 0.37
    mol = mol_of(np.vstack([A, B]), [(0, 0, [a], [1.0]), (1, 0, [b], [1.0])])
    T = np.array([[[0.0, 1.0], [0.0, 0.0]]])
    q = np.random.default_rng(1).uniform(-6, 6, size=(40, 3))
    f = oracle.form_factor(mol, T, q)[0]
    I, _ = _gpt(a, A, b, B, q)
    exp = prim_norm_textbook(a, 0, 0, 0) * prim_norm_textbook(b, 0, 0, 0) * I
    assert rel_err(f, exp) < 1e-13


def test_term_magnitudes_two_s_closed_form():
    # Sum of |T_mn integral_mn(q)| over the four function pairs of two s functions,
    # each integral from the Gaussian-product closed form; the sum bounds |f|.
    A, B = np.array([0.1, -0.3, 0.2]), np.array([-0.8, 0.6, 1.1])
    a, b = 0.9, 2.3
    mol = mol_of(np.vstack([A, B]), [(0, 0, [a], [1.0]), (1, 0, [b], [1.0])])
    T = np.array([[[0.7, -1.3], [0.4, -0.25]]])
    q = np.random.default_rng(5).uniform(-5, 5, size=(30, 3))
    f, term = oracle.form_factor(mol, T, q, scale=-2.0, terms=True)
    na, nb = prim_norm_textbook(a, 0, 0, 0), prim_norm_textbook(b, 0, 0, 0)
    Iaa, _ = _gpt(a, A, a, A, q)
    Iab, _ = _gpt(a, A, b, B, q)
    Ibb, _ = _gpt(b, B, b, B, q)
    exp = 2.0 * (abs(T[0, 0, 0]) * na * na * np.abs(Iaa) + (abs(T[0, 0, 1]) + abs(T[0, 1, 0])) * na * nb * np.abs(Iab)
                 + abs(T[0, 1, 1]) * nb * nb * np.abs(Ibb))
    assert np.max(np.abs(term[0] - exp) / exp) < 1e-13
    assert np.all(term[0] >= np.abs(f[0]) * (1 - 1e-14))
    f_plain = oracle.form_factor(mol, T, q, scale=-2.0)
    assert np.array_equal(f, f_plain)


def test_p_and_d_from_centre_derivatives():
    # d/dA_x exp(-a|r-A|^2) = 2a (x-A_x) exp(...): the p_x-s integral is the
    # A_x-derivative of the s-s closed form over 2a; d shells take two derivatives.
    A, B = np.array([0.1, -0.3, 0.5]), np.array([-0.8, 0.6, 1.2])
    a, b = 0.9, 0.45
    q = np.random.default_rng(2).uniform(-5, 5, size=(30, 3))
    I, p = _gpt(a, A, b, B, q)
    c1 = -2 * a * b * (A - B)[None, :] / p + 1j * q * a / p          # d(log I)/dA
    Ns = prim_norm_textbook(b, 0, 0, 0)
    # p shell on atom 0, s on atom 1: T picks phi_{p_k} phi_s
    mol = mol_of(np.vstack([A, B]), [(0, 1, [a], [1.0]), (1, 0, [b], [1.0])])
    for k in range(3):
        T = np.zeros((1, 4, 4))
        T[0, k, 3] = 1.0
        f = oracle.form_factor(mol, T, q)[0]
        exp = prim_norm_textbook(a, *[1 if i == k else 0 for i in range(3)]) * Ns * I * c1[:, k] / (2 * a)
        assert rel_err(f, exp) < 1e-13
    # Cartesian d: xx (index 0) and xy (index 1)
    mol = mol_of(np.vstack([A, B]), [(0, 2, [a], [1.0]), (1, 0, [b], [1.0])])
    T = np.zeros((1, 7, 7))
    T[0, 0, 6] = 1.0
    f = oracle.form_factor(mol, T, q)[0]
    exp = prim_norm_textbook(a, 2, 0, 0) * Ns * I * (c1[:, 0] ** 2 - 2 * a * b / p + 2 * a) / (4 * a * a)
    assert rel_err(f, exp) < 1e-12
    T = np.zeros((1, 7, 7))
    T[0, 1, 6] = 1.0
    f = oracle.form_factor(mol, T, q)[0]
    exp = prim_norm_textbook(a, 1, 1, 0) * Ns * I * c1[:, 0] * c1[:, 1] / (4 * a * a)
    assert rel_err(f, exp) < 1e-12


def test_f_from_centre_derivatives():
    # Three A_x-derivatives of g = exp(-a (x-A_x)^2) give
    # (x-A_x)^3 g = g^(3)/(8a^3) + 3 g^(1)/(4a^2); with d(log I)/dA = c1 and
    # d^2(log I)/dA_x^2 = c2 = -2ab/p the s-s integral gives I^(3) = (c1^3 + 3 c1 c2) I.
    A, B = np.array([0.4, 0.2, -0.6]), np.array([-0.5, 0.9, 0.7])
    a, b = 0.7, 1.3
    q = np.random.default_rng(12).uniform(-6, 6, size=(30, 3))
    I, p = _gpt(a, A, b, B, q)
    c1 = -2 * a * b * (A - B)[None, :] / p + 1j * q * a / p
    c2 = -2 * a * b / p
    Ns = prim_norm_textbook(b, 0, 0, 0)
    mol = mol_of(np.vstack([A, B]), [(0, 3, [a], [1.0]), (1, 0, [b], [1.0])])

    def f_of(i):
        T = np.zeros((1, 11, 11))
        T[0, i, 10] = 1.0
        return oracle.form_factor(mol, T, q)[0]

    cx, cy, cz = c1[:, 0], c1[:, 1], c1[:, 2]
    # xxx (index 0)
    exp = (prim_norm_textbook(a, 3, 0, 0) * Ns * I *
           ((cx ** 3 + 3 * cx * c2) / (8 * a ** 3) + 3 * cx / (4 * a * a)))
    assert rel_err(f_of(0), exp) < 1e-12
    # xxy (index 1): (x-A_x)^2 from two derivatives, (y-A_y) from one
    exp = prim_norm_textbook(a, 2, 1, 0) * Ns * I * (cx ** 2 + c2 + 2 * a) * cy / (8 * a ** 3)
    assert rel_err(f_of(1), exp) < 1e-12
    # xyz (index 4)
    exp = prim_norm_textbook(a, 1, 1, 1) * Ns * I * cx * cy * cz / (8 * a ** 3)
    assert rel_err(f_of(4), exp) < 1e-12
    # yzz (index 8)
    exp = prim_norm_textbook(a, 0, 1, 2) * Ns * I * cy * (cz ** 2 + c2 + 2 * a) / (8 * a ** 3)
    assert rel_err(f_of(8), exp) < 1e-12


# ---------------------------------------------------------------- brute force

def test_config1_against_quadrature():
    job = W.config1()
    rng = np.random.default_rng(3)
    q = np.vstack([np.zeros(3), rng.uniform(-10, 10, size=(7, 3)), [[0.05, -0.02, 0.01]]])
    f = oracle.form_factor(job.mol, job.T, q)
    g = Q.form_factor(job.mol, job.T, q)
    assert rel_err(f, g) < 1e-11


def test_sp_shells_against_quadrature():
    rng = np.random.default_rng(4)
    xyz = rng.uniform(-1.5, 1.5, size=(2, 3))
    mol = mol_of(xyz, [(0, -1, [3.1, 0.7], rng.standard_normal(4)),
                       (1, 0, [0.4], [1.0]), (1, 2, [0.8, 2.0], rng.standard_normal(2))])
    nbf = mol.nbf
    T = rng.standard_normal((2, nbf, nbf))
    q = rng.uniform(-7, 7, size=(6, 3))
    assert rel_err(oracle.form_factor(mol, T, q), Q.form_factor(mol, T, q)) < 1e-11


def test_f_shells_against_quadrature():
    # f on two centres (pair degree up to 6) plus d, sp and p partners, contracted.
    rng = np.random.default_rng(13)
    xyz = rng.uniform(-1.5, 1.5, size=(3, 3))
    mol = mol_of(xyz, [(0, 3, [1.4, 0.5], rng.standard_normal(2)),
                       (1, 3, [0.9], [1.0]),
                       (1, 2, [0.6, 2.2], rng.standard_normal(2)),
                       (2, -1, [2.5, 0.4], rng.standard_normal(4)),
                       (2, 1, [0.8], [1.0])])
    nbf = mol.nbf
    assert nbf == 10 + 10 + 6 + 4 + 3
    T = rng.standard_normal((2, nbf, nbf))
    q = np.vstack([np.zeros(3), rng.uniform(-7, 7, size=(6, 3))])
    assert rel_err(oracle.form_factor(mol, T, q), Q.form_factor(mol, T, q)) < 1e-11


# ---------------------------------------------------------------- pure (spherical-harmonic) shells

def _pure_mol(xyz, shells, pure=W.PURE_D | W.PURE_F):
    m = mol_of(xyz, shells)
    return W.Molecule(**{**m.__dict__, "pure": pure})


def _real_sph_harm(l, m, theta, phi):
    """Real spherical harmonics from scipy's complex Y_l^m (any fixed sign convention)."""
    from scipy.special import sph_harm_y
    y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return np.sqrt(2) * y.real
    if m < 0:
        return np.sqrt(2) * y.imag
    return y.real


@pytest.mark.parametrize("l", [2, 3])
def test_pure_polynomials_are_the_real_solid_harmonics(l):
    # Each polynomial of the quadrature reference's table is r^l Z_lm up to a
    # constant factor: their ratio is the same at random points of the sphere.
    rng = np.random.default_rng(40 + l)
    v = rng.standard_normal((25, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    theta, phi = np.arccos(v[:, 2]), np.arctan2(v[:, 1], v[:, 0])
    for i, terms in enumerate(Q.PURE[l]):
        m = i - l
        poly = sum(k * v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c for k, (a, b, c) in terms)
        ratio = poly / _real_sph_harm(l, m, theta, phi)
        assert np.ptp(ratio) < 1e-10 * np.max(np.abs(ratio)), (l, m)


def test_pure_shells_against_quadrature():
    rng = np.random.default_rng(41)
    xyz = rng.uniform(-1.4, 1.4, size=(3, 3))
    mol = _pure_mol(xyz, [(0, 2, [1.3, 0.4], rng.standard_normal(2)),
                          (0, 3, [0.9], [1.0]),
                          (1, 3, [1.6, 0.5], rng.standard_normal(2)),
                          (1, -1, [2.0, 0.6], rng.standard_normal(4)),
                          (2, 2, [0.7], [1.0]),
                          (2, 0, [0.5], [1.0])])
    assert mol.nbf == 5 + 7 + 7 + 4 + 5 + 1
    T = rng.standard_normal((2, mol.nbf, mol.nbf))
    q = np.vstack([np.zeros(3), rng.uniform(-6, 6, size=(5, 3))])
    for renorm in (True, False):
        f = oracle.form_factor(mol, T, q, renorm=renorm)
        g = Q.form_factor(mol, T, q, renorm=renorm)
        assert rel_err(f, g) < 1e-11


def test_pure_functions_orthonormal_on_one_centre():
    # One primitive per shell, no contraction rescaling: the Appendix A
    # normalisation (with its cross terms) must give unit norm by itself; the
    # harmonics are orthogonal to each other and to lower degrees on the same
    # centre (d to s, f to p).
    A = np.array([[0.3, -0.2, 0.5]])
    mol = _pure_mol(A, [(0, 0, [0.8], [1.0]), (0, 1, [1.1], [1.0]), (0, 2, [0.6], [1.0]), (0, 3, [0.9], [1.0])])
    n = mol.nbf
    assert n == 16
    E = np.zeros((n * n, n, n))
    for i in range(n):
        for j in range(n):
            E[i * n + j, i, j] = 1.0
    S = oracle.form_factor(mol, E, np.zeros((1, 3)), renorm=False)[:, 0].real.reshape(n, n)
    d, f = slice(4, 9), slice(9, 16)
    assert np.allclose(S[d, d], np.eye(5), atol=1e-13)
    assert np.allclose(S[f, f], np.eye(7), atol=1e-13)
    assert np.max(np.abs(S[0, d])) < 1e-13
    assert np.max(np.abs(S[1:4, f])) < 1e-13


@pytest.mark.parametrize("l", [2, 3])
def test_pure_shell_density_is_isotropic(l):
    # sum_m phi_m^2 over a full pure shell is spherically symmetric (addition
    # theorem), so with T = identity on the shell f(q) depends on |q| only.
    # A Cartesian shell fails this (its components are not equally normalised).
    mol = _pure_mol(np.zeros((1, 3)), [(0, l, [1.2, 0.35], [0.6, 0.5])])
    T = np.eye(mol.nbf)[None]
    rng = np.random.default_rng(42 + l)
    u = rng.standard_normal((12, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    for qn in (0.7, 2.5, 5.0):
        f = oracle.form_factor(mol, T, qn * u)[0]
        assert np.max(np.abs(f - f[0])) < 1e-12 * abs(f[0])
    cart = mol_of(np.zeros((1, 3)), [(0, l, [1.2, 0.35], [0.6, 0.5])])
    fc = oracle.form_factor(cart, np.eye(cart.nbf)[None], 2.5 * u)[0]
    assert np.max(np.abs(fc - fc[0])) > 1e-3 * abs(fc[0])


def test_real_space_3d_sum_tiny():
    # Phi(r) = sum T phi phi tabulated on a 3-D grid and Fourier-summed directly.
    xyz = np.array([[0.0, 0.0, -0.7], [0.2, 0.1, 0.8]])
    mol = mol_of(xyz, [(0, 0, [0.9], [1.0]), (0, 1, [0.6], [1.0]), (1, 0, [0.5], [1.0])])
    rng = np.random.default_rng(5)
    T = rng.standard_normal((1, 5, 5))
    qb = Q.QuadBasis(mol)
    h = 0.11
    x = np.arange(-9.0, 9.0 + h / 2, h)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    phis = []
    for (A, terms, al, w) in qb.fn:
        dx, dy, dz = X - A[0], Y - A[1], Z - A[2]
        r2 = dx * dx + dy * dy + dz * dz
        v = sum(wk * np.exp(-ak * r2) for ak, wk in zip(al, w))
        phis.append(sum(k * dx ** pw[0] * dy ** pw[1] * dz ** pw[2] for k, pw in terms) * v)
    Phi = sum(T[0, m, n] * phis[m] * phis[n] for m in range(5) for n in range(5))
    qs = np.array([[0.0, 0.0, 0.0], [0.5, -0.3, 1.1], [2.0, 1.0, -1.5], [-3.0, 0.4, 0.2]])
    f = oracle.form_factor(mol, T, qs)[0]
    g = np.array([np.sum(Phi * np.exp(1j * (q[0] * X + q[1] * Y + q[2] * Z))) * h ** 3 for q in qs])
    assert rel_err(f, g) < 1e-8


# ---------------------------------------------------------------- identities

def test_overlap_trace_at_q0():
    job = W.config1()
    S = Q.QuadBasis(job.mol).matrix(np.zeros(3)).real
    assert np.allclose(np.diag(S), 1.0, atol=1e-12)
    f0 = oracle.form_factor(job.mol, job.T, np.zeros((1, 3)))[0, 0]
    assert abs(f0 - np.trace(job.T[0] @ S.T)) < 1e-12
    assert abs(f0.imag) < 1e-15


def test_hermiticity_on_antisymmetric_grid():
    job = W.config1()
    idx = W.subset_indices(job.nq, 300, 11)
    n = len(job.qx)
    ix, iy, iz = idx // (n * n), (idx // n) % n, idx % n
    mirror = ((n - 1 - ix) * n + (n - 1 - iy)) * n + (n - 1 - iz)
    f = oracle.grid_form_factor(job, idx)
    g = oracle.grid_form_factor(job, mirror)
    assert np.array_equal(job.q_points(mirror), -job.q_points(idx))
    assert rel_err(np.conj(g), f) < 1e-14


def test_translation_phase_law():
    job = W.config2()
    a = np.array([0.37, -1.25, 2.1])
    q = np.random.default_rng(6).uniform(-15, 15, size=(40, 3))
    T = job.T[:3]
    f = oracle.form_factor(job.mol, T, q)
    g = oracle.form_factor(job.mol.translated(a), T, q)
    assert rel_err(g, f * np.exp(1j * q @ a)[None, :]) < 1e-11


def _rotation_map(mol, R):
    """G with phi_i o R^T = sum_j G[j, i] phi'_j, block-diagonal over shells."""
    blocks = []
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ratio = {(0, 0): 1 / np.sqrt(3), (1, 1): 1 / np.sqrt(3), (2, 2): 1 / np.sqrt(3)}
    for l in mol.shell_l:
        l = int(l)
        if l == 0:
            blocks.append(np.eye(1))
        elif l == 1:
            blocks.append(R.copy())
        elif l == -1:
            b = np.eye(4)
            b[1:, 1:] = R
            blocks.append(b)
        else:
            G = np.zeros((6, 6))
            for col, (a, b) in enumerate(pairs):
                Ka = ratio.get((a, b), 1.0)
                for row, (j, k) in enumerate(pairs):
                    Kj = ratio.get((j, k), 1.0)
                    c = R[j, a] * R[k, b] + (R[k, a] * R[j, b] if j != k else 0.0)
                    G[row, col] = Ka / Kj * c
            blocks.append(G)
    n = sum(b.shape[0] for b in blocks)
    G = np.zeros((n, n))
    o = 0
    for b in blocks:
        m = b.shape[0]
        G[o:o + m, o:o + m] = b
        o += m
    return G


def test_rotation_covariance():
    job = W.config1()  # has p and Cartesian d shells
    R = W.random_rotation(np.random.default_rng(7))
    mol2 = W.Molecule(**{**job.mol.__dict__, "xyz": job.mol.xyz @ R.T})
    G = _rotation_map(job.mol, R)
    T2 = np.einsum("ji,sik,lk->sjl", G, job.T, G)
    q = np.random.default_rng(8).uniform(-8, 8, size=(40, 3))
    f = oracle.form_factor(job.mol, job.T, q)
    g = oracle.form_factor(mol2, T2, q @ R.T)
    assert rel_err(g, f) < 1e-11


def _monomials(l):
    """Cartesian exponents of degree l, descending x power then descending y power."""
    return [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]


def _rotation_map_lsq(mol, R):
    """Same map as _rotation_map, found numerically for any shell.

    m_i(R^T x) = sum_j M[j, i] m_j(x) is solved by least squares on random
    points (exact: both sides are homogeneous of the same degree); the
    primitive normalisation ratio N_i / N_j = prod Gamma(a_j + 1/2)^(1/2) /
    prod Gamma(a_i + 1/2)^(1/2) does not depend on the exponent.
    """
    from math import gamma
    x = np.random.default_rng(99).standard_normal((64, 3))
    blocks = []
    for l in mol.shell_l:
        l = int(l)
        comps = [(0, 0, 0)] + _monomials(1) if l == -1 else _monomials(l)
        V = np.array([[np.prod(xx ** np.array(c)) for c in comps] for xx in x])
        Y = np.array([[np.prod((R.T @ xx) ** np.array(c)) for c in comps] for xx in x])
        M = np.linalg.lstsq(V, Y, rcond=None)[0]
        N = np.array([np.prod([gamma(e + 0.5) for e in c]) ** -0.5 for c in comps])
        blocks.append(M * N[None, :] / N[:, None])
    n = sum(b.shape[0] for b in blocks)
    G = np.zeros((n, n))
    o = 0
    for b in blocks:
        m = b.shape[0]
        G[o:o + m, o:o + m] = b
        o += m
    return G


def test_rotation_covariance_f_shells():
    job = W.config_f(n_heavy=2, n_states=2, n=8)
    R = W.random_rotation(np.random.default_rng(17))
    assert np.allclose(_rotation_map_lsq(W.config1().mol, R), _rotation_map(W.config1().mol, R), atol=1e-12)
    mol2 = W.Molecule(**{**job.mol.__dict__, "xyz": job.mol.xyz @ R.T})
    G = _rotation_map_lsq(job.mol, R)
    T2 = np.einsum("ji,sik,lk->sjl", G, job.T, G)
    q = np.random.default_rng(18).uniform(-8, 8, size=(30, 3))
    f = oracle.form_factor(job.mol, job.T, q)
    g = oracle.form_factor(mol2, T2, q @ R.T)
    assert rel_err(g, f) < 1e-11


def test_antisymmetric_T_gives_zero():
    job = W.config1()
    A = job.T - np.transpose(job.T, (0, 2, 1))
    q = np.random.default_rng(9).uniform(-10, 10, size=(40, 3))
    f = oracle.form_factor(job.mol, A, q)
    ref = oracle.form_factor(job.mol, np.abs(job.T), q)
    assert np.max(np.abs(f)) < 1e-13 * np.max(np.abs(ref))


def test_inversion_parity():
    # Centrosymmetric molecule: T' = (T +- P^T T P)/2 gives purely real / imaginary f.
    rng = np.random.default_rng(10)
    A = rng.uniform(-1.5, 1.5, size=(2, 3))
    xyz = np.vstack([A, -A])
    base = [(0, 0, [2.0, 0.5]), (0, -1, [1.1, 0.3]), (0, 2, [0.8]), (1, 0, [0.9, 0.2]),
            (1, 3, [0.7])]
    shells = []
    coefs = [rng.standard_normal(len(e) * (2 if l == -1 else 1)) for (_, l, e) in base]
    for partner in (0, 2):
        for (at, l, e), c in zip(base, coefs):
            shells.append((at + partner, l, e, c))
    mol = mol_of(xyz, shells)
    n = mol.nbf
    half = n // 2
    sign = []
    for (_, l, _) in base:
        sign += {0: [1], -1: [1, -1, -1, -1], 2: [1] * 6, 1: [-1] * 3, 3: [-1] * 10}[l]
    P = np.zeros((n, n))
    for i in range(half):
        P[half + i, i] = sign[i]
        P[i, half + i] = sign[i]
    T = rng.standard_normal((1, n, n))
    Tp = np.einsum("ji,sjk,kl->sil", P, T, P)
    q = rng.uniform(-6, 6, size=(30, 3))
    fe = oracle.form_factor(mol, (T + Tp) / 2, q)
    fo = oracle.form_factor(mol, (T - Tp) / 2, q)
    assert np.max(np.abs(fe.imag)) < 1e-13 * np.max(np.abs(fe))
    assert np.max(np.abs(fo.real)) < 1e-13 * np.max(np.abs(fo))


def test_small_q_dipole_limit():
    # f(q) = f(0) + i q.d + O(q^2), d = sum T <phi|r|phi> (transition dipole, Sec. Verification).
    job = W.config1()
    qb = Q.QuadBasis(job.mol)
    D = qb.dipole_matrices()
    d = np.einsum("mn,kmn->k", job.T[0], D)
    h = 1e-4
    for u in np.eye(3):
        fp = oracle.form_factor(job.mol, job.T, (h * u)[None])[0, 0]
        fm = oracle.form_factor(job.mol, job.T, (-h * u)[None])[0, 0]
        deriv = (fp - fm) / (2j * h)
        assert abs(deriv - d @ u) < 1e-7 * max(1.0, np.linalg.norm(d))


def test_angular_average_fit_gives_dipole():
    # <|f|^2>_Omega ~ A + B q^2 + C q^4 with B = |d|^2 / 3 for a T with f(0) = 0.
    job = W.config1()
    qb = Q.QuadBasis(job.mol)
    S = qb.matrix(np.zeros(3)).real
    T = job.T[0] - np.trace(job.T[0] @ S.T) / np.trace(S) * np.eye(job.mol.nbf)
    d = np.einsum("mn,kmn->k", T, qb.dipole_matrices())
    # Fibonacci sphere directions (area-uniform), radii up to 0.05 Bohr^-1
    m = 600
    i = np.arange(m) + 0.5
    th = np.arccos(1 - 2 * i / m)
    ph = np.pi * (1 + 5 ** 0.5) * i
    dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    radii = np.linspace(0.005, 0.05, 8)
    avg = []
    for r in radii:
        f = oracle.form_factor(job.mol, T[None], r * dirs)[0]
        avg.append(np.mean(np.abs(f) ** 2))
    Mfit = np.stack([np.ones_like(radii), radii ** 2, radii ** 4], 1)
    A_, B_, C_ = np.linalg.lstsq(Mfit, np.array(avg), rcond=None)[0]
    assert B_ == pytest.approx(np.dot(d, d) / 3, rel=2e-3)
