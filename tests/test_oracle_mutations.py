"""The oracle pins are sensitive: each plausible mistake planted in a copy of
the oracle source (a dropped term, a wrong sign, swapped operands, a wrong
exponent, a wrong offset) must fail at least one pin, and the unmodified
source must pass them all.  Mistakes are planted only in a temporary copy of
the oracle, compiled on the CPU."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2512_18010_b300 import workloads as W
from tests import quadrature_ref as Q
from tests.test_oracle_pins import _gpt, mol_of, prim_norm_textbook

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "scff_oracle.c")

MUTATIONS = {
    "phase_sign": ("total += m->w[k] * n->w[kk] * K * ang * cexp(I * phase);",
                   "total += m->w[k] * n->w[kk] * K * ang * cexp(-I * phase);"),
    "dropped_recurrence_term": ("J[t + 1] = (I * q * J[t] + (double)t * J[t - 1]) / (2.0 * p);",
                                "J[t + 1] = (I * q * J[t]) / (2.0 * p);"),
    "swapped_centres": ("binomial_product(m->pw[ti][i], P[i] - A[i], n->pw[tj][i], P[i] - B[i], e);",
                        "binomial_product(m->pw[ti][i], P[i] - B[i], n->pw[tj][i], P[i] - A[i], e);"),
    "gamma_argument": ("prod *= pow(sigma, 1.0 + 2.0 * e[i]) * tgamma(e[i] + 0.5);",
                       "prod *= pow(sigma, 1.0 + 2.0 * e[i]) * tgamma(e[i] + 1.5);"),
    "gaussian_width": ("J[0] = sqrt(M_PI / p) * exp(-q * q / (4.0 * p));",
                       "J[0] = sqrt(M_PI / p) * exp(-q * q / (2.0 * p));"),
    "gpt_prefactor": ("const double K = exp(-al * be * AB2 / p);",
                      "const double K = exp(-al * be * AB2 / (2.0 * p));"),
    "sp_coefficient_offset": ("const double *c = coefs + coff + ((l == -1 && i > 0) ? (size_t)np : 0);",
                              "const double *c = coefs + coff;"),
    "no_contraction_renorm": ("for (int k = 0; k < np; ++k) fn->w[k] *= r;", "(void)r;"),
    "d_component_order": ("{1, 1, 0}, {1, 0, 1},\n                                 {0, 2, 0}",
                          "{1, 0, 1}, {1, 1, 0},\n                                 {0, 2, 0}"),
    "binomial_power": ("ea[i] = C[a][i] * pow(u, a - i);", "ea[i] = C[a][i] * pow(u, i);"),
    "f_component_order": ("{{3, 0, 0}, {2, 1, 0}, {2, 0, 1}", "{{3, 0, 0}, {2, 0, 1}, {2, 1, 0}"),
    "cubic_binomial": ("{1, 2, 1, 0}, {1, 3, 3, 1}}", "{1, 2, 1, 0}, {1, 2, 2, 1}}"),
    "pure_dz2_coefficient": ("{2.0, -1.0, -1.0}},\n    {1, {{1, 0, 1}}", "{1.0, -1.0, -1.0}},\n    {1, {{1, 0, 1}}"),
    "pure_norm_cross_terms": ("        for (int j = 0; j < nterm; ++j) {\n            double prod = k[i] * k[j];",
                              "        for (int j = i; j <= i; ++j) {\n            double prod = k[i] * k[j];"),
    "pure_f_coefficient": ("{4.0, -1.0, -1.0}},\n    {3, {{0, 0, 3},", "{3.0, -1.0, -1.0}},\n    {3, {{0, 0, 3},"),
}


def compile_variant(src_text, path):
    c_path = path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", path, c_path, "-lm"],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.scff_oracle_form_factor.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                            ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_double, P, ctypes.c_int]
    lib.scff_oracle_prim_norm.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.scff_oracle_prim_norm.restype = ctypes.c_double
    return lib


def ff(lib, mol, T, q, flags=1):
    c = lambda a, d: np.ascontiguousarray(a, dtype=d)  # noqa: E731
    xyz, sa, sl, sn = c(mol.xyz, np.float64), c(mol.shell_atom, np.int32), c(mol.shell_l, np.int32), \
        c(mol.shell_nprim, np.int32)
    ex, co = c(mol.exponents, np.float64), c(mol.coefficients, np.float64)
    T = c(T, np.float64)
    q = c(q, np.float64).reshape(-1, 3)
    out = np.zeros((T.shape[0], q.shape[0], 2))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = lib.scff_oracle_form_factor(mol.n_atoms, p(xyz), mol.n_shells, p(sa), p(sl), p(sn), p(ex), p(co), flags,
                                     T.shape[0], p(T), q.shape[0], p(q), 1.0, p(out), 2)
    assert rc == 0
    return out[..., 0] + 1j * out[..., 1]


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def pins_pass(lib):
    """Quick versions of the oracle pins; True when all hold."""
    rng = np.random.default_rng(0)
    ok = []
    # p_z normalisation printed in Appendix A
    sigma = 1 / np.sqrt(2 * 0.7)
    ok.append(abs(lib.scff_oracle_prim_norm(0.7, 0, 0, 1) - (0.5 * np.pi ** 1.5 * sigma ** 5) ** -0.5) < 1e-12)
    # single normalised s primitive
    A = np.array([0.3, -1.1, 0.7])
    q = rng.uniform(-6, 6, size=(10, 3))
    f = ff(lib, mol_of(A, [(0, 0, [0.65], [1.0])]), np.ones((1, 1, 1)), q)[0]
    ok.append(rel(f, np.exp(1j * q @ A) * np.exp(-np.sum(q * q, 1) / (8 * 0.65))) < 1e-12)
    # two-centre s-s
    B = np.array([1.3, -0.5, 0.9])
    m = mol_of(np.vstack([A, B]), [(0, 0, [1.4], [1.0]), (1, 0, [0.37], [1.0])])
    I, _ = _gpt(1.4, A, 0.37, B, q)
    f = ff(lib, m, np.array([[[0.0, 1.0], [0.0, 0.0]]]), q)[0]
    ok.append(rel(f, prim_norm_textbook(1.4, 0, 0, 0) * prim_norm_textbook(0.37, 0, 0, 0) * I) < 1e-12)
    # quadrature brute force: config 1 (s, p, d) and an sp case
    job = W.config1()
    qq = np.vstack([np.zeros(3), rng.uniform(-8, 8, size=(2, 3))])
    ok.append(rel(ff(lib, job.mol, job.T, qq), Q.form_factor(job.mol, job.T, qq)) < 1e-10)
    msp = mol_of(rng.uniform(-1.5, 1.5, size=(2, 3)),
                 [(0, -1, [3.1, 0.7], rng.standard_normal(4)), (1, 0, [0.4], [1.0])])
    Tsp = rng.standard_normal((1, msp.nbf, msp.nbf))
    ok.append(rel(ff(lib, msp, Tsp, qq), Q.form_factor(msp, Tsp, qq)) < 1e-10)
    # f shells: one f primitive on each of two centres, every component pair
    mf = mol_of(rng.uniform(-1.5, 1.5, size=(2, 3)), [(0, 3, [1.1], [1.0]), (1, 3, [0.6], [1.0])])
    Tf = rng.standard_normal((1, 20, 20))
    ok.append(rel(ff(lib, mf, Tf, qq), Q.form_factor(mf, Tf, qq)) < 1e-10)
    # pure d and f shells, without contraction rescaling (which would hide a
    # wrong primitive normalisation)
    mp = mol_of(rng.uniform(-1.5, 1.5, size=(2, 3)), [(0, 2, [1.1], [1.0]), (1, 3, [0.6], [1.0])])
    mp = W.Molecule(**{**mp.__dict__, "pure": W.PURE_D | W.PURE_F})
    Tp = rng.standard_normal((1, 12, 12))
    ok.append(rel(ff(lib, mp, Tp, qq, flags=6), Q.form_factor(mp, Tp, qq, renorm=False)) < 1e-10)
    return all(ok)


def test_unmodified_oracle_passes_quick_pins(tmp_path):
    lib = compile_variant(open(SRC).read(), str(tmp_path / "ok.so"))
    assert pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, f"mutation site for {name} not found"
    lib = compile_variant(src.replace(old, new), str(tmp_path / f"{name}.so"))
    assert not pins_pass(lib), f"planted mistake '{name}' passed every pin"
