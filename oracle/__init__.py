"""FP64 CPU oracle for the transition form factor -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may load or call this package.  The product path (the CUDA
library and its Python binding) never imports it.

``build()`` compiles ``scff_oracle.c`` with gcc/OpenMP into
``oracle/libscff_oracle.so``; the wrappers below marshal numpy arrays into its
C entry points.  The definition it evaluates and the route it takes are
stated in the header of ``scff_oracle.c``.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, quadrature brute force,
symmetry identities); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scff_oracle.c")
_LIB = os.path.join(_HERE, "libscff_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, IEEE FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
               "-fno-fast-math", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.scff_oracle_form_factor.argtypes = [
            ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
            ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_double, P, ctypes.c_int]
        lib.scff_oracle_form_factor.restype = ctypes.c_int
        lib.scff_oracle_form_factor_terms.argtypes = [
            ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
            ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_double, P, P, ctypes.c_int]
        lib.scff_oracle_form_factor_terms.restype = ctypes.c_int
        lib.scff_oracle_functions.argtypes = [
            ctypes.c_int, ctypes.c_int, P, P, P, P, P, ctypes.c_int, P, P, P, P, P]
        lib.scff_oracle_functions.restype = ctypes.c_int
        lib.scff_oracle_prim_norm.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.scff_oracle_prim_norm.restype = ctypes.c_double
        lib.scff_oracle_nbf.argtypes = [ctypes.c_int, P, ctypes.c_int]
        lib.scff_oracle_density.argtypes = [
            ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
            ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_double, P, ctypes.c_int]
        lib.scff_oracle_density.restype = ctypes.c_int
        lib.scff_oracle_nbf.restype = ctypes.c_int
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# flag bits of the C entry points (same meaning as the library's basis flags)
RENORM, PURE_D, PURE_F = 1, 2, 4


def _flags(mol, renorm: bool) -> int:
    return (RENORM if renorm else 0) | (int(getattr(mol, "pure", 0)) & (PURE_D | PURE_F))


def form_factor(mol, T: np.ndarray, q: np.ndarray, scale: float = 1.0,
                renorm: bool = True, threads: int = 0, terms: bool = False):
    """f[s, iq] (complex128) for explicit q vectors q[n, 3].

    With terms=True also returns term[s, iq] = |scale| sum_{mu,nu} |T^s_{mu nu}
    integral_{mu nu}(q)|, the sum of the magnitudes of the terms whose sum is
    f (so term >= |f|); max term / max |f| measures how far cancellation
    amplifies the rounding of the terms.
    """
    lib = _load()
    xyz = _c(mol.xyz, np.float64)
    sa, sl, sn = _c(mol.shell_atom, np.int32), _c(mol.shell_l, np.int32), _c(mol.shell_nprim, np.int32)
    ex, co = _c(mol.exponents, np.float64), _c(mol.coefficients, np.float64)
    T = _c(T, np.float64)
    if T.ndim == 2:
        T = T[None]
    q = _c(q, np.float64).reshape(-1, 3)
    S = T.shape[0]
    out = np.zeros((S, q.shape[0], 2), dtype=np.float64)
    if terms:
        term = np.zeros((S, q.shape[0]), dtype=np.float64)
        rc = lib.scff_oracle_form_factor_terms(mol.n_atoms, _ptr(xyz), mol.n_shells, _ptr(sa), _ptr(sl),
                                               _ptr(sn), _ptr(ex), _ptr(co), _flags(mol, renorm), S, _ptr(T),
                                               q.shape[0], _ptr(q), float(scale), _ptr(out), _ptr(term),
                                               int(threads))
    else:
        rc = lib.scff_oracle_form_factor(mol.n_atoms, _ptr(xyz), mol.n_shells, _ptr(sa), _ptr(sl),
                                         _ptr(sn), _ptr(ex), _ptr(co), _flags(mol, renorm), S, _ptr(T),
                                         q.shape[0], _ptr(q), float(scale), _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    f = out[..., 0] + 1j * out[..., 1]
    return (f, term) if terms else f


def density(mol, T: np.ndarray, r: np.ndarray, scale: float = 1.0, renorm: bool = True,
            threads: int = 0) -> np.ndarray:
    """Phi[s, ir] = scale * sum T^s[mu][nu] phi_mu(r) phi_nu(r) at points r[n, 3]."""
    lib = _load()
    xyz = _c(mol.xyz, np.float64)
    sa, sl, sn = _c(mol.shell_atom, np.int32), _c(mol.shell_l, np.int32), _c(mol.shell_nprim, np.int32)
    ex, co = _c(mol.exponents, np.float64), _c(mol.coefficients, np.float64)
    T = _c(T, np.float64)
    if T.ndim == 2:
        T = T[None]
    r = _c(r, np.float64).reshape(-1, 3)
    out = np.zeros((T.shape[0], r.shape[0]), dtype=np.float64)
    rc = lib.scff_oracle_density(mol.n_atoms, _ptr(xyz), mol.n_shells, _ptr(sa), _ptr(sl), _ptr(sn),
                                 _ptr(ex), _ptr(co), _flags(mol, renorm), T.shape[0], _ptr(T), r.shape[0],
                                 _ptr(r), float(scale), _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return out


def functions(mol, renorm: bool = True):
    """Function table of a Cartesian basis: (atom[nbf], powers[nbf,3], list of (alpha[k], weight[k]))."""
    if _flags(mol, False):
        raise ValueError("functions() describes Cartesian shells only")
    lib = _load()
    sa, sl, sn = _c(mol.shell_atom, np.int32), _c(mol.shell_l, np.int32), _c(mol.shell_nprim, np.int32)
    ex, co = _c(mol.exponents, np.float64), _c(mol.coefficients, np.float64)
    nbf = lib.scff_oracle_nbf(mol.n_shells, _ptr(sl), 0)
    if nbf <= 0:
        raise ValueError("bad shell codes")
    maxp = int(np.sum(10 * np.asarray(mol.shell_nprim, dtype=np.int64))) + 1
    atom = np.zeros(nbf, np.int32)
    pw = np.zeros((nbf, 3), np.int32)
    npr = np.zeros(nbf, np.int32)
    al = np.zeros(maxp, np.float64)
    w = np.zeros(maxp, np.float64)
    rc = lib.scff_oracle_functions(mol.n_atoms, mol.n_shells, _ptr(sa), _ptr(sl), _ptr(sn), _ptr(ex),
                                   _ptr(co), int(renorm), _ptr(atom), _ptr(pw), _ptr(npr), _ptr(al), _ptr(w))
    if rc < 0:
        raise ValueError(f"oracle rejected the basis (code {rc})")
    prims, o = [], 0
    for f in range(nbf):
        prims.append((al[o:o + npr[f]].copy(), w[o:o + npr[f]].copy()))
        o += npr[f]
    return atom, pw, prims


def prim_norm(alpha: float, a: int, b: int, c: int) -> float:
    return float(_load().scff_oracle_prim_norm(alpha, a, b, c))


def grid_form_factor(job, flat_idx: Optional[np.ndarray] = None, scale: float = 1.0,
                     threads: int = 0, terms: bool = False):
    """Oracle on a product grid job, on all points or on the given flat indices."""
    if flat_idx is None:
        flat_idx = np.arange(job.nq)
    q = job.q_points(flat_idx)
    return form_factor(job.mol, job.T, q, scale=scale, threads=threads, terms=terms)
