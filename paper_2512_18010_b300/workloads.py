"""Seeded synthetic workloads: molecules, Gaussian basis definitions, transition
density matrices and q-grids.

This module only draws inputs.  It holds none of the form-factor arithmetic
(no normalisation, no integrals): both the CUDA path and the FP64 oracle read
what it produces and do all of the method's work themselves.

The workloads stand in for the paper's 100-molecule cc-pVDZ TD-DFT test set
(Sec. "Molecular Form Factors", Fig. of the molecule set), which is not
available: molecules are built from seeded random geometries and
double-zeta-shaped basis sets, and each transition density matrix is a seeded
T = U diag(exp(-k/4)) V^T with orthogonal U, V.

Conventions
-----------
* Lengths in Bohr, momenta in inverse Bohr.
* ``shell_l``: 0 = s, 1 = p, 2 = Cartesian d, -1 = sp (one exponent set shared
  by an s function and three p functions).
* ``exponents``: alpha of exp(-alpha r^2), concatenated over shells.
* ``coefficients``: raw contraction coefficients, concatenated over shells; an
  sp shell stores its s coefficients and then its p coefficients.  They are
  N(0,1) draws; the consumer normalises each contracted function.
* ``T[s, mu, nu]`` weights phi_mu phi_nu; functions are ordered shell by shell,
  Cartesian components in the order x,y,z / xx,xy,xz,yy,yz,zz, and an sp shell
  gives s,px,py,pz.
* Product q-grids are inclusive and antisymmetric: q_k = (2k-(N-1)) a/(N-1), so
  index k and N-1-k hold exactly opposite values.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

# Cartesian function count per shell code (bookkeeping only).
NFN = {0: 1, 1: 3, 2: 6, 3: 10, -1: 4}
# Basis flag bits for pure (spherical-harmonic) d and f shells: 2l+1 functions.
PURE_D, PURE_F = 2, 4
_PURE_BIT = {2: PURE_D, 3: PURE_F}


@dataclasses.dataclass
class Molecule:
    name: str
    xyz: np.ndarray            # [n_atoms, 3] float64, Bohr
    shell_atom: np.ndarray     # [n_shells] int32
    shell_l: np.ndarray        # [n_shells] int32
    shell_nprim: np.ndarray    # [n_shells] int32
    exponents: np.ndarray      # [sum nprim] float64
    coefficients: np.ndarray   # [sum nprim * (2 if sp else 1)] float64
    heavy: int = 0
    pure: int = 0              # PURE_D | PURE_F: those shells are spherical-harmonic

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_shells(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nbf(self) -> int:
        n = 0
        for l in self.shell_l:
            l = int(l)
            n += 2 * l + 1 if (self.pure & _PURE_BIT.get(l, 0)) else NFN[l]
        return n

    def translated(self, a) -> "Molecule":
        m = dataclasses.replace(self)
        m.xyz = self.xyz + np.asarray(a, dtype=np.float64)[None, :]
        return m


@dataclasses.dataclass
class Job:
    """One form-factor job: a molecule, its transitions and a product grid."""
    mol: Molecule
    T: np.ndarray              # [S, nbf, nbf] float64
    qx: np.ndarray
    qy: np.ndarray
    qz: np.ndarray
    seed: int = 0

    @property
    def n_states(self) -> int:
        return int(self.T.shape[0])

    @property
    def nq(self) -> int:
        return len(self.qx) * len(self.qy) * len(self.qz)

    def q_points(self, flat_idx: np.ndarray) -> np.ndarray:
        """Explicit q vectors [n,3] of flat grid indices (z fastest)."""
        flat_idx = np.asarray(flat_idx, dtype=np.int64)
        ny, nz = len(self.qy), len(self.qz)
        ix = flat_idx // (ny * nz)
        iy = (flat_idx // nz) % ny
        iz = flat_idx % nz
        return np.stack([self.qx[ix], self.qy[iy], self.qz[iz]], axis=1)


# --------------------------------------------------------------------------
# basic draws
# --------------------------------------------------------------------------

def log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def axis(n: int, a: float) -> np.ndarray:
    """Inclusive antisymmetric axis on [-a, a] with n points."""
    if n == 1:
        return np.zeros(1)
    k = np.arange(n, dtype=np.float64)
    return (2.0 * k - (n - 1)) * a / (n - 1)


def random_rotation(rng) -> np.ndarray:
    m = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(m)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def random_orthogonal(rng, n: int) -> np.ndarray:
    m = rng.standard_normal((n, n))
    q, r = np.linalg.qr(m)
    return q * np.sign(np.diag(r))[None, :]


def transition_matrices(seed: int, n_states: int, nbf: int) -> np.ndarray:
    """T^s = U_s diag(exp(-k/4)) V_s^T with seeded orthogonal U_s, V_s."""
    T = np.empty((n_states, nbf, nbf))
    d = np.exp(-np.arange(nbf) / 4.0)
    for s in range(n_states):
        rng = np.random.default_rng(seed * 100 + s)
        U = random_orthogonal(rng, nbf)
        V = random_orthogonal(rng, nbf)
        T[s] = (U * d[None, :]) @ V.T
    return T


def valence_transitions(mol: Molecule, T: np.ndarray, exponent_cut: float = 50.0) -> np.ndarray:
    """T with the rows and columns of core functions set to zero: functions of shells whose largest
    primitive exponent exceeds ``exponent_cut`` (the heavy atoms' tight s shells).  Transition
    densities of valence excitations carry next to no core weight; this is the input on which a
    real-space grid (the FFT method) can resolve the density."""
    keep = []
    off = 0
    for sh in range(mol.n_shells):
        l, npr = int(mol.shell_l[sh]), int(mol.shell_nprim[sh])
        amax = float(np.max(mol.exponents[off:off + npr]))
        off += npr
        nf = 2 * l + 1 if (mol.pure & _PURE_BIT.get(l, 0)) else NFN[l]
        keep += [amax <= exponent_cut] * nf
    keep = np.asarray(keep)
    Tv = np.array(T, dtype=np.float64, copy=True)
    Tv[:, ~keep, :] = 0.0
    Tv[:, :, ~keep] = 0.0
    return Tv


def subset_indices(n_total: int, n: int, seed: int) -> np.ndarray:
    """Seeded uniform sample of flat grid indices, sorted, without repeats."""
    rng = np.random.default_rng(seed)
    n = min(n, n_total)
    return np.sort(rng.choice(n_total, size=n, replace=False)).astype(np.int64)


# --------------------------------------------------------------------------
# basis assembly
# --------------------------------------------------------------------------

class _ShellList:
    def __init__(self):
        self.atom, self.l, self.nprim, self.exps, self.coefs = [], [], [], [], []

    def add(self, atom, l, exps, rng):
        exps = np.asarray(exps, dtype=np.float64)
        n = len(exps)
        self.atom.append(atom)
        self.l.append(l)
        self.nprim.append(n)
        self.exps.append(exps)
        ncoef = 2 * n if l == -1 else n
        self.coefs.append(rng.standard_normal(ncoef))

    def molecule(self, name, xyz, heavy, pure: int = 0) -> Molecule:
        return Molecule(
            name=name,
            xyz=np.ascontiguousarray(xyz, dtype=np.float64),
            shell_atom=np.asarray(self.atom, dtype=np.int32),
            shell_l=np.asarray(self.l, dtype=np.int32),
            shell_nprim=np.asarray(self.nprim, dtype=np.int32),
            exponents=np.concatenate(self.exps),
            coefficients=np.concatenate(self.coefs),
            heavy=heavy,
            pure=pure,
        )


def _double_zeta_heavy(sh: _ShellList, atom: int, rng, with_d: bool):
    sh.add(atom, 0, log_uniform(rng, 0.2, 3000.0, 6), rng)   # core s, 6 primitives
    sh.add(atom, -1, log_uniform(rng, 0.3, 30.0, 3), rng)    # inner sp, 3 primitives
    sh.add(atom, -1, log_uniform(rng, 0.08, 0.3, 1), rng)    # outer sp, 1 primitive
    if with_d:
        sh.add(atom, 2, [0.8], rng)                          # Cartesian d polarisation


def _double_zeta_h(sh: _ShellList, atom: int, rng):
    sh.add(atom, 0, log_uniform(rng, 0.15, 35.0, 3), rng)
    sh.add(atom, 0, log_uniform(rng, 0.08, 0.3, 1), rng)


def _unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def grow_geometry(rng, n_heavy: int, n_h: int, dmin=2.0, dhh=(2.6, 3.0), dh=2.05):
    """Random connected heavy-atom skeleton plus one H per heavy atom (cyclic).

    Each new heavy atom sits 2.6-3.0 Bohr from a random existing heavy atom;
    each H sits 2.05 Bohr from its heavy atom.  Any placement closer than
    ``dmin`` to an existing atom is redrawn.
    """
    heavy = [np.zeros(3)]
    tries = 0
    while len(heavy) < n_heavy:
        tries += 1
        if tries > 200000:
            raise RuntimeError("geometry growth failed")
        base = heavy[rng.integers(len(heavy))]
        cand = base + rng.uniform(*dhh) * _unit(rng)
        if min(np.linalg.norm(cand - h) for h in heavy) >= dmin:
            heavy.append(cand)
    atoms = list(heavy)
    hyd = []
    for i in range(n_h):
        host = heavy[i % n_heavy]
        for _ in range(100000):
            cand = host + dh * _unit(rng)
            if min(np.linalg.norm(cand - a) for a in atoms) >= dmin:
                break
        else:
            raise RuntimeError("hydrogen placement failed")
        atoms.append(cand)
        hyd.append(cand)
    return np.array(heavy), np.array(hyd) if hyd else np.zeros((0, 3))


# --------------------------------------------------------------------------
# the five workload shapes
# --------------------------------------------------------------------------

def config1(seed: int = 1000) -> Job:
    """Tiny: 1 heavy + 2 H; heavy s,s,p,d and H s, 3 primitives each (13 functions)."""
    rng = np.random.default_rng(seed)
    heavy = np.zeros((1, 3))
    hs = []
    while len(hs) < 2:
        c = rng.uniform(1.8, 2.2) * _unit(rng)
        if all(np.linalg.norm(c - h) >= 1.8 for h in hs):
            hs.append(c)
    xyz = np.vstack([heavy, np.array(hs)])
    sh = _ShellList()
    for l in (0, 0, 1, 2):
        sh.add(0, l, log_uniform(rng, 0.1, 50.0, 3), rng)
    for a in (1, 2):
        sh.add(a, 0, log_uniform(rng, 0.1, 50.0, 3), rng)
    mol = sh.molecule("cfg1-tiny", xyz, heavy=1)
    T = transition_matrices(seed, 1, mol.nbf)
    ax = axis(16, 10.0)
    return Job(mol, T, ax, ax.copy(), ax.copy(), seed)


def config2(seed: int = 2000) -> Job:
    """Benzene-scale ring: 6 heavy (9 functions each) + 6 H (2 each) = 66 functions."""
    rng = np.random.default_rng(seed)
    ang = np.arange(6) * (np.pi / 3.0)
    ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(6)], axis=1)
    heavy = 2.6 * ring
    hyd = (2.6 + 2.05) * ring
    R = random_rotation(rng)
    xyz = np.vstack([heavy, hyd]) @ R.T
    sh = _ShellList()
    for a in range(6):
        _double_zeta_heavy(sh, a, rng, with_d=False)
    for a in range(6, 12):
        _double_zeta_h(sh, a, rng)
    mol = sh.molecule("cfg2-benzene-ring", xyz, heavy=6)
    T = transition_matrices(seed, 12, mol.nbf)
    ax = axis(64, 15.0)
    return Job(mol, T, ax, ax.copy(), ax.copy(), seed)


def molecule_dz_d(seed: int, n_heavy: int, n_h: Optional[int] = None) -> Molecule:
    """Random connected molecule with the double-zeta + d basis (15 + 2 functions per heavy/H pair)."""
    rng = np.random.default_rng(seed)
    if n_h is None:
        n_h = n_heavy
    heavy, hyd = grow_geometry(rng, n_heavy, n_h)
    xyz = np.vstack([heavy, hyd]) if len(hyd) else heavy
    sh = _ShellList()
    for a in range(n_heavy):
        _double_zeta_heavy(sh, a, rng, with_d=True)
    for a in range(n_heavy, n_heavy + n_h):
        _double_zeta_h(sh, a, rng)
    return sh.molecule(f"dz-d-{n_heavy}h-{seed}", xyz, heavy=n_heavy)


def molecule_pol_f(seed: int, n_heavy: int, n_h: Optional[int] = None, pure: int = 0) -> Molecule:
    """Random connected molecule with double-zeta + d + f on heavy atoms and p on H.

    Heavy atoms carry core s, two sp shells, one Cartesian d (2 primitives) and
    one Cartesian f (1 primitive): 25 functions; each H carries two s shells
    and a p polarisation shell: 5 functions.
    """
    rng = np.random.default_rng(seed)
    if n_h is None:
        n_h = n_heavy
    heavy, hyd = grow_geometry(rng, n_heavy, n_h)
    xyz = np.vstack([heavy, hyd]) if len(hyd) else heavy
    sh = _ShellList()
    for a in range(n_heavy):
        sh.add(a, 0, log_uniform(rng, 0.2, 3000.0, 6), rng)
        sh.add(a, -1, log_uniform(rng, 0.3, 30.0, 3), rng)
        sh.add(a, -1, log_uniform(rng, 0.08, 0.3, 1), rng)
        sh.add(a, 2, log_uniform(rng, 0.4, 2.5, 2), rng)
        sh.add(a, 3, log_uniform(rng, 0.5, 1.5, 1), rng)
    for a in range(n_heavy, n_heavy + n_h):
        _double_zeta_h(sh, a, rng)
        sh.add(a, 1, log_uniform(rng, 0.5, 1.2, 1), rng)
    return sh.molecule(f"pol-f-{n_heavy}h-{seed}" + ("-pure" if pure else ""), xyz, heavy=n_heavy, pure=pure)


def config_f(seed: int = 3500, n_heavy: int = 4, n_states: int = 6, n: int = 48, pure: int = 0) -> Job:
    """f-shell workload: 4 heavy + 4 H with d and f polarisation, 48^3 on [-15,15].

    120 Cartesian functions; with pure = PURE_D | PURE_F the d and f shells
    are spherical-harmonic (5 and 7 functions) and the basis has 104.
    """
    mol = molecule_pol_f(seed, n_heavy, pure=pure)
    T = transition_matrices(seed, n_states, mol.nbf)
    ax = axis(n, 15.0)
    return Job(mol, T, ax, ax.copy(), ax.copy(), seed)


def config3(seed: int = 3000, n: int = 128) -> Job:
    """10 heavy + 10 H, double-zeta + d (170 functions), 12 states, 128^3 on [-20,20]."""
    mol = molecule_dz_d(seed, 10)
    T = transition_matrices(seed, 12, mol.nbf)
    ax = axis(n, 20.0)
    return Job(mol, T, ax, ax.copy(), ax.copy(), seed)


def config4_job(i: int) -> Job:
    """Molecule i of the 256-molecule batch: 5-30 heavy (+ equal H), 4-24 states, 48^3-96^3."""
    seed = 4000 + i
    rng = np.random.default_rng(seed * 7 + 1)
    n_heavy = int(rng.integers(5, 31))
    n_states = int(rng.integers(4, 25))
    n = int(rng.integers(48, 97))
    mol = molecule_dz_d(seed, n_heavy)
    T = transition_matrices(seed, n_states, mol.nbf)
    ax = axis(n, 20.0)
    return Job(mol, T, ax, ax.copy(), ax.copy(), seed)


def config4(n_mol: int = 256) -> List[Job]:
    return [config4_job(i) for i in range(n_mol)]


def config5_large(seed: int = 5999) -> Job:
    """The serving stream's large job: 40 heavy + 40 H (680 functions), 32 states, 128^3."""
    mol = molecule_dz_d(seed, 40)
    T = transition_matrices(seed, 32, mol.nbf)
    ax = axis(128, 20.0)
    return Job(mol, T, ax, ax.copy(), ax.copy(), seed)


def config5_job(i: int) -> Job:
    """Job i of the serving stream: the config-4 distribution plus 5% large jobs."""
    rng = np.random.default_rng(5000 + i)
    if rng.uniform() < 0.05:
        return config5_large(5000 + 100000 + i)
    return config4_job(1000 + i)


def config5_large_positions(n: int, frac: float = 0.05, seed: int = 5050) -> np.ndarray:
    """Indices of the large jobs in a serving stream of n jobs: exactly round(frac * n) of them,
    at seeded positions."""
    k = int(round(frac * n))
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False)) if k else np.zeros(0, int)


def config5_stream_job(i: int, n: int) -> Job:
    """Job i of a serving stream of n jobs: the config-4 size distribution, with exactly 5% of the
    positions (seeded) taken by the large job shape (40 heavy + 40 H, 680 functions, 32 states, 128^3)."""
    if i in set(config5_large_positions(n).tolist()):
        return config5_large(5000 + 100000 + i)
    return config4_job(1000 + i)


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 5555) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def scaled_job(job: Job, n_axis: int) -> Job:
    """Same molecule and states on a coarser or finer n_axis^3 grid of the same extent."""
    a = float(job.qx[-1])
    ax = axis(n_axis, a)
    return Job(job.mol, job.T, ax, ax.copy(), ax.copy(), job.seed)


CONFIGS = {1: config1, 2: config2, 3: config3}
