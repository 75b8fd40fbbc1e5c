"""FFT method of the form factor -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product path never does.

What it computes (Sec. "The (Fast) Fourier Transform", Eqs. Falbega,
continuFFT, fftABC, qabc; Sec. "Fast Fourier Transform Method" for the
grid): the transition density Phi_s(r) = sum T^s phi phi is tabulated on a
box of n points per axis, side L = 2 pi / dq, centred at `centre`,

    x_a = centre - L/2 + a L/n,   a = 0 .. n-1,

and the form factor is its discrete Fourier sum at q = dq (alpha - n/2),
alpha = 0 .. n-1 (ascending, the most negative frequency first):

    f_s(q) = V_pix sum_a Phi_s(x_a) e^{+i q.x_a},   V_pix = (L/n)^3 (per-axis product).

With q.x_a = q.x_min + 2 pi alpha.a / n this is V_pix e^{i q.x_min} times the
positive-exponent DFT of the samples, which numpy's ifftn (times n^3)
computes; the density itself comes from the FP64 C oracle.

Parity status: pinned in tests/test_oracle_fft.py (the direct Fourier sum,
the analytic transform of an s Gaussian, convergence to the exact Cartesian
oracle, discrete Parseval).
"""
from __future__ import annotations

import numpy as np

from . import density


def axes(n, dq, centre):
    """Per axis: real-space points x[a] and the q points of the result."""
    out = []
    for ax in range(3):
        L = 2.0 * np.pi / dq[ax]
        x = centre[ax] - L / 2 + (L / n[ax]) * np.arange(n[ax])
        q = dq[ax] * (np.arange(n[ax]) - n[ax] // 2)
        out.append((x, q))
    return out


def tabulate(mol, T, n, dq, centre, scale=1.0, threads=0):
    """Phi[s, a, b, c] on the box and the per-axis coordinates."""
    ax = axes(n, dq, centre)
    X, Y, Z = np.meshgrid(ax[0][0], ax[1][0], ax[2][0], indexing="ij")
    r = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    phi = density(mol, T, r, scale=scale, threads=threads)
    return phi.reshape((phi.shape[0],) + tuple(n)), ax


def form_factor(mol, T, n, dq, centre, scale=1.0, threads=0):
    """f[s, ix, iy, iz] at q = dq (index - n/2) per axis, and the density Phi."""
    phi, ax = tabulate(mol, T, n, dq, centre, scale=scale, threads=threads)
    N = int(np.prod(n))
    vpix = np.prod([(2.0 * np.pi / dq[i]) / n[i] for i in range(3)])
    G = np.fft.ifftn(phi, axes=(1, 2, 3)) * N          # sum_a Phi_a e^{+2 pi i alpha.a/n}
    f = np.empty_like(G)
    idx = [np.mod(np.arange(n[i]) - n[i] // 2, n[i]) for i in range(3)]
    f[:] = G[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
    xmin = [ax[i][0][0] for i in range(3)]
    qx, qy, qz = np.meshgrid(ax[0][1], ax[1][1], ax[2][1], indexing="ij")
    f *= vpix * np.exp(1j * (qx * xmin[0] + qy * xmin[1] + qz * xmin[2]))[None]
    return f, phi


def direct_sum(phi, n, dq, centre, q):
    """V_pix sum_a Phi(x_a) e^{i q.x_a} at explicit q[k, 3] (the definition)."""
    ax = axes(n, dq, centre)
    vpix = np.prod([(2.0 * np.pi / dq[i]) / n[i] for i in range(3)])
    X, Y, Z = np.meshgrid(ax[0][0], ax[1][0], ax[2][0], indexing="ij")
    out = np.zeros((phi.shape[0], len(q)), dtype=np.complex128)
    for k, qv in enumerate(np.asarray(q, float)):
        ph = np.exp(1j * (qv[0] * X + qv[1] * Y + qv[2] * Z))
        out[:, k] = vpix * np.einsum("sabc,abc->s", phi, ph)
    return out


def parseval(phi, f, n, dq):
    """(sum |Phi|^2 V_pix, sum |f|^2 dq^3 / (2 pi)^3) per state."""
    vpix = np.prod([(2.0 * np.pi / dq[i]) / n[i] for i in range(3)])
    dq3 = float(np.prod(dq))
    a = np.sum(np.abs(phi) ** 2, axis=(1, 2, 3)) * vpix
    b = np.sum(np.abs(f) ** 2, axis=(1, 2, 3)) * dq3 / (2.0 * np.pi) ** 3
    return a, b
