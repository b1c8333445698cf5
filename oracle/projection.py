"""FP64 restatement of the divergence-free projection of a periodic velocity field (the
surrogate's velocity hand-over to the lattice).

TEST INFRASTRUCTURE, like the rest of this package: only the test suite and the benchmark's
CPU legs use it. The paper has no surrogate. It states (Sec. 2.1, with the pressure evolution
equation) that at low Mach number the velocity field is approximately divergence-free; a
predicted velocity that is not makes the restarted lattice relax it away through pressure
waves. The library therefore replaces a predicted velocity by its divergence-free part.

Definition. On a grid periodic in x, y and z, with the central difference
    (D_a q)(x) = (q(x + e_a) - q(x - e_a)) / 2
along axis a and the divergence div u = D_x u + D_y v + D_z w, the projection P u is the field
closest to u in the sum of squares over all cells and components whose divergence is zero
(the orthogonal projection onto the kernel of div). It is unique, linear, idempotent and
symmetric, and u - P u is a discrete gradient D q.

Evaluation. The discrete Fourier transform diagonalises D_a: for a mode of wavenumbers k_a
(0 <= k_a < n_a) it multiplies by i s_a with s_a = sin(2 pi k_a / n_a). Per mode the projection is
    U <- U - s (s . U) / |s|^2      (|s| > 0; modes with s = 0 carry no divergence and are kept),
and the transform is unitary up to a constant, so the per-mode projections compose to the
orthogonal one. numpy's FFT serves as that step.
"""
from __future__ import annotations

import numpy as np


def divergence(u):
    """Central-difference divergence of a periodic u [3][nz][ny][nx] (components x, y, z)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros(u.shape[1:])
    for a, axis in ((0, 2), (1, 1), (2, 0)):
        out += 0.5 * (np.roll(u[a], -1, axis) - np.roll(u[a], 1, axis))
    return out


def gradient(q):
    """Central-difference gradient (D_x q, D_y q, D_z q) of a periodic scalar q [nz][ny][nx]."""
    q = np.asarray(q, dtype=np.float64)
    return np.stack([0.5 * (np.roll(q, -1, axis) - np.roll(q, 1, axis)) for axis in (2, 1, 0)])


def _sines(n):
    """sin(2 pi k / n) for k = 0 .. n - 1, exactly 0 where 2 k / n is an integer (k = 0 and, for
    even n, k = n / 2), where the floating-point sine of pi is not."""
    k = np.arange(n)
    return np.where((2 * k) % n == 0, 0.0, np.sin(2.0 * np.pi * k / n))


def project_solenoidal(u):
    """P u for a periodic u [3][nz][ny][nx] (see the module docstring), FP64."""
    u = np.asarray(u, dtype=np.float64)
    nz, ny, nx = u.shape[1:]
    sz = _sines(nz)[:, None, None]
    sy = _sines(ny)[None, :, None]
    sx = _sines(nx)[None, None, :]
    s = [np.broadcast_to(v, (nz, ny, nx)) for v in (sx, sy, sz)]
    U = [np.fft.fftn(u[a]) for a in range(3)]
    s2 = s[0] ** 2 + s[1] ** 2 + s[2] ** 2
    dot = s[0] * U[0] + s[1] * U[1] + s[2] * U[2]
    q = np.where(s2 > 0, dot / np.where(s2 > 0, s2, 1.0), 0.0)
    return np.stack([np.fft.ifftn(U[a] - s[a] * q).real for a in range(3)])
