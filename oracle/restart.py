"""FP64 restatement of the restart from coarse fields (the surrogate's hand-over to the lattice).

TEST INFRASTRUCTURE, like the rest of this package: only the test suite and the benchmark's
CPU legs use it. The paper has no such step (it advances every step with the LBM); the restart
is the library's own interface, and this module states what it computes:

1. upsampling. Each of the five coarse fields (phi, u, v, w, p on a grid of nc = n / f cells
   per axis) is interpolated trilinearly between coarse cell centres. Fine cell i (centre at
   i + 1/2 in fine units) sits at coarse coordinate (i + 1/2) / f - 1/2, where coarse cell k has
   its centre at coordinate k. Along a periodic axis the coarse indices wrap; along a walled
   axis the coordinate is clamped to [0, nc - 1] (the end centres);
2. phi is clamped to [-1, 1.5], the range the lattice accepts for its fixed-point phi;
3. the populations are the initial state of reading R9 built from the upsampled fields:
   f* = f^eq(p, u, rho(phi), Pi_s(grad phi)) (Eq. geq_s) and
   g* = g^eq(phi, u, S) - t_i (tau_phi - 1/2) e_i . grad phi (Eq. geq), with grad phi the
   isotropic central difference of the upsampled phi (mirror images across walls);
4. sum phi over the grid is set back to its value before the restart by adding the
   difference, spread evenly over the cells, to every cell's phi (the rest population g_0).

Trilinear interpolation is the composition of three one-dimensional linear interpolations, one
per axis, which is how it is evaluated here.
"""
from __future__ import annotations

import numpy as np


def _linear_along(field, axis, factor, walled):
    """One-dimensional linear interpolation of `field` along `axis` onto factor times as many
    points, at the fine cell centres described in the module docstring."""
    nc = field.shape[axis]
    n = nc * factor
    xc = (np.arange(n) + 0.5) / factor - 0.5
    if walled:
        xc = np.clip(xc, 0.0, nc - 1.0)
        a = np.minimum(np.floor(xc).astype(np.int64), nc - 1)
        b = np.minimum(a + 1, nc - 1)
    else:
        a = np.floor(xc).astype(np.int64)
        b = a + 1
    t = xc - a
    a %= nc
    b %= nc
    fa = np.take(field, a, axis=axis)
    fb = np.take(field, b, axis=axis)
    shape = [1] * field.ndim
    shape[axis] = n
    t = t.reshape(shape)
    return (1.0 - t) * fa + t * fb


def upsample_trilinear(coarse, factor, walls=0):
    """Fine field [nz f][ny f][nx f] from a coarse scalar field [nz][ny][nx]. walls: bit 0 x,
    bit 1 y, bit 2 z. factor 1 returns the field unchanged."""
    out = np.asarray(coarse, dtype=np.float64)
    for axis, bit in ((2, 1), (1, 2), (0, 4)):
        out = _linear_along(out, axis, factor, bool(walls & bit))
    return out


def upsample_fields(coarse, factor, walls=0):
    """phi (clamped to [-1, 1.5]), u (3 planes) and p from coarse [5][nz][ny][nx]."""
    coarse = np.asarray(coarse, dtype=np.float64)
    up = [upsample_trilinear(coarse[k], factor, walls) for k in range(5)]
    phi = np.clip(up[0], -1.0, 1.5)
    return phi, np.stack(up[1:4]), up[4]


def restart_from_coarse(ref, coarse, factor, p0):
    """Steps 1-4 on the oracle `ref` (an ``oracle.Oracle``): its state is replaced."""
    nx, ny, nz = ref.grid
    if nx % factor or ny % factor or nz % factor:
        raise ValueError("factor must divide nx, ny and nz")
    coarse = np.asarray(coarse, dtype=np.float64).reshape(5, nz // factor, ny // factor, nx // factor)
    mass_before = ref.get_pops()[1].sum()
    phi, u, p = upsample_fields(coarse, factor, ref.walls)
    ref.init_phi(phi, u, p0=p0, p=p)
    f, g = ref.get_pops()
    g[0] += (mass_before - g.sum()) / ref.N
    ref.set_pops(f, g)
