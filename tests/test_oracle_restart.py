"""Pins of the oracle's restart from coarse fields (oracle/restart.py), run without a GPU.

* upsampling equals scipy's first-order map_coordinates at the fine cell centres (periodic:
  grid-wrap; walled: nearest, i.e. clamped to the end centres), and is exact on trilinear
  polynomials in the coarse coordinates;
* restarting from block means of smooth fields reproduces the initial state of those fields
  (reading R9) to second order in the coarse spacing: a half-cell offset, swapped velocity
  components or a wrong pressure would leave first-order or no convergence;
* sum phi is set back exactly, and phi is clamped to [-1, 1.5];
* with factor 1 the restart is the initial state of the coarse fields themselves.
"""
import numpy as np
import pytest

import oracle as O
from oracle import restart as R

PARAMS = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3, rho_ratio=3.0, mu_ratio=2.0)


def _block_mean(a, f):
    nz, ny, nx = a.shape
    return a.reshape(nz // f, f, ny // f, f, nx // f, f).mean(axis=(1, 3, 5))


@pytest.mark.parametrize("factor", [1, 2, 3, 4])
@pytest.mark.parametrize("walls,mode", [(0, "grid-wrap"), (7, "nearest")])
def test_upsampling_is_linear_map_coordinates(factor, walls, mode):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(factor + walls)
    c = rng.standard_normal((3, 4, 5))
    up = R.upsample_trilinear(c, factor, walls)
    n = np.array(c.shape) * factor
    coords = np.meshgrid(*[(np.arange(k) + 0.5) / factor - 0.5 for k in n], indexing="ij")
    want = ndimage.map_coordinates(c, coords, order=1, mode=mode)
    np.testing.assert_allclose(up, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("walls", [0, 1, 2, 4, 7])
def test_upsampling_is_exact_on_trilinear_polynomials(walls):
    """P = a + bX + cY + dZ + eXY + gYZ + hXZ + kXYZ sampled at coarse centres (X the coarse x
    index): every fine cell whose coarse coordinates lie inside [0, nc - 1] on each axis gets P
    at those coordinates. Distinct coefficients catch swapped axes; the interior test catches a
    centre offset."""
    f = 4
    nc = (4, 5, 6)  # z, y, x
    Z, Y, X = np.meshgrid(*[np.arange(k, dtype=float) for k in nc], indexing="ij")
    P = lambda X, Y, Z: 0.3 + 1.1 * X - 0.7 * Y + 0.45 * Z + 0.2 * X * Y - 0.15 * Y * Z + 0.05 * X * Z + 0.01 * X * Y * Z  # noqa
    up = R.upsample_trilinear(P(X, Y, Z), f, walls)
    zf, yf, xf = np.meshgrid(*[(np.arange(k * f) + 0.5) / f - 0.5 for k in nc], indexing="ij")
    inside = (xf >= 0) & (xf <= nc[2] - 1) & (yf >= 0) & (yf <= nc[1] - 1) & (zf >= 0) & (zf <= nc[0] - 1)
    np.testing.assert_allclose(up[inside], P(xf, yf, zf)[inside], rtol=0, atol=1e-12)
    assert inside.mean() > 0.4


def _smooth_fields(n):
    z, y, x = np.meshgrid(*[np.arange(n) + 0.5] * 3, indexing="ij")
    k = 2 * np.pi / n
    phi = 0.5 + 0.3 * np.sin(k * x) * np.cos(k * y) + 0.1 * np.sin(k * z + 0.3)
    u = np.stack([0.02 * np.cos(k * y) * np.sin(k * z), 0.015 * np.sin(k * x + 0.5),
                  -0.01 * np.cos(k * x) * np.cos(k * y)])
    p = 1.0 / 3.0 + 1e-3 * np.cos(k * x + k * z)
    return phi, u, p


def test_restart_from_block_means_converges_at_second_order():
    n = 32
    phi, u, p = _smooth_fields(n)
    exact = O.Oracle(19, (n, n, n), **PARAMS)
    exact.init_phi(phi, u, p=p)
    fe, ge = exact.get_pops()
    errs = {}
    for f in (2, 4):
        coarse = np.stack([_block_mean(phi, f)] + [_block_mean(u[a], f) for a in range(3)] + [_block_mean(p, f)])
        o = O.Oracle(19, (n, n, n), **PARAMS)
        o.init_phi(phi, u, p=p)
        o.restart_from_coarse(coarse, f)
        fr, gr = o.get_pops()
        errs[f] = (np.abs(fr - fe).max(), np.abs(gr - ge).max(), np.abs(gr.sum(0) - ge.sum(0)).max())
    for a, b in zip(errs[4], errs[2]):
        assert 3.2 < a / b < 5.5, errs
    assert errs[2][2] < 0.02


@pytest.mark.parametrize("walls", [0, 7])
def test_restart_holds_sum_phi_and_clamps_phi(walls):
    n, f = 16, 2
    phi0 = np.full((n, n, n), 0.5)
    o = O.Oracle(19, (n, n, n), walls=walls, **PARAMS)
    o.init_phi(phi0)
    before = o.get_pops()[1].sum()
    rng = np.random.default_rng(4)
    coarse = np.zeros((5, n // f, n // f, n // f))
    coarse[0] = rng.uniform(0.0, 1.0, coarse[0].shape)
    coarse[0, 2, 3, 4] = 4.0     # upsampled values above 1.5 near this centre
    coarse[0, 5, 5, 5] = -5.0    # and below -1 near this one
    coarse[1:4] = rng.normal(0.0, 0.01, coarse[1:4].shape)
    coarse[4] = 1.0 / 3.0
    o.restart_from_coarse(coarse, f)
    g = o.get_pops()[1]
    assert abs(g.sum() - before) <= 1e-12 * abs(before)
    phi_up, _, _ = R.upsample_fields(coarse, f, walls)
    assert phi_up.max() == 1.5 and phi_up.min() == -1.0
    shift = (before - np.clip(R.upsample_trilinear(coarse[0], f, walls), -1.0, 1.5).sum()) / o.N
    np.testing.assert_allclose(g.sum(0), phi_up + shift, rtol=0, atol=1e-13)


def test_restart_with_factor_one_is_the_initial_state():
    grid = (9, 7, 5)
    rng = np.random.default_rng(8)
    shape = grid[::-1]
    coarse = np.stack([rng.uniform(0.0, 1.0, shape), *rng.normal(0.0, 0.01, (3,) + shape),
                       1.0 / 3.0 + rng.normal(0.0, 1e-3, shape)])
    o = O.Oracle(19, grid, walls=2, **PARAMS)
    o.init_phi(np.full(shape, 0.25))
    before = o.get_pops()[1].sum()
    o.restart_from_coarse(coarse, 1)
    fr, gr = o.get_pops()
    ref = O.Oracle(19, grid, walls=2, **PARAMS)
    ref.init_phi(coarse[0], coarse[1:4], p=coarse[4])
    fe, ge = ref.get_pops()
    np.testing.assert_allclose(fr, fe, rtol=0, atol=1e-15)
    ge[0] += (before - ge.sum()) / o.N
    np.testing.assert_allclose(gr, ge, rtol=0, atol=1e-15)
