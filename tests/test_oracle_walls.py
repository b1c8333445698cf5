"""Pins of the oracle's walls (no GPU): half-way bounce-back in the Lax-Wendroff stencil.

* a pressure-driven channel (Poiseuille) between walls has u(y) = G/(2 nu) y (H - y) with the
  walls half-way outside the first and last cells (nu = cs^2 tau_rho, Eq. c-n_m, Eq. body);
* gravity against a wall gives a hydrostatic pressure p' = rho G and no flow (Eq. pressure);
* sum phi is conserved to round-off in boxes with walls (the wall-face fluxes cancel);
* a uniform state at rest is a fixed point with walls on every side.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import inputs as I


@pytest.mark.parametrize("c,tau,tol", [(1.0, 0.8, 0.004), (1.0, 0.3, 0.002), (0.997, 0.8, 0.012)])
def test_poiseuille_profile(c, tau, tol):
    ny, G = 32, 1e-6
    o = O.Oracle(9, (3, ny, 1), tau, 0.8, 0.02, 4.0, 0.0, body_force=(G, 0, 0), courant=c, walls=2)
    o.init_phi(np.ones((1, ny, 3)))
    nu = tau / 3.0
    o.step(int(3 * ny * ny / nu))
    ux = o.moments()[2][0, 0, :, 1]
    y = np.arange(ny) + 0.5
    ana = G / (2 * nu) * y * (ny - y)
    assert np.abs(ux - ana).max() / ana.max() < tol


def test_poiseuille_3d_between_z_walls():
    nz, G, tau = 24, 1e-6, 0.8
    o = O.Oracle(19, (3, 3, nz), tau, 0.8, 0.02, 4.0, 0.0, body_force=(0, G, 0), courant=1.0, walls=4)
    o.init_phi(np.ones((nz, 3, 3)))
    nu = tau / 3.0
    o.step(int(3 * nz * nz / nu))
    uy = o.moments()[2][1, :, 1, 1]
    z = np.arange(nz) + 0.5
    ana = G / (2 * nu) * z * (nz - z)
    assert np.abs(uy - ana).max() / ana.max() < 0.006   # uniform slip of half-way bounce-back under BGK


def test_hydrostatic_balance():
    ny, G = 32, -1e-5
    o = O.Oracle(9, (3, ny, 1), 0.8, 0.8, 0.02, 4.0, 0.0, body_force=(0, G, 0), walls=2)
    o.init_phi(np.ones((1, ny, 3)))
    o.step(4000)
    phi, p, u = o.moments()
    slope = np.polyfit(np.arange(2, ny - 2), p[0, 2:-2, 1], 1)[0]
    assert slope == pytest.approx(G, rel=0.01)
    assert np.abs(u).max() < 1e-7


@pytest.mark.parametrize("Q,grid,walls", [(19, (14, 13, 12), 4), (19, (12, 11, 10), 7), (9, (20, 18, 1), 3)])
def test_phi_conserved_with_walls(Q, grid, walls):
    G = (0.0, 0.0, -2e-5) if Q == 19 else (1e-5, -2e-5, 0.0)
    o = O.Oracle(Q, grid, 0.8, 0.8, 0.02, 4.0, 1e-3, rho_ratio=3.0, mu_ratio=2.0, body_force=G, walls=walls)
    o.init_phi(I.multi_droplet_phi(grid, 7, 3, (3.0, 5.0), 3.0), I.smooth_velocity(grid, 8, 0.02))
    s0 = o.mass()[0]
    o.step(200)
    assert abs(o.mass()[0] - s0) / s0 < 1e-13


@pytest.mark.parametrize("Q,grid,walls", [(19, (6, 5, 4), 7), (9, (6, 5, 1), 3)])
def test_rest_state_is_fixed_point_with_walls(Q, grid, walls):
    o = O.Oracle(Q, grid, 0.8, 0.8, 0.02, 4.0, 1e-3, rho_ratio=2.0, walls=walls)
    o.init_phi(np.full(o.shape, 0.4), None, 0.3)
    f0, g0 = o.get_pops()
    o.step(20)
    f1, g1 = o.get_pops()
    np.testing.assert_allclose(f1, f0, atol=1e-14, rtol=0)
    np.testing.assert_allclose(g1, g0, atol=1e-14, rtol=0)


def test_invalid_wall_masks_rejected():
    with pytest.raises(ValueError):
        O.Oracle(9, (6, 5, 1), 0.8, 0.8, 0.02, 4.0, 1e-3, walls=4)
    with pytest.raises(ValueError):
        O.Oracle(19, (6, 5, 4), 0.8, 0.8, 0.02, 4.0, 1e-3, walls=8)
