"""Pins of the oracle's full time step against physics the paper and the mathematics fix (no GPU).

* invariants: a uniform state is a fixed point; sum phi is conserved to round-off; total
  momentum changes by exactly N rho G per step (Eq. momentum, Eq. body);
* transport coefficients: a shear wave decays with nu = cs^2 tau_rho (Eq. c-n_m), a phi
  perturbation diffuses with M = tau_phi cs^2 and is advected with u (Eq. geq, Eq. c-n_c);
* the interface: the 1D tanh profile of Eq. cac with width delta is a steady state, and the
  moment-based gradient of Sec. 2.3 equals dphi/dx = 4 phi (1 - phi) / delta there;
* the normal of Eq. norm points along +grad phi (outward for the droplet of Eq. initial_droplet);
* Laplace's law for the static droplet of Sec. 3.1 (p_in - p_out = sigma / R in 2D);
* the difference-free and finite-difference gradients and normals agree (Sec. 3.4);
* the printed forms of the ambiguous passages fail these pins.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import inputs as I

CS2 = 1.0 / 3.0


def _mk(Q, grid, **kw):
    args = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)
    args.update(kw)
    return O.Oracle(Q, grid, **args)


def _momentum(o):
    f, _ = o.get_pops()
    d, e, t = O.lattice(o.Q)
    return np.einsum("qzyx,qa->a", f, e.astype(float))


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("Q,grid", [(9, (6, 5, 1)), (19, (5, 4, 3))])
def test_uniform_state_is_fixed_point(Q, grid):
    o = _mk(Q, grid, rho_ratio=3.0, mu_ratio=0.5)
    u0 = np.zeros((3,) + o.shape)
    u0[0], u0[1] = 0.03, -0.02
    if Q == 19:
        u0[2] = 0.01
    o.init_phi(np.full(o.shape, 0.37), u0, 0.3)
    f0, g0 = o.get_pops()
    o.step(25)
    f1, g1 = o.get_pops()
    np.testing.assert_allclose(f1, f0, atol=1e-14, rtol=0)
    np.testing.assert_allclose(g1, g0, atol=1e-14, rtol=0)


@pytest.mark.parametrize("Q,grid,scheme", [(9, (40, 36, 1), 0), (19, (14, 13, 12), 0),
                                           (9, (40, 36, 1), 1), (19, (14, 13, 12), 1)])
def test_phi_conserved_to_roundoff(Q, grid, scheme):
    G = (2e-5, -1e-5, 0.0 if Q == 9 else 1.5e-5)
    o = _mk(Q, grid, rho_ratio=3.0, mu_ratio=2.0, body_force=G, scheme=scheme)
    phi0 = I.multi_droplet_phi(grid, seed=7, count=3, r_range=(3.0, 6.0), xi=3.0)
    o.init_phi(phi0, I.smooth_velocity(grid, seed=8, amplitude=0.02))
    s0, _ = o.mass()
    o.step(150)
    s1, _ = o.mass()
    assert abs(s1 - s0) / s0 < 1e-13
    assert abs(s0 - phi0.sum()) / s0 < 1e-3


@pytest.mark.parametrize("Q,grid", [(9, (20, 18, 1)), (19, (10, 9, 8))])
def test_momentum_budget(Q, grid):
    """sum_x sum_i f*_i e_i grows by exactly N rho G per step (density ratio 1)."""
    G = np.array([3e-5, -2e-5, 0.0 if Q == 9 else 1e-5])
    o = _mk(Q, grid, body_force=G)
    o.init_phi(I.multi_droplet_phi(grid, seed=3, count=2, r_range=(3.0, 5.0), xi=3.0),
               I.smooth_velocity(grid, seed=4, amplitude=0.01))
    P0 = _momentum(o)
    o.step(40)
    P1 = _momentum(o)
    np.testing.assert_allclose(P1 - P0, 40 * o.N * G, rtol=1e-9, atol=1e-15)


def test_printed_half_force_sign_breaks_momentum_budget():
    G = np.array([3e-5, -2e-5, 0.0])
    o = _mk(9, (20, 18, 1), body_force=G, half_force_sign=-1)
    o.init_phi(I.multi_droplet_phi((20, 18, 1), seed=3, count=2, r_range=(3.0, 5.0), xi=3.0))
    P0 = _momentum(o)
    o.step(40)
    got = (_momentum(o) - P0)[:2] / (40 * o.N * G[:2])
    assert np.all(np.abs(got - 1) > 0.1)


# ---------------------------------------------------------------- transport coefficients
def _amp(field, ref):
    return float((field * ref).sum() / (ref * ref).sum())


@pytest.mark.parametrize("Q,grid,c,tol", [(9, (3, 64, 1), 1.0, 0.005), (19, (3, 48, 3), 1.0, 0.005),
                                          (9, (3, 64, 1), 0.997, 0.01)])
def test_shear_wave_decay_gives_viscosity(Q, grid, c, tol):
    """u_x = U sin(k y) decays as exp(-nu k^2 t) with nu = cs^2 tau_rho (single phase, sigma = 0)."""
    tau = 0.8
    o = _mk(Q, grid, tau_f=tau, sigma=0.0, courant=c)
    u0 = I.shear_wave(grid, 1e-3, axis_u=0, axis_k=1)
    o.init_phi(np.ones(o.shape), u0, CS2)
    o.step(10)
    a0 = _amp(o.moments()[2][0], u0[0])
    o.step(300)
    a1 = _amp(o.moments()[2][0], u0[0])
    k = 2 * np.pi / grid[1]
    nu = -np.log(a1 / a0) / (300 * k * k)
    assert nu == pytest.approx(CS2 * tau, rel=tol)


def test_phi_diffusion_and_advection_give_mobility():
    """With delta -> infinity (S -> 0) phi obeys d_t phi + u . grad phi = M lap phi, M = tau_phi cs^2."""
    grid = (64, 3, 1)
    M = 0.02
    for U in (0.0, 0.05):
        o = _mk(9, grid, M=M, xi=1e12, sigma=0.0, courant=1.0)
        u0 = np.zeros((3,) + (1, 3, 64))
        u0[0] = U
        o.init_phi(I.sine_phi(grid, 0.5, 0.01), u0)
        k = 2 * np.pi / 64
        x = np.arange(64)

        def mode():
            ph = o.moments()[0][0, 1] - 0.5
            return (ph * np.exp(-1j * k * x)).sum()

        m0 = mode()
        o.step(2000)
        m1 = mode()
        rate = -np.log(abs(m1) / abs(m0)) / (2000 * k * k)
        assert rate == pytest.approx(M, rel=0.01)
        shift = -np.angle(m1 / m0) / k            # defined modulo the period 64
        lag = (shift - U * 2000 + 32) % 64 - 32
        assert abs(lag) < 0.01 * max(U * 2000, 1)


# ---------------------------------------------------------------- interface
def _fit_slab(phi_line, centre):
    from scipy.optimize import least_squares
    n = phi_line.size
    x = np.arange(n, dtype=float)

    def res(prm):
        d = np.abs(x - centre)
        d = np.minimum(d, n - d)
        return 0.5 * (1 + np.tanh(2 * (d - prm[0]) / prm[1])) - phi_line

    return least_squares(res, [n / 4, 4.0]).x


@pytest.mark.parametrize("M", [0.02, 0.8 / 3])
def test_tanh_interface_is_steady_with_width_delta(M):
    grid = (64, 3, 1)
    xi = 4.0
    o = _mk(9, grid, M=M, xi=xi)
    phi0 = I.slab_phi(grid, 16.0, xi)
    o.init_phi(phi0)
    o.step(2000)
    phi, p, u = o.moments()
    hw, width = _fit_slab(phi[0, 1], 31.5)
    assert hw == pytest.approx(16.0, abs=1e-6)
    assert width == pytest.approx(xi, rel=0.02)
    assert np.abs(phi - phi0).max() < 1e-2
    assert np.abs(u).max() < 1e-12          # flat interface: no flow
    assert p.max() - p.min() < 1e-12        # and no pressure jump
    # Sec. 2.3 gradient from moments equals dphi/dx of the steady profile
    gphi, n = o.gradients()
    band = (phi > 0.1) & (phi < 0.9)
    ana = 4 * phi * (1 - phi) / xi
    np.testing.assert_allclose(np.abs(gphi[0][band]), ana[band], rtol=0.02)
    np.testing.assert_allclose(np.abs(gphi[1][band]), 0, atol=1e-12)


def test_printed_geq_source_scale_fails_tanh_pin():
    grid = (64, 3, 1)
    o = _mk(9, grid, geq_source_tau=0)
    phi0 = I.slab_phi(grid, 16.0, 4.0)
    o.init_phi(phi0)
    o.step(300)
    phi = o.moments()[0]
    assert not np.all(np.isfinite(phi)) or np.abs(phi - phi0).max() > 0.05


@pytest.mark.parametrize("tau_g", [0.06, 0.8, 1.5])
def test_normal_points_along_grad_phi(tau_g):
    """n of Eq. norm points outward (along +grad phi) for the phi = 0 droplet, first step and later."""
    grid = (20, 19, 18)
    R, xi = 6.0, 4.0
    o = _mk(19, grid, tau_g=tau_g, M=0.0, xi=xi)
    centre = (9.5, 9.0, 8.5)
    o.init_phi(I.droplet_phi(grid, R, xi, centre=centre))
    x, y, z = I.cell_coords(grid)
    r = np.stack([x - centre[0], y - centre[1], z - centre[2]])
    rhat = r / np.maximum(np.linalg.norm(r, axis=0), 1e-9)
    for steps in (0, 20):
        o.step(steps)
        phi = o.moments()[0]
        _, n = o.gradients()
        band = (phi > 0.1) & (phi < 0.9)
        assert band.sum() > 100
        assert (n * rhat).sum(0)[band].min() > 0.99


def test_laplace_law_2d():
    """Static droplet of Sec. 3.1 (D2Q9, 64^2, R = 16, xi = 4): p_in - p_out = sigma / R_eff."""
    w = I.WORKLOADS["droplet2d_64"]
    o = O.Oracle(9, w["grid"], w["tau_f"], w["tau_g"], w["M"], w["xi"], w["sigma"])
    o.init_phi(I.droplet_phi(w["grid"], w["R"], w["xi"]))
    s0 = o.mass()[0]
    o.step(w["steps"])
    phi, p, u = o.moments()
    r = I.periodic_distance(w["grid"], (31.5, 31.5, 0.0))
    jump = p[r < w["R"] - 2 * w["xi"]].mean() - p[r > w["R"] + 2 * w["xi"]].mean()
    r_eff = np.sqrt((1 - phi).sum() / np.pi)
    assert jump == pytest.approx(w["sigma"] / r_eff, rel=0.05)
    assert abs(o.mass()[0] - s0) / s0 < 1e-12
    assert np.abs(u).max() < 1e-4           # spurious currents stay small


def test_printed_pis_sign_gives_negative_laplace_jump():
    w = I.WORKLOADS["droplet2d_64"]
    o = O.Oracle(9, w["grid"], w["tau_f"], w["tau_g"], w["M"], w["xi"], w["sigma"], pis_sign=+1)
    o.init_phi(I.droplet_phi(w["grid"], w["R"], w["xi"]))
    o.step(1000)
    phi, p, u = o.moments()
    r = I.periodic_distance(w["grid"], (31.5, 31.5, 0.0))
    jump = p[r < w["R"] - 2 * w["xi"]].mean() - p[r > w["R"] + 2 * w["xi"]].mean()
    assert jump < -0.5 * w["sigma"] / w["R"]


def test_laplace_law_3d_small():
    """3D static droplet (D3Q19, 32^3, R = 10): p_in - p_out = 2 sigma / R_eff within 10%."""
    grid, R, xi = (32, 32, 32), 10.0, 4.0
    o = _mk(19, grid, xi=xi)
    o.init_phi(I.droplet_phi(grid, R, xi))
    o.step(1000)
    phi, p, u = o.moments()
    r = I.periodic_distance(grid, (15.5, 15.5, 15.5))
    jump = p[r < R - 2 * xi].mean() - p[r > R + 2 * xi].mean()
    r_eff = ((1 - phi).sum() * 3 / (4 * np.pi)) ** (1 / 3)
    assert jump == pytest.approx(2e-3 / r_eff, rel=0.10)


@pytest.mark.parametrize("xi", [4.0, 8.0])
@pytest.mark.parametrize("Q,grid,R", [(9, (48, 48, 1), 12.0), (19, (24, 24, 24), 7.0)])
def test_difference_free_and_fd_gradients_agree(Q, grid, R, xi):
    """Both gradients match dphi/dn = 4 phi (1 - phi)/xi across the interface: the moment-based
    one to 1%, the central difference within its truncation error h^2/6 |phi'''/phi'|, at most
    4/(3 xi^2) for the tanh profile."""
    out = {}
    for scheme in (0, 1):
        o = _mk(Q, grid, xi=xi, scheme=scheme)
        o.init_phi(I.droplet_phi(grid, R, xi))
        o.step(100)
        phi = o.moments()[0]
        gphi, n = o.gradients()
        out[scheme] = (phi, gphi, n)
    phi = out[0][0]
    band = (phi > 0.1) & (phi < 0.9)
    ana = (4 * phi * (1 - phi) / xi)[band]
    g0, g1 = out[0][1][:, band], out[1][1][:, band]
    n0, n1 = out[0][2][:, band], out[1][2][:, band]
    trunc = 4.0 / (3.0 * xi * xi)
    assert abs(np.median(np.linalg.norm(g0, axis=0) / ana) - 1) < 0.01
    assert abs(np.median(np.linalg.norm(g1, axis=0) / ana) - 1) < trunc + 0.01
    assert np.linalg.norm(g0 - g1) / np.linalg.norm(g1) < trunc + 0.02
    cosang = (n0 * n1).sum(0)
    assert np.degrees(np.arccos(np.clip(cosang.min(), -1, 1))) < 5.0
    assert np.abs(out[0][0] - out[1][0]).max() < 0.02


@pytest.mark.parametrize("Q,grid", [(9, (12, 11, 1)), (19, (8, 7, 6))])
def test_initial_state_moments(Q, grid):
    """The initial populations carry phi0, p0 and rho0 u0 exactly (post-collision form of the
    Chapman-Enskog state; see the initialisation reading in the oracle header)."""
    o = _mk(Q, grid, rho_ratio=2.0)
    phi0 = I.multi_droplet_phi(grid, seed=1, count=2, r_range=(2.0, 4.0), xi=3.0)
    u0 = I.smooth_velocity(grid, seed=2, amplitude=0.02)
    o.init_phi(phi0, u0, 0.31)
    f, g = o.get_pops()
    d, e, t = O.lattice(Q)
    np.testing.assert_allclose(g.sum(0), phi0, atol=1e-15)
    np.testing.assert_allclose(f.sum(0), 0.31 / CS2, atol=1e-14)
    rho0 = 1.0 + phi0
    np.testing.assert_allclose(np.einsum("q...,qa->a...", f, e.astype(float)), rho0 * u0, atol=1e-15)
    gphi0 = O.isotropic_gradient(Q, phi0)
    S0 = 4 * phi0 * (1 - phi0) / 4.0 * gphi0 / np.maximum(np.linalg.norm(gphi0, axis=0), 1e-300)
    want = phi0 * u0 + o.tau_phi * CS2 * S0 - (o.tau_phi - 0.5) * CS2 * gphi0
    np.testing.assert_allclose(np.einsum("q...,qa->a...", g, e.astype(float)), want, atol=1e-14)
