"""Pins of the oracle's building blocks against closed forms (no GPU).

Each test checks one function the oracle's time step calls against what the paper and
lattice-Boltzmann moment algebra fix: lattice isotropy, the moments of f^eq, g^eq and the
forcing terms (App. A), Lax-Wendroff exactness on quadratics (Sec. 2.2), the recovery of
p, u, grad phi and n from populations built with known moments (Sec. 2.2, Sec. 2.3, App. B),
and the isotropic finite-difference gradient on quadratic fields.
"""
from pathlib import Path

import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0
GOLDEN = Path(__file__).parent / "golden"
RNG = np.random.default_rng(12263)


def _moments(Q, pops):
    d, e, t = O.lattice(Q)
    e = e.astype(float)
    return pops.sum(), e.T @ pops, np.einsum("i,ia,ib->ab", pops, e, e)


# ---------------------------------------------------------------- lattices
def test_d2q9_matches_paper_velocity_set():
    rows = np.loadtxt(GOLDEN / "d2q9_velocity_set.txt")
    d, e, t = O.lattice(9)
    assert d == 2
    np.testing.assert_array_equal(e[:, :2], rows[:, 1:3].astype(int))
    np.testing.assert_allclose(t, rows[:, 3] / rows[:, 4], rtol=0, atol=1e-16)
    # the angle formula of Sec. 2.2
    for i in range(1, 9):
        th = (i - 1) * np.pi / 2 if i <= 4 else (i - 5) * np.pi / 2 + np.pi / 4
        r = 1.0 if i <= 4 else np.sqrt(2.0)
        np.testing.assert_allclose(e[i, :2], [r * np.cos(th), r * np.sin(th)], atol=1e-12)


@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_isotropy(Q):
    d, e, t = O.lattice(Q)
    e = e.astype(float)
    I = np.eye(3)
    I[d:, d:] = 0
    assert abs(t.sum() - 1) < 1e-15
    np.testing.assert_allclose(t @ e, 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", t, e, e), CS2 * I, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", t, e, e, e), 0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", t, e, e, e, e)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                      + np.einsum("ad,bc->abcd", I, I))
    np.testing.assert_allclose(four, iso, atol=1e-16)
    # every velocity has its opposite
    for i in range(Q):
        assert any((e[j] == -e[i]).all() for j in range(Q))
    assert len({tuple(v) for v in e}) == Q


def test_d3q19_weights_by_speed():
    d, e, t = O.lattice(19)
    e2 = (e * e).sum(1)
    assert d == 3 and sorted(np.bincount(e2)) == [1, 6, 12]
    np.testing.assert_allclose(t[e2 == 0], 1 / 3)
    np.testing.assert_allclose(t[e2 == 1], 1 / 18)
    np.testing.assert_allclose(t[e2 == 2], 1 / 36)


# ---------------------------------------------------------------- propagation
def test_lax_wendroff_is_exact_shift_on_quadratics():
    """LW along a link moves a quadratic profile by exactly c cells (second-order scheme)."""
    for _ in range(50):
        a, b, q = RNG.normal(size=3)
        c = RNG.uniform(0.05, 1.0)
        f = lambda s: a + b * s + q * s * s
        got = O.lax_wendroff(c, f(-1.0), f(0.0), f(1.0))
        assert abs(got - f(-c)) < 1e-12 * (1 + abs(f(-c)))


def test_lax_wendroff_unit_courant_is_streaming():
    for _ in range(10):
        v = RNG.normal(size=3)
        assert O.lax_wendroff(1.0, *v) == pytest.approx(v[0], abs=1e-15)
    c = 0.997  # Sec. 2.2
    am, a0, ap = (O.lax_wendroff(c, 1, 0, 0), O.lax_wendroff(c, 0, 1, 0), O.lax_wendroff(c, 0, 0, 1))
    assert am + a0 + ap == pytest.approx(1.0, abs=1e-15)
    assert am - ap == pytest.approx(c, abs=1e-15)   # first moment: shift by c


# ---------------------------------------------------------------- equilibria
def _random_state(d):
    u = RNG.normal(size=3) * 0.05
    n = RNG.normal(size=3)
    if d == 2:
        u[2] = n[2] = 0
    n /= np.linalg.norm(n)
    return u, n


@pytest.mark.parametrize("Q", [9, 19])
def test_feq_moments(Q):
    d = 2 if Q == 9 else 3
    I = np.eye(3)
    I[d:, d:] = 0
    for _ in range(20):
        u, n = _random_state(d)
        p, rho = RNG.uniform(0.2, 0.5), RNG.uniform(0.5, 3)
        pis = O.css_tensor(d, RNG.uniform(0, 0.01), RNG.uniform(0, 0.5), n)
        m0, m1, m2 = _moments(Q, O.feq(Q, p, rho, u, pis))
        assert m0 == pytest.approx(p / CS2, abs=1e-14)
        np.testing.assert_allclose(m1, rho * u, atol=1e-15)
        # App. A: Pi^eq = rho u u + p I - Pi_s
        np.testing.assert_allclose(m2, p * I + rho * np.outer(u, u) - pis, atol=1e-14)


def test_feq_printed_sign_gives_plus_pis():
    """With the sign as printed in Eq. geq_s the second moment carries +Pi_s (not App. A's -Pi_s)."""
    u, n = _random_state(3)
    pis = O.css_tensor(3, 0.01, 0.3, n)
    _, _, m2 = _moments(19, O.feq(19, 0.3, 1.0, u, pis, pis_sign=+1))
    np.testing.assert_allclose(m2 - (0.3 * np.eye(3) + np.outer(u, u)), pis, atol=1e-14)


@pytest.mark.parametrize("Q", [9, 19])
def test_geq_moments(Q):
    d = 2 if Q == 9 else 3
    I = np.eye(3)
    I[d:, d:] = 0
    for _ in range(20):
        u, n = _random_state(d)
        phi, tau = RNG.uniform(0, 1), RNG.uniform(0.05, 2)
        S = 4 * phi * (1 - phi) / 4.0 * n
        m0, m1, m2 = _moments(Q, O.geq(Q, phi, u, S, tau))
        assert m0 == pytest.approx(phi, abs=1e-15)
        # first moment phi u + tau cs^2 S: the flux the CPF equation needs with M = tau cs^2
        np.testing.assert_allclose(m1, phi * u + tau * CS2 * S, atol=1e-15)
        np.testing.assert_allclose(m2, CS2 * phi * I + phi * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("Q", [9, 19])
def test_forcing_moments(Q):
    d = 2 if Q == 9 else 3
    for _ in range(20):
        u, _ = _random_state(d)
        grho = RNG.normal(size=3) * 0.1
        G = RNG.normal(size=3) * 1e-4
        if d == 2:
            grho[2] = G[2] = 0
        rho = RNG.uniform(0.5, 3)
        Si, Ri = O.forcing(Q, rho, u, grho, G)
        s0, s1, _ = _moments(Q, Si)
        r0, r1, r2 = _moments(Q, Ri)
        assert s0 == pytest.approx(u @ grho, abs=1e-15)        # App. A: sum S_i = u . grad rho
        np.testing.assert_allclose(s1, 0, atol=1e-15)           # compensation carries no momentum
        assert abs(r0) < 1e-16
        np.testing.assert_allclose(r1, rho * G, atol=1e-17)     # Eq. body: sum R_i e_i = rho G
        F = rho * G
        np.testing.assert_allclose(r2, np.outer(u, F) + np.outer(F, u), atol=1e-17)


def test_css_tensor_is_tangential_projector():
    for d in (2, 3):
        _, n = _random_state(d)
        pis = O.css_tensor(d, 0.02, 0.7, n)
        np.testing.assert_allclose(pis, pis.T, atol=0)
        np.testing.assert_allclose(pis @ n, 0, atol=1e-16)
        assert np.trace(pis) == pytest.approx(0.02 * 0.7 * (d - 1), rel=1e-14)
        if d == 2:
            assert np.abs(pis[2]).max() == 0 and np.abs(pis[:, 2]).max() == 0


# ---------------------------------------------------------------- recovery of macroscopic fields
def _consistent_populations(o, Q, phi, u, p, gphi, G, delta, sigma, drho):
    """fbar = f^eq - F/2 and g = g^eq - (tau+1/2) t e.grad phi: populations whose moments the
    scheme must turn back into exactly (phi, u, p, grad phi, n)."""
    d, e, t = O.lattice(Q)
    n = gphi / np.linalg.norm(gphi)
    S = 4 * phi * (1 - phi) / delta * n
    rho = 1.0 + drho * phi
    pis = O.css_tensor(d, sigma, np.linalg.norm(gphi), n)
    Si, Ri = O.forcing(Q, rho, u, drho * gphi, G)
    fbar = O.feq(Q, p, rho, u, pis) - 0.5 * (Si + Ri)
    g = O.geq(Q, phi, u, S, o.tau_phi) - (o.tau_phi + 0.5) * t * (e @ gphi)
    return fbar, g, n, S, rho


@pytest.mark.parametrize("Q", [9, 19])
def test_macroscopic_recovery(Q):
    d = 2 if Q == 9 else 3
    for trial in range(20):
        rho_ratio = [1.0, 3.0, 0.1][trial % 3]
        G = RNG.normal(size=3) * 1e-4
        if d == 2:
            G[2] = 0
        tau_g = RNG.uniform(0.05, 1.5)
        grid = (3, 3, 1) if Q == 9 else (3, 3, 3)
        o = O.Oracle(Q, grid, 0.8, tau_g, 0.0, 4.0, 1e-3, rho_ratio=rho_ratio, body_force=G)
        u, n = _random_state(d)
        phi = RNG.uniform(0.1, 0.9)
        gphi = 4 * phi * (1 - phi) / 4.0 * RNG.uniform(0.8, 1.2) * n
        p = RNG.uniform(0.3, 0.4)
        fbar, g, n, S, rho = _consistent_populations(o, Q, phi, u, p, gphi, G, 4.0, 1e-3, rho_ratio - 1)
        m = o.macroscopic_cell(fbar, g)
        assert m["phi"] == pytest.approx(phi, abs=1e-14)
        assert m["rho"] == pytest.approx(rho, abs=1e-14)
        np.testing.assert_allclose(m["u"], u, atol=1e-14)              # Eq. momentum (+ rho G / 2)
        np.testing.assert_allclose(m["n"], n, atol=1e-12)              # Eq. norm
        np.testing.assert_allclose(m["S"], S, atol=1e-13)
        np.testing.assert_allclose(m["grad_phi"], gphi, atol=1e-13)    # Sec. 2.3 / App. B
        np.testing.assert_allclose(m["grad_rho"], (rho_ratio - 1) * gphi, atol=1e-13)
        assert m["p"] == pytest.approx(p, abs=1e-14)                    # Eq. pressure
        # the finite-difference variant takes grad phi as given
        mf = o.macroscopic_cell(fbar, g, fd_grad=gphi)
        np.testing.assert_allclose(mf["n"], n, atol=1e-14)
        assert mf["p"] == pytest.approx(p, abs=1e-14)
        o.close()


def test_printed_half_force_sign_misses_velocity():
    G = np.array([1e-3, -2e-3, 5e-4])
    o = O.Oracle(19, (3, 3, 3), 0.8, 0.8, 0.0, 4.0, 1e-3, body_force=G, half_force_sign=-1)
    u, n = _random_state(3)
    gphi = 0.05 * n
    fbar, g, *_ = _consistent_populations(o, 19, 0.5, u, 0.33, gphi, G, 4.0, 1e-3, 0.0)
    m = o.macroscopic_cell(fbar, g)
    np.testing.assert_allclose(m["u"], u - G, atol=1e-14)   # off by exactly rho G / rho


# ---------------------------------------------------------------- collision
@pytest.mark.parametrize("Q", [9, 19])
def test_collision_relaxes_nonequilibrium_and_conserves(Q):
    d, e, t = O.lattice(Q)
    G = np.array([2e-4, -1e-4, 0.0 if Q == 9 else 3e-4])
    o = O.Oracle(Q, (3, 3, 1) if Q == 9 else (3, 3, 3), 0.7, 0.4, 0.0, 4.0, 2e-3,
                 rho_ratio=2.0, mu_ratio=3.0, body_force=G)
    u, n = _random_state(d)
    phi = 0.4
    gphi = 4 * phi * (1 - phi) / 4.0 * 0.9 * n   # near the equilibrium slope, so -K1 points along n
    fbar_eq, g_eq_ce, n, S, rho = _consistent_populations(o, Q, phi, u, 0.33, gphi, G, 4.0, 2e-3, 1.0)
    m = o.macroscopic_cell(fbar_eq, g_eq_ce)
    # non-equilibrium with vanishing conserved moments (0th and 1st)
    ghost = RNG.normal(size=Q) * 1e-3
    A = np.vstack([np.ones(Q), e.T.astype(float)])
    ghost -= A.T @ np.linalg.lstsq(A.T, ghost, rcond=None)[0]
    fs, gs = o.collide_cell(fbar_eq + ghost, g_eq_ce, m)
    Si, Ri = O.forcing(Q, rho, m["u"], m["grad_rho"], G)
    fs0, _ = o.collide_cell(fbar_eq, g_eq_ce, m)
    np.testing.assert_allclose(fs0, fbar_eq + (Si + Ri), atol=1e-15)   # f* = fbar^eq + F at equilibrium
    # Eq. c-n_m with the local viscosity reading: eta = eta2 + (eta1 - eta2) phi, tau = eta/(rho cs^2)
    tau_rho = 0.7 * (1 + (3.0 - 1) * phi) / rho
    np.testing.assert_allclose(fs - fs0, (1 - 1 / (tau_rho + 0.5)) * ghost, atol=1e-15)
    # g: phi conserved cell by cell, relaxation factor 1 - 1/(tau_phi + 1/2) (Eq. c-n_c)
    assert gs.sum() == pytest.approx(g_eq_ce.sum(), abs=1e-15)
    geq = O.geq(Q, phi, m["u"], m["S"], o.tau_phi)
    np.testing.assert_allclose(gs - geq, (1 - 1 / (o.tau_phi + 0.5)) * (g_eq_ce - geq), atol=1e-15)


# ---------------------------------------------------------------- finite-difference gradient
@pytest.mark.parametrize("Q", [9, 19])
def test_isotropic_gradient_exact_on_quadratics(Q):
    nx, ny, nz = (12, 10, 1) if Q == 9 else (10, 9, 8)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = RNG.normal(size=10)
    if Q == 9:
        c[[3, 6, 8, 9]] = 0   # no z dependence in 2D
    f = (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
         + c[7] * x * y + c[8] * x * z + c[9] * y * z)
    gx = c[1] + 2 * c[4] * x + c[7] * y + c[8] * z
    gy = c[2] + 2 * c[5] * y + c[7] * x + c[9] * z
    gz = c[3] + 2 * c[6] * z + c[8] * x + c[9] * y
    grad = O.isotropic_gradient(Q, f)
    inner = (slice(1, -1) if nz > 1 else slice(None), slice(1, -1), slice(1, -1))
    for a, ref in enumerate((gx, gy, gz)):
        np.testing.assert_allclose(grad[a][inner], ref[inner], atol=1e-11)
