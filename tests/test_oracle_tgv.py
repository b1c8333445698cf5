"""Oracle pins of the Taylor-Green initial condition (Sec. 3.4): the pressure field enters f^eq,
a single-phase vortex decays at the viscous rate, and the printed pressure field is the one
that balances the initial vortex (a uniform or sign-flipped pressure launches an acoustic
transient). Arguments are taken as 2 pi x / n, so the vortex is periodic on the grid."""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import inputs as I

CS2 = 1.0 / 3.0
N = 32
GRID = (N, N, N)
U0 = 0.01
NU = 0.05
K2 = 3 * (2 * np.pi / N) ** 2          # |k|^2 of every Fourier mode of the vortex
AMP = U0 * U0 / 16 * 4                  # largest pressure deviation of the field


def _single_phase(p=None):
    o = O.Oracle(19, GRID, 3 * NU, 0.8, 0.02, 4.0, 0.0)
    o.init_phi(np.ones((N, N, N)), I.taylor_green_velocity(GRID, U0), p=p)
    return o


def test_initial_pressure_field_enters_feq():
    """sum_i f*_i = p / cs^2 and sum_i f*_i e_i = rho u in every cell of the initial state
    (moments of the equilibrium of Eq. geq_s)."""
    p = I.taylor_green_pressure(GRID, U0)
    o = _single_phase(p)
    f, _ = o.get_pops()
    _, e, _ = O.lattice(19)
    np.testing.assert_allclose(f.sum(axis=0) * CS2, p, rtol=0, atol=1e-15)
    j = np.einsum("qzyx,qa->azyx", f, e.astype(float))
    np.testing.assert_allclose(j, I.taylor_green_velocity(GRID, U0), rtol=0, atol=1e-15)


def test_taylor_green_pressure_is_the_closed_form():
    """The pressure recipe against the expression written out at a few cells."""
    p = I.taylor_green_pressure(GRID, 0.04, p0=0.5, rho0=2.0)
    for x, y, z in ((0, 0, 0), (3, 17, 30), (31, 8, 16)):
        X, Y, Z = (2 * np.pi * x / N, 2 * np.pi * y / N, 2 * np.pi * z / N)
        want = 0.5 + 2.0 * 0.04 ** 2 / 16 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2)
        assert p[z, y, x] == pytest.approx(want, abs=1e-16)


def test_vortex_decays_at_the_viscous_rate():
    """Kinetic energy ~ exp(-2 nu k^2 t) with nu = cs^2 tau (low amplitude, linear regime):
    the fitted rate within 0.5% after 100 steps and 0.1% after 200."""
    o = _single_phase(I.taylor_green_pressure(GRID, U0))
    e0 = (o.moments()[2] ** 2).sum()
    o.step(100)
    rate100 = -np.log((o.moments()[2] ** 2).sum() / e0) / (2 * NU * K2 * 100)
    o.step(100)
    rate200 = -np.log((o.moments()[2] ** 2).sum() / e0) / (2 * NU * K2 * 200)
    assert rate100 == pytest.approx(1.0, abs=5e-3)
    assert rate200 == pytest.approx(1.0, abs=1e-3)


@pytest.mark.parametrize("start,bound", [("field", (0.0, 0.1)), ("uniform", (0.3, 10.0)), ("flipped", (0.6, 10.0))])
def test_printed_pressure_balances_the_vortex(start, bound):
    """After 50 steps the pressure follows the decaying closed form
    p0 + (p_TG - p0) exp(-2 nu k^2 t) to within 10% of its amplitude when the run starts from
    the printed field; starting from a uniform pressure, or from the field with its sign
    flipped, leaves a transient of 30% and 60% or more."""
    p_tg = I.taylor_green_pressure(GRID, U0)
    p = {"field": p_tg, "uniform": None, "flipped": 2 * CS2 - p_tg}[start]
    o = _single_phase(p)
    o.step(50)
    expect = CS2 + (p_tg - CS2) * np.exp(-2 * NU * K2 * 50)
    dev = np.abs(o.moments()[1] - expect).max() / AMP
    assert bound[0] <= dev <= bound[1]
