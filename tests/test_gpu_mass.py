"""Parity of the mass diagnostic (sum phi and sum rho phi, the mass m = sum rho phi of Sec. 3.3)
with the FP64 oracle, through the C ABI.

Two comparisons:
* matched states: the oracle's populations are first rounded to values the storage holds
  exactly (g_i - t_i on the FP32, scaled FP16 or BF16 grid: a handle given populations by
  lbm_set_pops before any lbm_init_phi holds g_i - t_i), then loaded both into the oracle and
  into a handle, and lbm_mass is compared with oracle.mass() on that state. What remains is the
  FP32 evaluation of the integer face fluxes and the fixed-point rounding of phi, bounded per
  cell below. The bound is small enough that a sum over the pre-propagation state, a wrong
  fixed-point scale or a wrong density would fail it (the test checks the first margin);
* independent runs: the GPU and the oracle start from the same phi0 and each takes 150 steps;
  sum phi is conserved on both sides, and sum rho phi differs by no more than the element-wise
  difference of their phi fields allows.

Cases: D2Q9 and D3Q19, periodic and walled, density ratio 3 with viscosity ratio and body
force, FP32, FP16 and BF16 storage, after 0 and 150 oracle steps.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu

STORAGES = [lbm.LBM_STORAGE_FP32, lbm.LBM_STORAGE_FP16, lbm.LBM_STORAGE_BF16]
FX_HALF = 2.0 ** -31    # half the fixed-point resolution of phi
COURANT = 0.997
A_M, A_P = 0.5 * COURANT * (1 + COURANT), -0.5 * COURANT * (1 - COURANT)

PARAMS = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3, rho_ratio=3.0, mu_ratio=2.0)
GEOMETRIES = [  # (Q, grid, walls)
    (9, (45, 39, 1), 0), (9, (45, 39, 1), 3),
    (19, (37, 21, 19), 0), (19, (37, 21, 19), 4), (19, (26, 22, 18), 7),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _force(Q):
    return (2e-5, -1e-5, 0.0) if Q == 9 else (2e-5, -1e-5, 1.5e-5)


def _inputs(Q, grid):
    phi0 = I.multi_droplet_phi(grid, seed=91, count=3, r_range=(3.0, 7.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=92, amplitude=0.03)
    if Q == 9:
        u0[2] = 0
    return phi0, u0


@functools.lru_cache(maxsize=None)
def _oracle_state(Q, grid, walls, steps):
    """(f, g, sum phi, sum rho phi) of the oracle after `steps` steps."""
    phi0, u0 = _inputs(Q, grid)
    ref = O.Oracle(Q, grid, body_force=_force(Q), walls=walls, courant=COURANT, **PARAMS)
    ref.init_phi(phi0, u0)
    ref.step(steps)
    f, g = ref.get_pops()
    s_phi, s_rphi = ref.mass()
    ref.close()
    return f, g, s_phi, s_rphi


def _representable(Q, g, storage):
    """g with every g_i - t_i (i >= 1) rounded to the storage's grid: FP32, FP16 after scaling by
    2^10, or BF16 (round to nearest even on the upper 16 bits of the FP32 pattern)."""
    _, _, t = O.lattice(Q)
    tb = t[1:, None, None, None]
    d = (g[1:] - tb).astype(np.float32)
    if storage == lbm.LBM_STORAGE_FP16:
        d = (d * np.float32(1024.0)).astype(np.float16).astype(np.float32) / np.float32(1024.0)
    elif storage == lbm.LBM_STORAGE_BF16:
        bits = d.view(np.uint32).astype(np.uint64)
        bits = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
        d = bits.astype(np.uint32).view(np.float32)
    out = g.copy()
    out[1:] = tb + d.astype(np.float64)
    return out


def _oracle_mass_of(Q, grid, walls, f, g):
    ref = O.Oracle(Q, grid, body_force=_force(Q), walls=walls, courant=COURANT, **PARAMS)
    ref.set_pops(f, g)
    m = ref.mass()
    ref.close()
    return m


def _rounding_bounds(Q, g):
    """Worst-case |d sum phi| and |d sum rho phi| between the oracle and a handle holding the
    same (exactly representable) state. Each cell's propagated phi is its fixed-point phi*
    (rounded by at most 2^-31) plus the integer net fluxes across its Q - 1 faces. A flux
    a- (A) - a+ (B) takes differences A, B of stored values within one cell's stencil (at most
    2 D, D the largest |g_i - t_i| around the cell) and a few FP32 operations, each rounded by
    2^-24 of its result, then it is rounded to the fixed-point grid (2^-31). sum phi is exact on
    the device, because the fluxes cancel in pairs."""
    _, _, t = O.lattice(Q)
    dev = np.abs(g[1:] - t[1:, None, None, None]).max(0)
    D = dev.copy()
    for ax in range(3):
        if D.shape[ax] > 1:
            D = np.maximum(D, np.maximum(np.roll(D, 1, ax), np.roll(D, -1, ax)))
    per_face = 4 * 2.0 ** -24 * 2 * D * (abs(A_M) + abs(A_P)) + FX_HALF
    per_cell = FX_HALF + (Q - 1) * per_face
    phi = g.sum(0)
    slope = np.abs(1.0 + 2.0 * (PARAMS["rho_ratio"] - 1.0) * phi) + 1e-3
    n = phi.size
    return n * FX_HALF + 1e-12 * n, float((slope * per_cell).sum()) + 1e-12 * n


@pytest.mark.parametrize("steps", [0, 150])
@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("Q,grid,walls", GEOMETRIES)
def test_mass_matches_oracle_on_the_same_state(Q, grid, walls, storage, steps):
    f, g0, _, _ = _oracle_state(Q, grid, walls, steps)
    g = _representable(Q, g0, storage)
    s_phi, s_rphi = _oracle_mass_of(Q, grid, walls, f, g)
    tol_phi, tol_rphi = _rounding_bounds(Q, g)
    with lbm.Lattice(grid, Q, body_force=_force(Q), walls=walls, storage=storage, courant=COURANT, **PARAMS) as h:
        h.set_pops(f, g)
        got_phi, got_rphi = h.mass()
    assert abs(got_phi - s_phi) <= tol_phi, (got_phi, s_phi, tol_phi)
    assert abs(got_rphi - s_rphi) <= tol_rphi, (got_rphi, s_rphi, tol_rphi)
    # the same sum over the pre-propagation phi* = sum_i g*_i misses by far more than the bound
    phis = g.sum(0)
    pre = float(((1.0 + (PARAMS["rho_ratio"] - 1.0) * phis) * phis).sum())
    assert abs(pre - s_rphi) > 5 * tol_rphi


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("Q,grid,walls", [GEOMETRIES[1], GEOMETRIES[2], GEOMETRIES[4]])
def test_mass_after_independent_runs_matches_oracle(Q, grid, walls, storage):
    """GPU and oracle each take 150 steps from the same phi0. sum phi: exact on the GPU and
    conserved to round-off by the oracle, so the two agree to the fixed-point rounding of phi0.
    sum rho phi: within the sum over cells of |rho phi| differences of the two phi fields (FP32
    moments of the GPU: a further 2^-24 relative per cell)."""
    phi0, u0 = _inputs(Q, grid)
    ref = O.Oracle(Q, grid, body_force=_force(Q), walls=walls, courant=COURANT, **PARAMS)
    ref.init_phi(phi0, u0)
    with lbm.Lattice(grid, Q, body_force=_force(Q), walls=walls, storage=storage, courant=COURANT, **PARAMS) as h:
        h.init_phi(phi0, u0)
        m0 = h.mass()
        h.step(150)
        got_phi, got_rphi = h.mass()
        phi_g = h.moments()[0]
    ref.step(150)
    s_phi, s_rphi = ref.mass()
    phi_o = ref.moments()[0]
    n = phi0.size
    assert got_phi == m0[0]
    assert abs(got_phi - phi0.sum()) <= n * FX_HALF + 1e-12 * n
    assert abs(got_phi - s_phi) <= n * FX_HALF + 1e-12 * n
    drho = PARAMS["rho_ratio"] - 1.0
    rphi = lambda p: (1.0 + drho * p) * p  # noqa: E731
    slope = np.abs(1.0 + 2.0 * drho * np.maximum(np.abs(phi_g), np.abs(phi_o))).max() + 1.0
    bound = np.abs(rphi(phi_g) - rphi(phi_o)).sum() + n * slope * 2.0 ** -24 * (np.abs(phi_g).max() + 1.0)
    assert abs(got_rphi - s_rphi) <= bound, (got_rphi, s_rphi, bound)
    ref.close()
