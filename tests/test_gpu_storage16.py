"""16-bit population storage (FP16 scaled, BF16) against the FP64 oracle.

The moving (f_i, g_i) pairs are stored in 16 bits; the zeroth-moment plane and all arithmetic
stay FP32. The stated bounds, after the step counts below, are looser than FP32's:
  FP16: max |phi - phi_oracle| <= 1e-3, rel-L2(u) <= 1e-2 on a moving flow, max |p| error <= 5e-6
  BF16: max |phi - phi_oracle| <= 1e-2, rel-L2(u) <= 3e-2 on a moving flow, max |p| error <= 3e-5
Sum phi does not change at all: the fixed-point phi plane advances by integer face fluxes that
cancel in pairs, whatever precision the moving populations carry.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu

# pop: half an ulp of a stored moving population (|deviation| <= 0.06 for g); the rest
# population is rebuilt from the FP32 moment minus the 18 stored ones, so it gets 18 of those
BOUNDS = {lbm.LBM_STORAGE_FP16: dict(phi=1e-3, u=1e-2, p=5e-6, pop=2e-5, u_static=2e-6),
          lbm.LBM_STORAGE_BF16: dict(phi=1e-2, u=3e-2, p=3e-5, pop=3e-4, u_static=2e-5)}
STORAGES = [lbm.LBM_STORAGE_FP16, lbm.LBM_STORAGE_BF16]


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _pair(storage, Q, grid, phi0, u0=None, scheme=0, **params):
    base = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)
    base.update(params)
    gpu = lbm.Lattice(grid, Q, storage=storage, scheme=scheme, **base)
    ref = O.Oracle(Q, grid, scheme=scheme, **base)
    gpu.init_phi(phi0, u0)
    ref.init_phi(phi0, u0)
    return gpu, ref


@pytest.mark.parametrize("storage", STORAGES)
def test_initial_populations_within_16bit_rounding(storage):
    grid = (21, 13, 9)
    phi0 = I.multi_droplet_phi(grid, seed=71, count=2, r_range=(3.0, 5.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=72, amplitude=0.03)
    gpu, ref = _pair(storage, 19, grid, phi0, u0, rho_ratio=2.0)
    (fg, gg), (fo, go) = gpu.get_pops(), ref.get_pops()
    b = BOUNDS[storage]["pop"]
    np.testing.assert_allclose(fg[1:], fo[1:], rtol=0, atol=b)
    np.testing.assert_allclose(gg[1:], go[1:], rtol=0, atol=b)
    np.testing.assert_allclose(fg[0], fo[0], rtol=0, atol=18 * b)
    np.testing.assert_allclose(gg[0], go[0], rtol=0, atol=18 * b)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("scheme", [0, 1])
def test_moving_flow_parity(storage, scheme):
    """Droplets in a smooth flow, density/viscosity ratio and body force on, 150 steps."""
    grid = (37, 21, 19)
    phi0 = I.multi_droplet_phi(grid, seed=73, count=3, r_range=(3.0, 7.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=74, amplitude=0.03)
    gpu, ref = _pair(storage, 19, grid, phi0, u0, scheme=scheme, rho_ratio=3.0, mu_ratio=2.0,
                     body_force=(2e-5, -1e-5, 1.5e-5))
    s0 = gpu.mass()[0]
    gpu.step(150)
    ref.step(150)
    (phi_g, p_g, u_g), (phi_o, p_o, u_o) = gpu.moments(), ref.moments()
    b = BOUNDS[storage]
    assert np.abs(phi_g - phi_o).max() <= b["phi"]
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) <= b["u"]
    assert np.abs(p_g - p_o).max() <= b["p"]
    assert gpu.mass()[0] == s0


@pytest.mark.parametrize("storage", STORAGES)
def test_static_droplet_parity(storage):
    """The 2D droplet workload (64^2, R = 16), 150 steps: spurious currents of |u| ~ 2e-5 are
    compared in absolute terms."""
    grid = (64, 64, 1)
    phi0 = I.droplet_phi(grid, 16.0, 4.0)
    gpu, ref = _pair(storage, 9, grid, phi0)
    s0 = gpu.mass()[0]
    gpu.step(150)
    ref.step(150)
    (phi_g, p_g, u_g), (phi_o, p_o, u_o) = gpu.moments(), ref.moments()
    b = BOUNDS[storage]
    assert np.abs(phi_g - phi_o).max() <= b["phi"]
    assert np.abs(u_g - u_o).max() <= b["u_static"]
    assert np.abs(p_g - p_o).max() <= b["p"]
    assert gpu.mass()[0] == s0


def test_fp16_laplace_law_3d_full_size():
    """The 128^3 droplet with FP16 storage, 5000 steps: Laplace's law within 5%, sum phi
    unchanged."""
    w = I.WORKLOADS["droplet3d_128"]
    grid, R, xi = w["grid"], w["R"], w["xi"]
    g = lbm.Lattice(grid, 19, w["tau_f"], w["tau_g"], w["M"], xi, w["sigma"], storage=lbm.LBM_STORAGE_FP16)
    g.init_phi(I.droplet_phi(grid, R, xi))
    s0 = g.mass()[0]
    g.step(w["steps"])
    phi, p, u = g.moments()
    r = I.periodic_distance(grid, (63.5, 63.5, 63.5))
    jump = p[r < R - 2 * xi].mean() - p[r > R + 2 * xi].mean()
    r_eff = ((1 - phi).sum() * 3 / (4 * np.pi)) ** (1 / 3)
    assert jump == pytest.approx(2 * w["sigma"] / r_eff, rel=0.05)
    assert g.mass()[0] == s0
    assert np.abs(u).max() < 1e-4


@pytest.mark.parametrize("storage", STORAGES)
def test_16bit_overflow_is_reported_as_nonfinite(storage):
    """A population far outside the 16-bit range (set on the host) reads back as non-finite."""
    grid = (8, 7, 6)
    g = lbm.Lattice(grid, 19, 0.8, 0.8, 0.02, 4.0, 1e-3, storage=storage)
    g.init_phi(I.droplet_phi(grid, 2.5, 4.0))
    f, gg = g.get_pops()
    f[3, 2, 2, 2] = 1e39 if storage == lbm.LBM_STORAGE_BF16 else 1e6
    g.set_pops(f, gg)
    with pytest.raises(lbm.LBMError) as e:
        g.mass()
    assert e.value.status == lbm.LBM_ENONFINITE


@pytest.mark.parametrize("storage", [0] + STORAGES)
@pytest.mark.parametrize("walls", [0, 7])
def test_repeat_runs_are_bit_identical(storage, walls):
    """Two runs from the same state give the same bits (every thread writes only its own cell of
    the other buffer, so nothing may depend on timing), for every storage, periodic and walled,
    with all forcing terms active."""
    grid = (40, 24, 18)
    phi0 = I.multi_droplet_phi(grid, seed=91, count=3, r_range=(3.0, 5.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=92, amplitude=0.02)
    runs = []
    for _ in range(2):
        g = lbm.Lattice(grid, 19, 0.8, 0.8, 0.02, 4.0, 2e-3, 3.0, 2.0, (2e-5, -1e-5, 1.5e-5), storage=storage,
                        walls=walls)
        g.init_phi(phi0, u0)
        g.step(45)
        runs.append(g.get_pops())
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
