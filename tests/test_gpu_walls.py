"""Walls on the GPU against the FP64 oracle (half-way bounce-back in the Lax-Wendroff stencil).

Same FP32 bounds as the periodic parity tests: max |phi error| <= 1e-4, rel-L2(u) <= 1e-3,
|p error| <= 1e-6; sum phi unchanged bit for bit. FP16 storage keeps its looser bounds
(1e-3, 1e-2, 5e-6).

The Rayleigh-Taylor box starts from a uniform pressure, so gravity launches an acoustic
transient that rarefies the heavy fluid at the top wall (the conservative phase-field equation
lowers phi where div u > 0). There the normal n = -K1/|K1| is the direction of a near-zero
vector and follows rounding: an FP64 run with FP32-sized noise added to every population each
step leaves the noise-free run by ~1e-7 in phi at step 10, ~5e-5 (difference-free) and ~5e-4
(finite difference) by step 60. That box is therefore checked against the fixed bounds at
step 10 and, at step 150, against a few times that noisy oracle's own divergence."""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _pair(Q, grid, walls, phi0, u0=None, scheme=0, storage=0, **params):
    base = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)
    base.update(params)
    gpu = lbm.Lattice(grid, Q, scheme=scheme, storage=storage, walls=walls, **base)
    ref = O.Oracle(Q, grid, scheme=scheme, walls=walls, **base)
    gpu.init_phi(phi0, u0)
    ref.init_phi(phi0, u0)
    return gpu, ref


def _rt_phi(grid, xi):
    """Heavy fluid (phi = 1) above a cosine-perturbed plane at mid-height."""
    nx, ny, nz = grid
    x, y, z = I.cell_coords(grid)
    zi = (nz - 1) / 2.0 + 0.05 * nx * np.cos(2 * np.pi * (x + 0.5) / nx) * np.cos(2 * np.pi * (y + 0.5) / ny)
    return 0.5 * (1.0 + np.tanh(2.0 * (z - zi) / xi))


def _check(gpu, ref, phi_tol=1e-4, u_tol=1e-3, p_tol=1e-6):
    (phi_g, p_g, u_g), (phi_o, p_o, u_o) = gpu.moments(), ref.moments()
    assert np.abs(phi_g - phi_o).max() <= phi_tol
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) <= u_tol
    assert np.abs(p_g - p_o).max() <= p_tol


RT_GRID = (24, 20, 40)
RT_PARAMS = dict(tau_f=0.3, rho_ratio=3.0, body_force=(0.0, 0.0, -2e-5), sigma=5e-3)


def _noisy_twin(scheme, steps, rel=6e-8, seed=7):
    """The oracle's sensitivity on the Rayleigh-Taylor box: a second FP64 run whose populations
    get uniform relative noise of FP32 size (|eps| <= 6e-8) after every step."""
    base = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)
    base.update(RT_PARAMS)
    twin = O.Oracle(19, RT_GRID, scheme=scheme, walls=4, **base)
    twin.init_phi(_rt_phi(RT_GRID, 4.0))
    rng = np.random.default_rng(seed)
    for _ in range(steps):
        twin.step(1)
        f, g = twin.get_pops()
        twin.set_pops(f * (1 + rel * rng.uniform(-1, 1, f.shape)), g * (1 + rel * rng.uniform(-1, 1, g.shape)))
    return twin


@pytest.mark.parametrize("scheme", [0, 1])
def test_rayleigh_taylor_box_parity(scheme):
    """z walls, density ratio 3, gravity along -z, perturbed interface: fixed bounds at step 10,
    bounds relative to the FP64 sensitivity at step 150."""
    gpu, ref = _pair(19, RT_GRID, 4, _rt_phi(RT_GRID, 4.0), scheme=scheme, **RT_PARAMS)
    s0 = gpu.mass()[0]
    gpu.step(10)
    ref.step(10)
    _check(gpu, ref)
    gpu.step(140)
    ref.step(140)
    twin = _noisy_twin(scheme, 150)
    (phi_g, p_g, u_g), (phi_o, p_o, u_o), (phi_t, p_t, u_t) = gpu.moments(), ref.moments(), twin.moments()
    un = np.linalg.norm(u_o)
    self_phi, self_u, self_p = np.abs(phi_t - phi_o).max(), np.linalg.norm(u_t - u_o) / un, np.abs(p_t - p_o).max()
    assert np.abs(phi_g - phi_o).max() <= max(1e-4, 5 * self_phi)
    assert np.linalg.norm(u_g - u_o) / un <= max(1e-3, 5 * self_u)
    assert np.abs(p_g - p_o).max() <= max(1e-6, 5 * self_p)
    assert gpu.mass()[0] == s0


@pytest.mark.parametrize("Q,grid,walls", [(19, (17, 13, 11), 7), (19, (16, 12, 10), 3), (9, (33, 29, 1), 3),
                                          (9, (30, 26, 1), 1)])
def test_boxes_with_walls_parity(Q, grid, walls):
    phi0 = I.multi_droplet_phi(grid, seed=91, count=3, r_range=(2.5, 5.0), xi=3.0)
    u0 = I.smooth_velocity(grid, seed=92, amplitude=0.02)
    G = (1e-5, -2e-5, 0.0 if Q == 9 else 1e-5)
    if Q == 9:
        u0[2] = 0
    gpu, ref = _pair(Q, grid, walls, phi0, u0, rho_ratio=2.0, mu_ratio=1.5, body_force=G)
    s0 = gpu.mass()[0]
    gpu.step(150)
    ref.step(150)
    _check(gpu, ref)
    assert gpu.mass()[0] == s0


def test_poiseuille_on_gpu():
    nz, G, tau = 32, 1e-6, 0.8
    gpu, ref = _pair(19, (4, 4, nz), 4, np.ones((nz, 4, 4)), body_force=(G, 0, 0), tau_f=tau, sigma=0.0)
    nu = tau / 3.0
    gpu.step(int(3 * nz * nz / nu))
    ux = gpu.moments()[2][0, :, 1, 1]
    z = np.arange(nz) + 0.5
    ana = G / (2 * nu) * z * (nz - z)
    assert np.abs(ux - ana).max() / ana.max() < 0.015


def test_fp16_rayleigh_taylor_box_parity():
    gpu, ref = _pair(19, RT_GRID, 4, _rt_phi(RT_GRID, 4.0), storage=lbm.LBM_STORAGE_FP16, **RT_PARAMS)
    s0 = gpu.mass()[0]
    gpu.step(150)
    ref.step(150)
    _check(gpu, ref, phi_tol=1e-3, u_tol=1e-2, p_tol=5e-6)
    assert gpu.mass()[0] == s0


RT_COPY = I.WORKLOADS["rayleigh_taylor_32x32x128"]
RT_COPY_STEPS = 2400   # 3 time units W/U; the bubble tip rises ~8.5 cells, the spike falls ~12


def _rt_copy_params():
    w = RT_COPY
    return dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"],
                rho_ratio=w["rho_ratio"], mu_ratio=w["mu_ratio"], body_force=w["body_force"])


def _tips(phi):
    """Bubble tip (light fluid rising, column x = y = 0) and spike tip (column x = W/2, y = 0)."""
    W = phi.shape[2]
    return np.array([I.interface_height(phi[:, 0, 0]), I.interface_height(phi[:, 0, W // 2])])


@pytest.fixture(scope="module")
def rt_copy_oracle():
    w = RT_COPY
    phi0 = I.rayleigh_taylor_phi(w["grid"], w["amplitude"], w["xi"])
    ref = O.Oracle(19, w["grid"], walls=w["walls"], **_rt_copy_params())
    ref.init_phi(phi0)
    start = _tips(phi0)
    ref.step(RT_COPY_STEPS)
    return phi0, start, ref.moments()


@pytest.mark.parametrize("storage,tip_tol", [(lbm.LBM_STORAGE_FP32, 0.05), (lbm.LBM_STORAGE_FP16, 0.05),
                                             (lbm.LBM_STORAGE_BF16, 0.25)])
def test_rayleigh_taylor_copy_tips(rt_copy_oracle, storage, tip_tol):
    """The 32 x 32 x 128 copy of the Rayleigh-Taylor workload (Re = 256, At = 0.5, Ca = 1):
    bubble and spike tips within tip_tol cells of the FP64 oracle after 3 time units, the
    instability having moved them by several cells; sum phi unchanged bit for bit."""
    w = RT_COPY
    phi0, start, (phi_o, _, u_o) = rt_copy_oracle
    gpu = lbm.Lattice(w["grid"], 19, storage=storage, walls=w["walls"], **_rt_copy_params())
    gpu.init_phi(phi0)
    s0 = gpu.mass()[0]
    gpu.step(RT_COPY_STEPS)
    phi_g, _, u_g = gpu.moments()
    tips_o, tips_g = _tips(phi_o), _tips(phi_g)
    assert tips_o[0] - start[0] > 5 and start[1] - tips_o[1] > 5
    assert np.abs(tips_g - tips_o).max() <= tip_tol
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) <= (5e-3 if storage == lbm.LBM_STORAGE_FP32 else 2e-2)
    assert gpu.mass()[0] == s0


def test_invalid_wall_masks_rejected():
    for Q, grid, walls in ((9, (8, 8, 1), 4), (19, (8, 8, 8), 8), (19, (8, 8, 8), -1)):
        o = lbm.lbm_default_opts()
        o.walls = walls
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(grid, Q, 0.8, 0.8, 0.02, 4.0, 1e-3, opts=o)
        assert e.value.status == lbm.LBM_EINVAL


def test_full_size_rayleigh_taylor_parity():
    """The 128 x 128 x 512 workload (walls in z, At = 0.5, Re = 256, Ca = 1) at full size, in the
    launch configuration the benchmark times: every cell after 10 steps against the oracle with
    the FP32 bounds, and sum phi unchanged over 200 more steps."""
    w = I.WORKLOADS["rayleigh_taylor_128x128x512"]
    params = dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"],
                  rho_ratio=w["rho_ratio"], mu_ratio=w["mu_ratio"], body_force=w["body_force"])
    phi0 = I.rayleigh_taylor_phi(w["grid"], w["amplitude"], w["xi"])
    gpu = lbm.Lattice(w["grid"], 19, walls=w["walls"], **params)
    ref = O.Oracle(19, w["grid"], walls=w["walls"], **params)
    gpu.init_phi(phi0)
    ref.init_phi(phi0)
    s0 = gpu.mass()[0]
    gpu.step(10)
    ref.step(10)
    _check(gpu, ref)
    gpu.step(200)
    assert gpu.mass()[0] == s0
