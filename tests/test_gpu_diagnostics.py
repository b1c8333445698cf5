"""Device diagnostics (lbm_diagnostics): the largest |u| and its cell, the kinetic energy and
the mean pressure inside and outside a sphere.

Against the same definitions (oracle/diagnostics.py) evaluated on the host from lbm_moments'
output: the per-cell fields come from the same device code, but inlined into another kernel
the compiler may fuse a multiply-add of the FP32 macroscopic stage differently, so a value can
differ in its last FP32 bit (6e-8 relative). The counts agree exactly (distances from integer
coordinates, FP64, every operation rounded once on both sides); the largest speed, the speed at
the device's cell and the mean pressures agree to 2e-7 relative, the kinetic energy (FP32 per
cell and over runs of 8 cells on the device) to 1e-6. Against the FP64 oracle's own
fields: within the FP32 parity bounds of the fields.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as DG
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


FP32_REL = 2e-7


def _host(g, rho_ratio, centre, r_in, r_out, walls):
    phi, p, u = g.moments()
    d = DG.diagnostics(phi, p, u, rho_ratio, centre, r_in, r_out, walls)
    d["speed"] = np.sqrt(((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]).reshape(-1))
    return d


def _same(dev, host):
    assert dev["max_speed"] == pytest.approx(host["max_speed"], rel=FP32_REL)
    assert host["speed"][dev["argmax"]] == pytest.approx(host["max_speed"], rel=FP32_REL)
    assert dev["n_in"] == host["n_in"] and dev["n_out"] == host["n_out"]
    for k in ("kinetic", "p_in", "p_out"):
        if math.isnan(host[k]):
            assert math.isnan(dev[k])
        else:  # the kinetic terms are FP32 per cell and over runs of 8 cells
            assert dev[k] == pytest.approx(host[k], rel=1e-6 if k == "kinetic" else FP32_REL)


CASES = [dict(Q=19, grid=(36, 20, 14), scheme=0, storage=0, walls=0, rho_ratio=1.0),
         dict(Q=19, grid=(24, 18, 22), scheme=1, storage=0, walls=5, rho_ratio=3.0),
         dict(Q=19, grid=(32, 16, 12), scheme=0, storage=lbm.LBM_STORAGE_FP16, walls=2, rho_ratio=2.0),
         dict(Q=19, grid=(20, 20, 20), scheme=0, storage=lbm.LBM_STORAGE_BF16, walls=0, rho_ratio=1.5),
         dict(Q=9, grid=(40, 28, 1), scheme=0, storage=0, walls=1, rho_ratio=2.0)]


@pytest.mark.parametrize("case", CASES)
def test_diagnostics_equal_the_host_reduction_of_the_moments(case):
    grid = case["grid"]
    phi0 = I.multi_droplet_phi(grid, seed=61, count=2, r_range=(3.0, 5.0), xi=3.0)
    u0 = I.smooth_velocity(grid, seed=62, amplitude=0.03)
    if case["Q"] == 9:
        u0[2] = 0.0
    g = lbm.Lattice(grid, case["Q"], 0.8, 0.8, 0.02, 3.0, 2e-3, case["rho_ratio"], 1.5,
                    (1e-5, -2e-5, 0.0), scheme=case["scheme"], storage=case["storage"], walls=case["walls"])
    g.init_phi(phi0, u0)
    g.step(9)
    for centre, r_in, r_out in (((grid[0] / 2, grid[1] / 2, grid[2] / 2), 4.0, 7.0),
                                ((0.0, 1.5, grid[2] - 0.5), 3.5, 5.0),       # across the periodic edges
                                ((2.0, 2.0, 0.0), 0.0, 1e9)):                # no cell inside or outside
        dev = g.diagnostics(centre, r_in, r_out)
        _same(dev, _host(g, case["rho_ratio"], centre, r_in, r_out, case["walls"]))
    again = g.diagnostics((grid[0] / 2, grid[1] / 2, grid[2] / 2), 4.0, 7.0)
    assert again == g.diagnostics((grid[0] / 2, grid[1] / 2, grid[2] / 2), 4.0, 7.0)  # same bits


@pytest.mark.parametrize("scheme", [0, 1])
def test_diagnostics_against_the_oracle(scheme):
    """A droplet in a smooth flow with density ratio 2 and gravity, 40 steps: the device
    diagnostics against the same quantities of the FP64 oracle's fields, within the FP32
    bounds of the fields (|u| and p to 1e-6 absolute; the kinetic energy to 1e-4 relative).
    Where speeds nearly tie the largest may sit in another cell: the oracle's speed at the
    device's cell must then be within the same bound of its maximum."""
    grid = (24, 20, 16)
    params = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=2e-3, rho_ratio=2.0, mu_ratio=1.0,
                  body_force=(0.0, 0.0, -1e-5))
    phi0 = I.droplet_phi(grid, 6.0, 4.0)
    u0 = I.smooth_velocity(grid, seed=63, amplitude=0.02)
    g = lbm.Lattice(grid, 19, scheme=scheme, **params)
    ref = O.Oracle(19, grid, scheme=scheme, **params)
    g.init_phi(phi0, u0)
    ref.init_phi(phi0, u0)
    g.step(40)
    ref.step(40)
    centre = ((grid[0] - 1) / 2, (grid[1] - 1) / 2, (grid[2] - 1) / 2)
    dev = g.diagnostics(centre, 6.0 - 2 * 4.0 + 4.0, 6.0 + 4.0)
    phi, p, u = ref.moments()
    want = DG.diagnostics(phi, p, u, 2.0, centre, 6.0 - 2 * 4.0 + 4.0, 6.0 + 4.0)
    assert dev["n_in"] == want["n_in"] > 0 and dev["n_out"] == want["n_out"] > 0
    assert abs(dev["max_speed"] - want["max_speed"]) <= 1e-6
    speed = np.sqrt((u ** 2).sum(0)).reshape(-1)
    assert want["max_speed"] - speed[dev["argmax"]] <= 2e-6
    assert abs(dev["p_in"] - want["p_in"]) <= 1e-6 and abs(dev["p_out"] - want["p_out"]) <= 1e-6
    assert dev["kinetic"] == pytest.approx(want["kinetic"], rel=1e-4)


def test_full_size_droplet_diagnostics():
    """The 128^3 droplet workload after 100 steps: the device reduction equals the host reduction
    of the moments; the Laplace jump it gives is positive (pressure higher inside)."""
    w = I.WORKLOADS["droplet3d_128"]
    g = lbm.Lattice(w["grid"], 19, w["tau_f"], w["tau_g"], w["M"], w["xi"], w["sigma"])
    g.init_phi(I.droplet_phi(w["grid"], w["R"], w["xi"]))
    g.step(100)
    centre = tuple((n - 1) / 2 for n in w["grid"])
    r_in, r_out = w["R"] - 2 * w["xi"], w["R"] + 2 * w["xi"]
    dev = g.diagnostics(centre, r_in, r_out)
    _same(dev, _host(g, 1.0, centre, r_in, r_out, 0))
    assert dev["p_in"] > dev["p_out"]


def test_invalid_arguments():
    g = lbm.Lattice((8, 8, 8), 19)
    with pytest.raises(lbm.LBMError):
        g.diagnostics((1.0, 1.0, 1.0), 1.0, 2.0)  # no state yet
    g.init_phi(np.full((8, 8, 8), 1.0))
    with pytest.raises(lbm.LBMError):
        g.diagnostics((float("nan"), 1.0, 1.0), 1.0, 2.0)
    with pytest.raises(lbm.LBMError):
        g.diagnostics((1.0, 1.0, 1.0), float("inf"), 2.0)


def test_diagnostics_on_the_256_cube_taylor_green_workload():
    """The 256^3 Taylor-Green breakup workload (FP16 storage) after 50 steps: 64 cells per
    thread of the reduction (8 runs of 8), against the host reduction of the moments."""
    w = I.WORKLOADS["taylor_green_256"]
    grid = w["grid"]
    g = lbm.Lattice(grid, 19, tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"],
                    storage=lbm.LBM_STORAGE_FP16)
    g.init_phi(I.droplet_phi(grid, w["R"], w["xi"]), I.taylor_green_velocity(grid, w["u0"]),
               p=I.taylor_green_pressure(grid, w["u0"]))
    g.step(50)
    centre = tuple((n - 1) / 2 for n in grid)
    dev = g.diagnostics(centre, w["R"] - 2 * w["xi"], w["R"] + 2 * w["xi"])
    _same(dev, _host(g, 1.0, centre, w["R"] - 2 * w["xi"], w["R"] + 2 * w["xi"], 0))
    g.close()
