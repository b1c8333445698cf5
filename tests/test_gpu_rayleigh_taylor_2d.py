"""The 2D Rayleigh-Taylor set-up of Sec. 3.2 on the GPU: an L0 x 4 L0 pool with walls at the
bottom and top and periodic sides, heavy fluid (rho1 / rho2 = 3, At = 0.5) above the interface
y / L0 = 0.1 cos(2 pi x / L0) about the centre line, eta1 / eta2 = 1, U = sqrt(g L0) = 0.04,
t0 = sqrt(2 L0 / g). Re = rho1 U L0 / eta1 = 256 and Ca = eta1 U / sigma = 1 (the values of the
Rayleigh-Taylor workload; at the paper's Re = 2000 the smaller pools would need relaxation times
below 0.01).

The paper compares the peak (x = 0) and trough (x = L0 / 2) interface heights with published
curves; here the pool is resolved three times (L0 = 64, 128, 256) and both heights at
T / t0 = 2 must converge: the change from 128 to 256 at most half that from 64 to 128
(measured: peak 0.486, 0.494, 0.494 L0; trough -0.691, -0.708, -0.713 L0). Both amplitudes grow
from T / t0 = 1 to 2 and sum phi does not change.
"""
import math

import numpy as np
import pytest

from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu

U, RE, CA = 0.04, 256.0, 1.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _tips(L0):
    g = U * U / L0
    eta1 = 3.0 * U * L0 / RE        # rho1 nu1 with rho1 = 3
    grid = (L0, 4 * L0, 1)
    x, y, _ = I.cell_coords(grid)
    mid = (4 * L0 - 1) / 2.0
    yi = mid + 0.1 * L0 * np.cos(2 * np.pi * (x + 0.5) / L0)
    phi0 = 0.5 * (1.0 + np.tanh(2.0 * (y - yi) / 4.0))
    # tau_f is fluid 2's: nu2 = eta2 / rho2 = eta1
    h = lbm.Lattice(grid, 9, tau_f=3.0 * eta1, tau_g=0.8, M=0.02, xi=4.0, sigma=eta1 * U / CA, rho_ratio=3.0,
                    mu_ratio=1.0, body_force=(0.0, -g, 0.0), walls=2)
    h.init_phi(phi0)
    s0 = h.mass()[0]
    t0 = math.sqrt(2 * L0 / g)
    out, done = [], 0
    for T in (1.0, 2.0):
        n = int(round(T * t0))
        h.step(n - done)
        done = n
        phi = h.moments()[0][0]
        peak = I.interface_height(0.5 * (phi[:, 0] + phi[:, L0 - 1])) - mid
        trough = I.interface_height(0.5 * (phi[:, L0 // 2 - 1] + phi[:, L0 // 2])) - mid
        out.append((peak / L0, trough / L0))
    assert h.mass()[0] == s0
    h.close()
    return out


def test_rayleigh_taylor_tips_converge():
    runs = {L0: _tips(L0) for L0 in (64, 128, 256)}
    for L0, ((p1, t1), (p2, t2)) in runs.items():
        assert 0 < p1 < p2 and t2 < t1 < 0, (L0, runs[L0])
    for k in (0, 1):  # peak, trough at T / t0 = 2
        a, b, c = (runs[L][1][k] for L in (64, 128, 256))
        assert abs(c - b) <= 0.5 * abs(b - a), (k, a, b, c)
    assert 0.4 < runs[256][1][0] < 0.6 and -0.8 < runs[256][1][1] < -0.6
