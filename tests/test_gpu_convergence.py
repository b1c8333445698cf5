"""The convergence study of Sec. 3.1 on the GPU: a static 2D droplet of diameter D = L0 / 2 at
Cn = delta / D = 0.06, tau_rho = 0.02 and La = rho sigma D / eta^2 = 1, its phi compared with
the initial tanh profile by the relative L2 error ||phi - phi0||_2 / ||phi0||_2 after 5
diffusive times delta^2 / M (the error is steady by then: at 20 the same to 2%). The paper
reports second-order accuracy for L0 = 100 .. 400; measured here, both schemes: 2.7e-3, 5.5e-4,
1.4e-4, slopes 2.28 and 1.94. The test asks for slopes in [1.7, 2.6] and errors below 5e-3.
"""
import math

import pytest

from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


@pytest.mark.parametrize("scheme", [0, 1])
def test_static_droplet_converges_at_second_order(scheme):
    errs = []
    for L0 in (100, 200, 400):
        D = L0 / 2
        xi = 0.06 * D
        tau_f = 0.02
        eta = tau_f / 3.0          # rho cs^2 tau_rho with rho = 1
        sigma = eta * eta / D      # La = 1
        M = 0.02
        grid = (L0, L0, 1)
        phi0 = I.droplet_phi(grid, D / 2, xi)
        g = lbm.Lattice(grid, 9, tau_f=tau_f, tau_g=0.8, M=M, xi=xi, sigma=sigma, scheme=scheme)
        g.init_phi(phi0)
        steps = int(5.0 * xi * xi / M)
        g.step(steps + steps % 2)
        phi = g.moments()[0]
        g.close()
        errs.append(math.sqrt(float(((phi - phi0) ** 2).sum() / (phi0 ** 2).sum())))
    slopes = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert max(errs) < 5e-3, errs
    assert all(1.7 <= s <= 2.6 for s in slopes), (errs, slopes)
