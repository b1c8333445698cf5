"""lbm_mass_noalloc, the mass diagnostic for callers that cannot allocate device memory.

Such a caller might be a solver whose populations already fill the GPU, or code whose device
memory belongs to a framework's pool. It passes its own FP32 populations and a device result
buffer, and the library keeps its partial sums in a static device array instead of memory it
allocates. This file runs last, so a failure here cannot hide one elsewhere, and it also
passes when run on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu

REL_TOL = 1e-7  # the relative tolerance the parity tests use for sums of phi


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


@pytest.mark.parametrize("Q,grid,rho_ratio", [(19, (37, 21, 19), 3.0), (9, (64, 64, 1), 1.0)])
def test_noalloc_mass_matches_lbm_mass_twice(Q, grid, rho_ratio):
    torch = pytest.importorskip("torch")
    phi0 = I.multi_droplet_phi(grid, seed=61, count=3, r_range=(3.0, 8.0), xi=4.0)
    with lbm.Lattice(grid, Q, 0.8, 0.8, 0.02, 4.0, 1e-3, rho_ratio=rho_ratio) as h:
        h.init_phi(phi0)
        h.step(25)
        want = h.mass()
        _, g = h.get_pops()
    g_dev = torch.tensor(g, dtype=torch.float32, device="cuda")
    result = torch.empty(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        result.fill_(float("nan"))
        st = lbm.lbm_mass_noalloc(g_dev.data_ptr(), Q, grid, 0.997, rho_ratio, result.data_ptr(), stream.cuda_stream)
        assert st == lbm.LBM_OK
        torch.cuda.synchronize()
        got = result.cpu().numpy()
        assert got[0] == pytest.approx(want[0], rel=REL_TOL)
        assert got[1] == pytest.approx(want[1], rel=REL_TOL)
        assert got[2] == 0.0


def test_noalloc_mass_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    g_dev = torch.zeros(19 * 27, dtype=torch.float32, device="cuda")
    result = torch.zeros(3, dtype=torch.float64, device="cuda")
    args = (g_dev.data_ptr(), 19)
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 2049), 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 2), 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 3), 0.0, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(0, 19, (3, 3, 3), 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
