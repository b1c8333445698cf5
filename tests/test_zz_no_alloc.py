"""lbm_mass_noalloc, the mass diagnostic for callers that cannot allocate device memory.

Such a caller might be a solver whose populations already fill the GPU, or code whose device
memory belongs to a framework's pool. It passes its own FP32 populations and a device result
buffer, and the library keeps its partial sums in a static device array instead of memory it
allocates. This file runs last, so a failure here cannot hide one elsewhere, and it also
passes when run on its own in a fresh process.

Each cell's phi is an FP32 sum of 19 (or 9) propagated FP32 values, accumulated in FP64. In
bulk cells every cell rounds the same constants t_i phi the same way, so these errors do not
cancel over the grid: REL_TOL allows a few units of 2^-24 (6e-8) of the sum.
"""
import numpy as np
import pytest

import oracle as O
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu

REL_TOL = 2.5e-7  # about four units of FP32 rounding of each cell's phi
PARAMS = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _noalloc(torch, g_dev, Q, grid, walls, rho_ratio, result):
    stream = torch.cuda.current_stream()
    result.fill_(float("nan"))
    st = lbm.lbm_mass_noalloc(g_dev.data_ptr(), Q, grid, walls, 0.997, rho_ratio, result.data_ptr(),
                              stream.cuda_stream)
    assert st == lbm.LBM_OK
    torch.cuda.synchronize()
    return result.cpu().numpy()


@pytest.mark.parametrize("Q,grid,walls,rho_ratio", [
    (19, (37, 21, 19), 0, 3.0),
    (9, (64, 64, 1), 0, 1.0),
    (19, (26, 22, 18), 7, 3.0),      # walls on every face
    (9, (45, 39, 1), 3, 2.0),        # 2D box
    (19, (16, 300, 19), 4, 1.0),     # several rows per block, trailing blocks of a layer empty
])
def test_noalloc_mass_matches_lbm_mass_twice(Q, grid, walls, rho_ratio):
    torch = pytest.importorskip("torch")
    phi0 = I.multi_droplet_phi(grid, seed=61, count=3, r_range=(3.0, 8.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=62, amplitude=0.02)
    if Q == 9:
        u0[2] = 0
    with lbm.Lattice(grid, Q, rho_ratio=rho_ratio, walls=walls, **PARAMS) as h:
        h.init_phi(phi0, u0)
        h.step(25)
        want = h.mass()
        _, g = h.get_pops()
    g_dev = torch.tensor(g, dtype=torch.float32, device="cuda")
    result = torch.empty(3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        got = _noalloc(torch, g_dev, Q, grid, walls, rho_ratio, result)
        assert got[0] == pytest.approx(want[0], rel=REL_TOL)
        assert got[1] == pytest.approx(want[1], rel=REL_TOL)
        assert got[2] == 0.0


@pytest.mark.parametrize("Q,grid,walls", [
    (19, (37, 21, 19), 0), (19, (26, 22, 18), 7), (9, (45, 39, 1), 3), (19, (3, 3, 2048), 0),
])
def test_noalloc_mass_matches_the_oracle(Q, grid, walls):
    """The oracle's own FP64 state after 40 steps, rounded to FP32 and passed in: the sums
    agree with oracle.mass() on that state. The 3 x 3 x 2048 grid is the deepest one the static
    scratch allows (one block per z-layer)."""
    torch = pytest.importorskip("torch")
    rho_ratio = 3.0
    if grid[0] == 3:
        phi0 = I.sine_phi(grid, 0.5, 0.4, axis=2, k=7)
        u0 = None
    else:
        phi0 = I.multi_droplet_phi(grid, seed=63, count=3, r_range=(3.0, 7.0), xi=4.0)
        u0 = I.smooth_velocity(grid, seed=64, amplitude=0.02)
        if Q == 9:
            u0[2] = 0
    ref = O.Oracle(Q, grid, rho_ratio=rho_ratio, walls=walls, **PARAMS)
    ref.init_phi(phi0, u0)
    ref.step(40)
    want = ref.mass()
    _, g = ref.get_pops()
    ref.close()
    g_dev = torch.tensor(g, dtype=torch.float32, device="cuda")
    result = torch.empty(3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        got = _noalloc(torch, g_dev, Q, grid, walls, rho_ratio, result)
        assert got[0] == pytest.approx(want[0], rel=REL_TOL)
        assert got[1] == pytest.approx(want[1], rel=REL_TOL)
        assert got[2] == 0.0


def test_noalloc_mass_counts_nonfinite_values():
    torch = pytest.importorskip("torch")
    grid = (12, 10, 8)
    _, _, t = O.lattice(19)
    g = np.broadcast_to(t[:, None, None, None], (19, 8, 10, 12)).copy()
    g[5, 3, 4, 5] = np.nan
    g[11, 7, 9, 11] = np.inf
    g_dev = torch.tensor(g, dtype=torch.float32, device="cuda")
    result = torch.empty(3, dtype=torch.float64, device="cuda")
    got = _noalloc(torch, g_dev, 19, grid, 0, 1.0, result)
    assert got[2] == 2.0


def test_noalloc_mass_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    g_dev = torch.zeros(19 * 27, dtype=torch.float32, device="cuda")
    result = torch.zeros(3, dtype=torch.float64, device="cuda")
    args = (g_dev.data_ptr(), 19)
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 2049), 0, 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 2), 0, 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 3), 0, 0.0, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 3), 8, 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(*args, (3, 3, 3), -1, 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(g_dev.data_ptr(), 9, (3, 3, 1), 4, 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
    assert lbm.lbm_mass_noalloc(0, 19, (3, 3, 3), 0, 0.997, 1.0, result.data_ptr()) == lbm.LBM_EINVAL
