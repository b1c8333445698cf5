"""The divergence-free projection of a periodic velocity (lbm_project_solenoidal) against the FP64
oracle (oracle/projection.py), called through the C ABI.

Tolerance: every pass is a direct DFT sum of n <= 512 FP32 products with FP32 accumulation; over
the six passes the rounding stays near sqrt(n) * 6e-8 relative per pass for these random fields
(about 1e-6 of max |u| at 64^3). The bound is 1e-5 of max |u|, element by element, and the same
for the divergence of the result.
"""
import numpy as np
import pytest
import torch

from oracle import projection as PR
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _project(u, grid):
    """u: host FP64 [3][nz][ny][nx]; returns the CUDA projection as FP64."""
    d = torch.tensor(u, dtype=torch.float32, device="cuda").contiguous()
    nb = lbm.lbm_project_workspace_bytes(grid)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    assert lbm.lbm_project_solenoidal(d.data_ptr(), grid, work.data_ptr(), nb, s.cuda_stream) == lbm.LBM_OK
    s.synchronize()
    return d.double().cpu().numpy()


def _field(grid, seed, smooth=False):
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(3, nz, ny, nx))
    if smooth:  # a coarse velocity-like field: a few long waves plus 10% noise
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        for a in range(3):
            kx, ky, kz = rng.integers(0, 3, size=3)
            u[a] = 0.1 * u[a] + np.sin(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + rng.uniform(0, 6))
        u *= 0.04
    return u


@pytest.mark.parametrize("grid,smooth", [((64, 64, 64), True), ((64, 64, 64), False), ((12, 10, 6), False),
                                         ((9, 7, 5), False), ((8, 8, 1), True), ((40, 24, 3), False),
                                         ((512, 2, 3), False), ((1, 1, 1), False), ((2, 1, 6), False)])
def test_projection_matches_oracle(grid, smooth):
    u = _field(grid, 11, smooth)
    got = _project(u, grid)
    ref = PR.project_solenoidal(u.astype(np.float32).astype(np.float64))
    scale = np.abs(u).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=TOL * scale)
    assert np.abs(PR.divergence(got)).max() <= TOL * scale


def test_projection_is_deterministic_and_keeps_solenoidal_fields():
    grid = (32, 24, 16)
    u = _field(grid, 12, True)
    a, b = _project(u, grid), _project(u, grid)
    np.testing.assert_array_equal(a, b)
    # projecting the result again changes it by rounding only
    np.testing.assert_allclose(_project(a, grid), a, rtol=0, atol=TOL * np.abs(u).max())


def test_invalid_arguments_launch_nothing():
    grid = (8, 8, 8)
    nb = lbm.lbm_project_workspace_bytes(grid)
    u = torch.zeros((3, 8, 8, 8), device="cuda")
    work = torch.empty(nb + 16, dtype=torch.uint8, device="cuda")
    sentinel = u.clone()
    assert lbm.lbm_project_solenoidal(u.data_ptr(), grid, work.data_ptr(), nb - 1, None) == lbm.LBM_EINVAL
    assert lbm.lbm_project_solenoidal(u.data_ptr(), grid, work.data_ptr() + 8, nb, None) == lbm.LBM_EINVAL
    assert lbm.lbm_project_solenoidal(u.data_ptr(), (8, 8, 513), work.data_ptr(), nb, None) == lbm.LBM_EINVAL
    assert lbm.lbm_project_solenoidal(u.data_ptr() + 2, grid, work.data_ptr(), nb, None) == lbm.LBM_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(u, sentinel)
