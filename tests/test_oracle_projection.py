"""Pins of the oracle's divergence-free projection (oracle/projection.py) to what its definition
fixes independently of the Fourier evaluation: the explicit least-squares projection on tiny
grids, zero divergence, idempotence, gradients removed and divergence-free fields kept."""
import numpy as np
import pytest

from oracle import projection as PR

GRIDS = [(4, 3, 5), (6, 4, 2), (5, 5, 1), (3, 7, 4)]  # (nx, ny, nz): odd, even, extent 1 and 2


def _rand(grid, seed):
    nx, ny, nz = grid
    return np.random.default_rng(seed).normal(size=(3, nz, ny, nx))


def _div_matrix(grid):
    """The divergence as an explicit N x 3N matrix, built entry by entry from the central
    difference (no FFT, no roll)."""
    nx, ny, nz = grid
    N = nx * ny * nz
    idx = lambda x, y, z: ((z % nz) * ny + (y % ny)) * nx + (x % nx)
    A = np.zeros((N, 3 * N))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                r = idx(x, y, z)
                for a, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    A[r, a * N + idx(x + dx, y + dy, z + dz)] += 0.5
                    A[r, a * N + idx(x - dx, y - dy, z - dz)] -= 0.5
    return A


@pytest.mark.parametrize("grid", GRIDS)
def test_projection_is_the_least_squares_projection_onto_zero_divergence(grid):
    """P = I - A+ A for the explicit divergence matrix A (the closest field with A u = 0)."""
    A = _div_matrix(grid)
    u = _rand(grid, 1)
    flat = u.reshape(-1)
    # the row space of A from its singular vectors (rank by an explicit threshold); removing the
    # component of u in it leaves the closest field with A u = 0
    _, sv, vt = np.linalg.svd(A)
    rows = vt[:int(np.sum(sv > 1e-9))]
    ref = flat - rows.T @ (rows @ flat)
    assert np.abs(A @ ref).max() < 1e-13
    np.testing.assert_allclose(PR.project_solenoidal(u).reshape(-1), ref, rtol=0, atol=1e-12)
    # the explicit matrix and the rolled divergence agree
    np.testing.assert_allclose(PR.divergence(u).reshape(-1), A @ flat, rtol=0, atol=1e-13)


@pytest.mark.parametrize("grid", GRIDS + [(16, 12, 10)])
def test_projection_properties(grid):
    u = _rand(grid, 2)
    pu = PR.project_solenoidal(u)
    scale = np.abs(u).max()
    assert np.abs(PR.divergence(pu)).max() < 1e-13 * scale
    np.testing.assert_allclose(PR.project_solenoidal(pu), pu, rtol=0, atol=1e-13 * scale)  # idempotent
    # u - P u is orthogonal to P u (orthogonal projection)
    assert abs(np.sum((u - pu) * pu)) < 1e-12 * np.sum(u * u)
    # a discrete gradient is removed entirely; a discrete curl is kept
    q = np.random.default_rng(3).normal(size=u.shape[1:])
    assert np.abs(PR.project_solenoidal(PR.gradient(q))).max() < 1e-13
    psi = _rand(grid, 4)
    g = [PR.gradient(psi[a]) for a in range(3)]  # g[a][b] = D_b psi_a
    curl = np.stack([g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]])
    assert np.abs(PR.divergence(curl)).max() < 1e-13
    np.testing.assert_allclose(PR.project_solenoidal(curl), curl, rtol=0, atol=1e-13)


def test_component_order_and_axes():
    """A shear flow u = u(y) along x has zero divergence and is kept; the compressive flow
    u = sin(2 pi x / n) along x is removed (it is a gradient); the same profile in v along x is a
    shear again and is kept. A swapped component or axis fails one of these."""
    nx, ny, nz = 8, 6, 4
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    shear = np.zeros((3, nz, ny, nx))
    shear[0] = np.broadcast_to(np.sin(2 * np.pi * y / ny), (nz, ny, nx))
    np.testing.assert_allclose(PR.project_solenoidal(shear), shear, rtol=0, atol=1e-14)
    comp = np.zeros((3, nz, ny, nx))
    comp[0] = np.broadcast_to(np.sin(2 * np.pi * x / nx), (nz, ny, nx))
    assert np.abs(PR.project_solenoidal(comp)).max() < 1e-14
    comp_v = np.zeros((3, nz, ny, nx))
    comp_v[1] = comp[0]
    np.testing.assert_allclose(PR.project_solenoidal(comp_v), comp_v, rtol=0, atol=1e-14)
