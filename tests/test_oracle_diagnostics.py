"""Pins of the oracle's state diagnostics (oracle/diagnostics.py): a cell-by-cell loop written
separately on tiny grids, and fields whose answers are known in closed form."""
import math

import numpy as np
import pytest

from oracle import diagnostics as DG


def _loop(phi, p, u, rho_ratio, centre, r_in, r_out, walls):
    """The definitions evaluated one cell at a time with Python floats."""
    nz, ny, nx = phi.shape
    best, arg, kin = -1.0, -1, 0.0
    s_in = s_out = 0.0
    n_in = n_out = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                ux, uy, uz = float(u[0, z, y, x]), float(u[1, z, y, x]), float(u[2, z, y, x])
                s2 = (ux * ux + uy * uy) + uz * uz
                if s2 > best:
                    best, arg = s2, (z * ny + y) * nx + x
                rho = 1.0 + (rho_ratio - 1.0) * float(phi[z, y, x])
                kin += 0.5 * rho * ((ux * ux + uy * uy) + uz * uz)
                d2 = 0.0
                for coord, c, n, bit in ((x, centre[0], nx, 1), (y, centre[1], ny, 2), (z, centre[2], nz, 4)):
                    if n == 1:
                        continue
                    dd = abs(coord - c)
                    if not walls & bit:
                        while dd >= n:
                            dd -= n
                        dd = min(dd, n - dd)
                    d2 += dd * dd
                d = math.sqrt(d2)
                if d < r_in:
                    s_in += float(p[z, y, x])
                    n_in += 1
                if d > r_out:
                    s_out += float(p[z, y, x])
                    n_out += 1
    return {"max_speed": math.sqrt(best), "argmax": arg, "kinetic": kin, "p_in": s_in / n_in if n_in else math.nan,
            "p_out": s_out / n_out if n_out else math.nan, "n_in": n_in, "n_out": n_out}


@pytest.mark.parametrize("grid,walls,centre", [((5, 4, 3), 0, (2.0, 1.5, 1.0)), ((6, 5, 4), 5, (0.3, 4.7, 3.9)),
                                               ((7, 6, 1), 0, (6.5, 0.0, 0.0)), ((4, 4, 4), 7, (1.5, 1.5, 1.5))])
def test_diagnostics_match_a_cell_by_cell_loop(grid, walls, centre):
    nx, ny, nz = grid
    rng = np.random.default_rng(7)
    phi = rng.uniform(0, 1, (nz, ny, nx))
    p = rng.normal(1 / 3, 1e-3, (nz, ny, nx))
    u = rng.normal(0, 0.01, (3, nz, ny, nx))
    got = DG.diagnostics(phi, p, u, 3.0, centre, 1.6, 2.1, walls)
    want = _loop(phi, p, u, 3.0, centre, 1.6, 2.1, walls)
    assert got["argmax"] == want["argmax"] and got["max_speed"] == want["max_speed"]
    assert got["n_in"] == want["n_in"] and got["n_out"] == want["n_out"] and got["n_in"] > 0 and got["n_out"] > 0
    for k in ("kinetic", "p_in", "p_out"):
        assert got[k] == pytest.approx(want[k], rel=1e-13)


def test_closed_forms():
    nx = ny = nz = 8
    grid = (nx, ny, nz)
    shape = (nz, ny, nx)
    u = np.zeros((3,) + shape)
    u[0] += 0.02
    u[1] -= 0.01
    phi = np.zeros(shape)
    # uniform flow over fluid 2 (rho = 1): kinetic = N |u|^2 / 2, every speed equal: argmax 0
    d = DG.diagnostics(phi, np.zeros(shape), u, 5.0, (3.5, 3.5, 3.5), 1.0, 2.0)
    assert d["kinetic"] == pytest.approx(nx * ny * nz * 0.5 * (0.02 ** 2 + 0.01 ** 2), rel=1e-14)
    assert d["argmax"] == 0
    # a spike, then a tie at a later index: the first occurrence wins
    u2 = np.zeros((3,) + shape)
    u2[2, 3, 2, 1] = -0.5
    u2[0, 5, 5, 5] = 0.5
    d = DG.diagnostics(phi, np.zeros(shape), u2, 1.0, (3.5, 3.5, 3.5), 1.0, 2.0)
    assert d["max_speed"] == 0.5 and d["argmax"] == (3 * ny + 2) * nx + 1
    # phi = 1 doubles the density at rho_ratio 2
    d1 = DG.diagnostics(np.ones(shape), np.zeros(shape), u, 2.0, (3.5, 3.5, 3.5), 1.0, 2.0)
    assert d1["kinetic"] == pytest.approx(2 * nx * ny * nz * 0.5 * (0.02 ** 2 + 0.01 ** 2), rel=1e-14)
    # p = 1 within radius 2.5 of a centre on the boundary (minimum image), 0 elsewhere
    dist = DG.distance(grid, (0.0, 0.0, 0.0))
    assert dist[0, 0, 7] == 1.0 and dist[7, 7, 7] == pytest.approx(math.sqrt(3.0))
    p = np.where(dist < 2.5, 1.0, 0.0)
    d = DG.diagnostics(phi, p, u, 1.0, (0.0, 0.0, 0.0), 2.0, 3.0)
    assert d["p_in"] == 1.0 and d["p_out"] == 0.0
    # with walls in x the image across x = 0 is not taken
    assert DG.distance(grid, (0.0, 0.0, 0.0), walls=1)[0, 0, 7] == 7.0
    # no cell inside: NaN mean, count 0
    d = DG.diagnostics(phi, p, u, 1.0, (0.5, 0.5, 0.5), 0.1, 100.0)
    assert d["n_in"] == 0 and math.isnan(d["p_in"]) and d["n_out"] == 0 and math.isnan(d["p_out"])
