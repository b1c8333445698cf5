"""FP64 definitions of the state diagnostics (lbm_diagnostics): the largest speed and where it
occurs, the kinetic energy, and the mean pressure inside and outside a sphere.

TEST INFRASTRUCTURE, like the rest of this package: only the test suite and the benchmark's
CPU legs use it. The paper reports, for its static droplets, the spurious currents (the largest
|u|, Sec. 3.1 and Table 1) and the pressure jump across the interface against Laplace's law
(Sec. 3.1); these are those quantities written out as plain reductions over the cells of
fields given as arrays [nz][ny][nx] (u as [3][nz][ny][nx]):

* s2 = (u_x^2 + u_y^2) + u_z^2 per cell, each product and sum rounded once (FP64); argmax is
  the cell index (x fastest) of the largest s2, the smallest index on ties, and max_speed the
  square root of that s2;
* kinetic = sum over cells of rho |u|^2 / 2 with rho = 1 + (rho_ratio - 1) phi (the density of
  the one-fluid model, fluid 2 of unit density);
* the distance of a cell centre (integer coordinates) from `centre`: along an axis with walls
  the plain difference, along a periodic axis the minimum image, and an axis of extent 1 (the
  2D lattice's z) left out;
* p_in, p_out: the mean of p over the cells closer than r_in and farther than r_out (NaN when
  no cell qualifies), with their counts n_in, n_out.
"""
from __future__ import annotations

import numpy as np


def distance(grid, centre, walls=0):
    """Distance of every cell centre from `centre` as described above; walls: bit 0 x, 1 y, 2 z."""
    nx, ny, nz = grid
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    d2 = np.zeros((nz, ny, nx))
    for coord, c, n, bit in ((x, centre[0], nx, 1), (y, centre[1], ny, 2), (z, centre[2], nz, 4)):
        if n == 1:
            continue
        dd = np.abs(coord - c)
        if not walls & bit:
            dd = np.mod(dd, n)
            dd = np.minimum(dd, n - dd)
        d2 = d2 + dd * dd
    return np.sqrt(d2)


def diagnostics(phi, p, u, rho_ratio, centre, r_in, r_out, walls=0):
    """The quantities of the module docstring, as a dict."""
    phi = np.asarray(phi, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    nz, ny, nx = phi.shape
    s2 = ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]).reshape(-1)
    k = int(np.argmax(s2))  # the first occurrence of the largest value
    rho = 1.0 + (rho_ratio - 1.0) * phi
    kinetic = float(np.sum(0.5 * rho * ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2])))
    d = distance((nx, ny, nz), centre, walls)
    inside, outside = d < r_in, d > r_out
    n_in, n_out = int(inside.sum()), int(outside.sum())
    return {"max_speed": float(np.sqrt(s2[k])), "argmax": k, "kinetic": kinetic,
            "p_in": float(p[inside].mean()) if n_in else float("nan"),
            "p_out": float(p[outside].mean()) if n_out else float("nan"),
            "n_in": n_in, "n_out": n_out}
