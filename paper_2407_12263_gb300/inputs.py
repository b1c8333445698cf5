"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This module holds input recipes only (initial order-parameter and velocity fields and the
workload parameter sets); none of the scheme's arithmetic lives here. Arrays are FP64,
shaped (nz, ny, nx) with x fastest; vector fields carry a leading axis of 3.

The static droplet profile is Eq. initial_droplet of arXiv:2407.12263 (Sec. 3.1):
phi = 1/2 [1 + tanh(2 (|z| - D/2) / delta)], so phi = 0 inside the droplet.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0

# Workloads. Lattice units throughout; tau_phi follows from M (M = tau_phi cs^2).
WORKLOADS = {
    # 2D static droplet, D2Q9, 64x64 periodic, R = 16, xi = 4, 5000 steps (FP64 oracle size).
    "droplet2d_64": dict(Q=9, grid=(64, 64, 1), R=16.0, xi=4.0, sigma=1e-3, tau_f=0.8, tau_g=0.8,
                         M=0.02, rho_ratio=1.0, mu_ratio=1.0, body_force=(0.0, 0.0, 0.0), steps=5000),
    # 3D static droplet, D3Q19, 128^3 periodic, R = 24, xi = 4 (the measured workload).
    "droplet3d_128": dict(Q=19, grid=(128, 128, 128), R=24.0, xi=4.0, sigma=1e-3, tau_f=0.8,
                          tau_g=0.8, M=0.02, rho_ratio=1.0, mu_ratio=1.0,
                          body_force=(0.0, 0.0, 0.0), steps=5000),
}


def lattice_parameters(L0, U, Re, rho_ratio=1.0, mu_ratio=1.0, Ca=None, We=None, D=None, Cn=None, xi=4.0,
                       Pe=None, M=0.02, g=(0.0, 0.0, 0.0)):
    """The arguments of lbm_create (lattice units, dx = dt = 1) from the dimensionless groups of
    a two-phase flow with reference length L0 and velocity U (cells, cells per step).

    Fluid 1 (phi = 1) is the reference: rho1 = rho_ratio (fluid 2 has rho2 = 1) and
    eta1 = mu_ratio eta2, with
      Re = rho1 U L0 / eta1                 ->  eta1, and tau_f = eta2 / (rho2 cs^2);
      Ca = eta1 U / sigma, or We = rho1 U^2 D / sigma (D defaults to L0)  ->  sigma;
      Cn = xi / L0 (or xi given)            ->  xi;
      Pe = U L0 / M (or M given)            ->  M, the mobility (M = tau_phi cs^2);
    g is the body force (acceleration) vector. Exactly one of Ca and We must be given."""
    if (Ca is None) == (We is None):
        raise ValueError("give exactly one of Ca and We")
    rho1 = float(rho_ratio)
    eta1 = rho1 * U * L0 / Re
    eta2 = eta1 / mu_ratio
    sigma = eta1 * U / Ca if Ca is not None else rho1 * U * U * (L0 if D is None else D) / We
    return dict(tau_f=eta2 / CS2, tau_g=0.8, M=(U * L0 / Pe) if Pe is not None else M,
                xi=(Cn * L0) if Cn is not None else xi, sigma=sigma, rho_ratio=rho1, mu_ratio=float(mu_ratio),
                body_force=tuple(float(v) for v in g))


def _rayleigh_taylor(grid, Re=256.0, At=0.5, U=0.04, Ca=1.0, xi=4.0, M=0.02, steps=3600):
    """Single-mode Rayleigh-Taylor box (heavy fluid 1 on top, walls in z): lattice parameters
    from the dimensionless groups. Width W = nx, U = sqrt(g W), Re = rho1 U W / eta1,
    At = (rho1 - rho2)/(rho1 + rho2), Ca = eta1 U / sigma, viscosity ratio 1."""
    W = grid[0]
    rho1 = (1.0 + At) / (1.0 - At)          # rho2 = 1
    params = lattice_parameters(W, U, Re, rho_ratio=rho1, Ca=Ca, xi=xi, M=M, g=(0.0, 0.0, -U * U / W))
    return dict(Q=19, grid=grid, **params, walls=4, amplitude=0.05 * W, steps=steps, time_scale=W / U)


def cell_coords(grid):
    """Integer cell-centre coordinates (x, y, z) broadcast to (nz, ny, nx)."""
    nx, ny, nz = grid
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def periodic_distance(grid, centre):
    """Minimum-image distance of every cell centre from `centre` on the periodic grid."""
    nx, ny, nz = grid
    x, y, z = cell_coords(grid)
    d2 = np.zeros_like(x)
    for coord, c, n in ((x, centre[0], nx), (y, centre[1], ny), (z, centre[2], nz)):
        if n == 1:
            continue
        dd = np.abs(coord - c)
        dd = np.minimum(dd, n - dd)
        d2 += dd * dd
    return np.sqrt(d2)


def droplet_phi(grid, radius, xi, centre=None):
    """Static droplet (Eq. initial_droplet): phi = 0 inside, 1 outside, tanh interface of width xi."""
    nx, ny, nz = grid
    if centre is None:
        centre = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0 if nz > 1 else 0.0)
    r = periodic_distance(grid, centre)
    return 0.5 * (1.0 + np.tanh(2.0 * (r - radius) / xi))


def slab_phi(grid, half_width, xi, axis=0, centre=None):
    """Planar slab of phi = 0 between two flat interfaces normal to `axis` (1D tanh profile)."""
    n = grid[axis]
    if centre is None:
        centre = (n - 1) / 2.0
    coords = cell_coords(grid)[axis]
    d = np.abs(coords - centre)
    d = np.minimum(d, n - d)
    return 0.5 * (1.0 + np.tanh(2.0 * (d - half_width) / xi))


# Rayleigh-Taylor: 128 x 128 x 512 with walls in z, At = 0.5 (density ratio 3), Re = 256,
# U = sqrt(g W) = 0.04, cosine perturbation of amplitude 0.05 W; Ca = 1 (the workload gives none:
# at Ca = 0.1 surface tension makes the single mode stable at this Re), and a 32 x 32 x 128 copy
# with the same dimensionless groups.
WORKLOADS["rayleigh_taylor_128x128x512"] = _rayleigh_taylor((128, 128, 512))
WORKLOADS["rayleigh_taylor_32x32x128"] = _rayleigh_taylor((32, 32, 128))


def _taylor_green(n, Re=1000.0, We=20.0, u0=0.04, xi=4.0, M=0.02):
    """Droplet breakup in a Taylor-Green vortex (Sec. 3.4): periodic cube of side L0 = n, droplet
    of radius n/8 at the centre (phi = 0 inside), density and viscosity ratio 1,
    Re = rho0 u0 L0 / eta, We = rho0 u0^2 D / sigma (D = n/4), tau_f = eta / (rho0 cs^2)."""
    R = n / 8.0
    params = lattice_parameters(n, u0, Re, We=We, D=2 * R, xi=xi, M=M)
    return dict(Q=19, grid=(n, n, n), R=R, **params, u0=u0, steps=int(n / u0), time_scale=n / u0)


# Taylor-Green breakup: 256^3, u0 = 0.04, Re = 1000, R = 32, We = 20 (16-bit storage in the
# benchmark), and a 64^3 copy with the same dimensionless groups for the comparison with the
# oracle.
WORKLOADS["taylor_green_256"] = _taylor_green(256)
WORKLOADS["taylor_green_64"] = _taylor_green(64)


def rayleigh_taylor_phi(grid, amplitude, xi):
    """Heavy fluid (phi = 1) above the plane z = (nz - 1)/2 + A cos(2 pi (x + 1/2)/nx) cos(2 pi (y + 1/2)/ny)."""
    nx, ny, nz = grid
    x, y, z = cell_coords(grid)
    zi = (nz - 1) / 2.0 + amplitude * np.cos(2 * np.pi * (x + 0.5) / nx) * np.cos(2 * np.pi * (y + 0.5) / ny)
    return 0.5 * (1.0 + np.tanh(2.0 * (z - zi) / xi))


def interface_height(phi_column):
    """Height where a column of phi (bottom to top, rising from 0 to 1) crosses 1/2."""
    c = np.asarray(phi_column, dtype=np.float64)
    k = int(np.argmax(c >= 0.5))
    if k == 0:
        return float("nan")
    return (k - 1) + (0.5 - c[k - 1]) / (c[k] - c[k - 1])


def droplet_workload_phi(name):
    w = WORKLOADS[name]
    return droplet_phi(w["grid"], w["R"], w["xi"])


def multi_droplet_phi(grid, seed, count, r_range, xi):
    """Seeded union of `count` droplets with radii in r_range (phi = product of the profiles)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid
    phi = np.ones((nz, ny, nx))
    for _ in range(count):
        c = (rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz) if nz > 1 else 0.0)
        phi *= droplet_phi(grid, rng.uniform(*r_range), xi, centre=c)
    return phi


def smooth_velocity(grid, seed, amplitude, modes=3):
    """Seeded smooth periodic velocity field: a few random Fourier modes per component."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid
    x, y, z = cell_coords(grid)
    u = np.zeros((3, nz, ny, nx))
    dims = 3 if nz > 1 else 2
    for a in range(dims):
        for _ in range(modes):
            kx, ky = rng.integers(-2, 3, size=2)
            kz = rng.integers(-2, 3) if nz > 1 else 0
            ph = rng.uniform(0, 2 * np.pi)
            amp = amplitude * rng.uniform(0.3, 1.0) / modes
            u[a] += amp * np.sin(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / max(nz, 1)) + ph)
    return u


def shear_wave(grid, amplitude, axis_u=0, axis_k=1, k=1):
    """u_axis_u = A sin(2 pi k x_axis_k / L): a single decaying shear mode."""
    coords = cell_coords(grid)
    L = grid[axis_k]
    u = np.zeros((3,) + coords[0].shape)
    u[axis_u] = amplitude * np.sin(2 * np.pi * k * coords[axis_k] / L)
    return u


def sine_phi(grid, mean, amplitude, axis=0, k=1):
    coords = cell_coords(grid)
    return mean + amplitude * np.sin(2 * np.pi * k * coords[axis] / grid[axis])


def rising_bubble_cases(n=256, seed=12263, sizes=(32, 48, 64, 96), heights=(1, 2), xi=4.0, M=0.02,
                        U=0.04, U_max=0.1, tau_min=0.01):
    """Seeded batch of independent rising-bubble boxes (D3Q19, walls on every side, gravity along
    -z). Per case: width s from `sizes` and height factor h from `heights` (uniform), grid
    (s, s, h s); bubble radius R = s/8 (D = 2R), centred at (s/2, s/2, 2D) with phi = 0 inside;
    density ratio rho1/rho2 uniform in [2, 10], viscosity ratio eta1/eta2 uniform in [1, 10];
    Eotvos Eo = drho g D^2 / sigma log-uniform in [1, 50] and Morton
    Mo = g eta1^4 drho / (rho1^2 sigma^3) log-uniform in [1e-5, 1e-1]. The velocity scale
    U = sqrt(g D) is 0.04, raised (up to 0.1) where the smaller relaxation time
    3 min(eta1/rho1, eta2/rho2) would fall below tau_min. Returns a list of dicts with the
    lbm_create arguments, plus 'R', 'centre', 'Eo', 'Mo', 'U'."""
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        s = int(rng.choice(sizes))
        h = int(rng.choice(heights))
        rho1 = rng.uniform(2.0, 10.0)
        mu_ratio = rng.uniform(1.0, 10.0)
        Eo = float(np.exp(rng.uniform(np.log(1.0), np.log(50.0))))
        Mo = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-1))))
        R = s / 8.0
        D = 2.0 * R
        drho = rho1 - 1.0

        def groups(u):
            g = u * u / D
            sigma = drho * g * D * D / Eo
            eta1 = (Mo * rho1 * rho1 * sigma ** 3 / (g * drho)) ** 0.25
            return g, sigma, eta1

        g, sigma, eta1 = groups(U)
        u = U
        tau = 3.0 * min(eta1 / rho1, eta1 / mu_ratio)
        if tau < tau_min:  # eta1 grows linearly with U at fixed Eo and Mo
            u = min(U_max, U * tau_min / tau)
            g, sigma, eta1 = groups(u)
        eta2 = eta1 / mu_ratio
        cases.append(dict(grid=(s, s, h * s), lattice=19, tau_f=3.0 * eta2, tau_g=0.8, M=M, xi=xi, sigma=sigma,
                          rho_ratio=rho1, mu_ratio=mu_ratio, body_force=(0.0, 0.0, -g), walls=7,
                          R=R, centre=(s / 2.0 - 0.5, s / 2.0 - 0.5, 2.0 * D), Eo=Eo, Mo=Mo, U=u))
    return cases


def bubble_phi(case):
    """phi = 1 in the liquid, 0 inside the bubble (tanh of width xi), no periodic images."""
    x, y, z = cell_coords(case["grid"])
    c = case["centre"]
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    return 0.5 * (1.0 + np.tanh(2.0 * (r - case["R"]) / case["xi"]))


def taylor_green_velocity(grid, u0):
    """Taylor-Green vortex of the Taylor-Green case (Sec. 3.4) with period = the domain side
    (arguments 2 pi x / n): u = u0 sin X cos Y cos Z, v = -u0 cos X sin Y cos Z, w = 0."""
    x, y, z = cell_coords(grid)
    X, Y, Z = (2 * np.pi * x / grid[0], 2 * np.pi * y / grid[1], 2 * np.pi * z / grid[2])
    u = np.zeros((3,) + x.shape)
    u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    return u


def taylor_green_pressure(grid, u0, p0=CS2, rho0=1.0):
    """Its pressure: p = p0 + rho0 u0^2 / 16 (cos 2X + cos 2Y)(cos 2Z + 2)."""
    x, y, z = cell_coords(grid)
    X, Y, Z = (2 * np.pi * x / grid[0], 2 * np.pi * y / grid[1], 2 * np.pi * z / grid[2])
    return p0 + rho0 * u0 * u0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
