"""Host input and output paths of the C ABI.

lbm_moments and lbm_gradients write page-locked host buffers directly from the kernel (one launch
over the grid, no staging copy) and any other host memory through device staging: both must give
the same bits. lbm_init_fields checks and stages phi0 and p once when one slab holds the whole
grid: the state must not depend on whether the inputs sit in page-locked memory.
"""
import numpy as np
import pytest
import torch

from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def _pinned(shape):
    n = int(np.prod(shape))
    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy().reshape(shape)


@pytest.mark.parametrize("scheme,walls,storage", [(0, 0, 0), (1, 7, 0), (0, 4, 1)])
def test_pinned_and_pageable_outputs_are_the_same_bits(scheme, walls, storage):
    grid = (36, 20, 14)
    phi0 = I.multi_droplet_phi(grid, seed=81, count=2, r_range=(3.0, 5.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=82, amplitude=0.02)
    g = lbm.Lattice(grid, 19, 0.8, 0.8, 0.02, 4.0, 2e-3, 2.0, 1.5, (1e-5, 0.0, -1e-5), scheme=scheme,
                    storage=storage, walls=walls)
    g.init_phi(phi0, u0)
    g.step(7)
    shape = g.shape
    page = [np.empty(shape), np.empty(shape), np.empty((3,) + shape)]
    pin = [_pinned(shape), _pinned(shape), _pinned((3,) + shape)]
    lbm.lbm_moments(g.h, *page)
    lbm.lbm_moments(g.h, *pin)
    for a, b in zip(page, pin):
        np.testing.assert_array_equal(a, b)
    # subsets of the fields, pinned and pageable mixed (the staged path) and pinned alone
    only_u = _pinned((3,) + shape)
    lbm.lbm_moments(g.h, None, None, only_u)
    np.testing.assert_array_equal(only_u, page[2])
    mixed_phi, mixed_p = _pinned(shape), np.empty(shape)
    lbm.lbm_moments(g.h, mixed_phi, mixed_p, None)
    np.testing.assert_array_equal(mixed_phi, page[0])
    np.testing.assert_array_equal(mixed_p, page[1])
    gp, npg = np.empty((3,) + shape), np.empty((3,) + shape)
    gq, nq = _pinned((3,) + shape), _pinned((3,) + shape)
    lbm.lbm_gradients(g.h, gp, npg)
    lbm.lbm_gradients(g.h, gq, nq)
    np.testing.assert_array_equal(gp, gq)
    np.testing.assert_array_equal(npg, nq)


@pytest.mark.parametrize("walls", [0, 4])
def test_init_from_pinned_and_pageable_inputs_is_the_same_state(walls):
    grid = (24, 16, 20)
    phi0 = I.multi_droplet_phi(grid, seed=83, count=2, r_range=(3.0, 5.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=84, amplitude=0.02)
    p = 1.0 / 3.0 + 1e-4 * I.smooth_velocity(grid, seed=85, amplitude=1.0)[0]
    states = []
    for pinned in (False, True):
        args = [phi0, u0, p]
        if pinned:
            args = [_pinned(a.shape) for a in args]
            for dst, src in zip(args, (phi0, u0, p)):
                dst[...] = src
        g = lbm.Lattice(grid, 19, 0.8, 0.8, 0.02, 4.0, 2e-3, walls=walls)
        g.init_phi(args[0], args[1], p=args[2])
        states.append(g.get_pops())
    np.testing.assert_array_equal(states[0][0], states[1][0])
    np.testing.assert_array_equal(states[0][1], states[1][1])
