"""lbm_create_ext: a handle whose two state buffers belong to the caller (here torch tensors).

The handle keeps its state in them, gives the same bits as a handle that allocated its own
state, and leaves them to the caller at lbm_destroy. Buffers that are too small, misaligned,
overlapping or not device memory are refused.
"""
import numpy as np
import pytest

from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PARAMS = dict(tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3, rho_ratio=3.0, mu_ratio=2.0,
              body_force=(2e-5, -1e-5, 1.5e-5))


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


@pytest.mark.parametrize("storage,walls,scheme", [(0, 0, 0), (1, 4, 0), (2, 7, 0), (0, 0, 1)])
def test_caller_buffers_give_the_same_bits(storage, walls, scheme):
    grid = (24, 20, 16)
    phi0 = I.multi_droplet_phi(grid, seed=71, count=2, r_range=(3.0, 6.0), xi=4.0)
    u0 = I.smooth_velocity(grid, seed=72, amplitude=0.02)
    nbytes = lbm.lbm_state_bytes(19, grid, storage)
    bufs = [torch.full((nbytes,), 0x7F, dtype=torch.uint8, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    kw = dict(storage=storage, walls=walls, scheme=scheme, **PARAMS)
    out = []
    for buffers in (None, (bufs[0].data_ptr(), bufs[1].data_ptr(), nbytes)):
        with lbm.Lattice(grid, 19, buffers=buffers, **kw) as h:
            h.init_phi(phi0, u0)
            h.step(41)
            out.append(h.get_pops() + h.mass())
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]
    # the state lived in the caller's tensors, and they are still the caller's after destroy
    assert all(int((b != 0x7F).sum()) > nbytes // 2 for b in bufs)
    bufs[0].zero_()
    torch.cuda.synchronize()
    assert int(bufs[0].sum()) == 0


def test_invalid_caller_buffers_are_refused():
    grid = (16, 16, 16)
    nbytes = lbm.lbm_state_bytes(19, grid, 0)
    big = torch.empty(2 * nbytes + 64, dtype=torch.uint8, device="cuda")
    p = big.data_ptr()
    host = torch.empty(nbytes, dtype=torch.uint8)
    cases = [
        (p, p + nbytes, nbytes - 8),      # too small for this grid
        (p + 8, p + 8 + nbytes + 16, nbytes),  # not on a 16-byte boundary
        (p, p + nbytes // 2, nbytes),     # overlapping
        (p, p, nbytes),                   # the same buffer twice
        (0, p + nbytes, nbytes),          # NULL
        (host.data_ptr(), p, nbytes),     # host memory
    ]
    for fg0, fg1, size in cases:
        with pytest.raises(lbm.LBMError) as e:
            lbm.Lattice(grid, 19, buffers=(fg0, fg1, size), tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3)
        assert e.value.status == lbm.LBM_EINVAL
    # a valid pair inside the same allocation works
    with lbm.Lattice(grid, 19, buffers=(p, p + nbytes + 16, nbytes), tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0,
                     sigma=1e-3) as h:
        h.init_phi(I.droplet_phi(grid, 4.0, 4.0))
        h.step(3)
        h.mass()
