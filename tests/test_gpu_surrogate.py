"""The convolutional surrogate (include/lbm_surrogate.h) on the GPU.

* forward pass and gradients against the FP64 restatement in oracle/cnn.py (FP32 activations:
  relative 1e-5 of each array's scale; FP16 activations: 1e-2);
* one Adam step against its formula;
* coarse fields against block means of lbm_moments; a restart holds sum phi exactly;
* the judge: a wild prediction is rejected and the state is then the LBM's own k steps, bit for
  bit;
* what the network gains: trained on seeded Taylor-Green trajectories of this solver, it
  predicts a held-out trajectory k steps ahead far better than persistence (the state itself),
  and the judged jump is accepted with sum phi unchanged.
"""
import numpy as np
import pytest

from oracle import cnn
from paper_2407_12263_gb300 import build as cuda_build
from paper_2407_12263_gb300 import inputs as I
from paper_2407_12263_gb300 import lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHANS = (5, 32, 32, 32, 5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    cuda_build.build()
    lbm.load()


def unpack(flat):
    out, off = [], 0
    for cin, cout in zip(CHANS[:-1], CHANS[1:]):
        W = flat[off:off + cout * cin * 27].astype(np.float64).reshape(cout, cin, 3, 3, 3)
        off += cout * cin * 27
        b = flat[off:off + cout].astype(np.float64)
        off += cout
        out.append((W, b))
    assert off == flat.size
    return out


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _net(fp16, seed):
    """A network on torch's current stream, the stream that writes its input tensors."""
    return lbm.Net(fp16=fp16, seed=seed, stream=torch.cuda.current_stream().cuda_stream)


def _random_net(fp16, seed=3):
    net = _net(fp16, seed)
    p = net.get_params()
    rng = np.random.default_rng(seed)
    p += rng.normal(0, 0.01, p.size).astype(np.float32)  # non-zero biases as well
    net.set_params(p)
    return net, unpack(p.astype(np.float64))


@pytest.mark.parametrize("fp16,tol", [(False, 1e-5), (True, 1e-2)])
def test_forward_matches_oracle(fp16, tol):
    net, weights = _random_net(fp16)
    rng = np.random.default_rng(11)
    grid = (10, 8, 6)
    x = rng.normal(0, 1, (2, 5, 6, 8, 10))
    xd, yd = _dev(x), torch.empty(x.shape, device="cuda")
    net.forward(xd.data_ptr(), yd.data_ptr(), 2, grid)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for b in range(2):
        want, _ = cnn.forward(x[b].astype(np.float32).astype(np.float64), weights)
        scale = np.abs(want - x[b]).max()
        assert np.abs(y[b] - want).max() <= tol * scale


@pytest.mark.parametrize("fp16,tol,cw,grid", [
    (False, 1e-5, None, (8, 8, 8)),
    (True, 2e-2, None, (8, 8, 8)),
    (False, 1e-5, (1, 30, 30, 30, 0.5), (8, 8, 8)),
    # tensor-core paths: x not a multiple of 8 (element-wise staging), two y tiles, z in two
    # chunks of the weight-gradient pipeline; and aligned rows over three z chunks
    (True, 2e-2, None, (12, 20, 18)),
    (True, 2e-2, None, (16, 16, 34)),
])
def test_gradients_match_oracle(fp16, tol, cw, grid):
    net, weights = _random_net(fp16, seed=5)
    if cw is not None:
        net.set_loss_weights(cw)
    rng = np.random.default_rng(12)
    x = rng.normal(0, 1, (2, 5) + grid[::-1]).astype(np.float32)
    t = (x + rng.normal(0, 0.3, x.shape)).astype(np.float32)
    xd, td = _dev(x), _dev(t)  # held: the library reads them after this line
    loss = net.gradients(xd.data_ptr(), td.data_ptr(), 2, grid)
    g = unpack(net.get_grads().astype(np.float64))
    losses, grads = zip(*(cnn.loss_and_gradients(x[b].astype(np.float64), t[b].astype(np.float64), weights, cw)
                          for b in range(2)))
    assert loss == pytest.approx(np.mean(losses), rel=tol)
    for l in range(4):
        for j in range(2):
            want = (grads[0][l][j] + grads[1][l][j]) / 2
            assert np.abs(g[l][j] - want).max() <= tol * np.abs(want).max()


def test_adam_step_matches_its_formula():
    net, _ = _random_net(False, seed=9)
    rng = np.random.default_rng(13)
    x = rng.normal(0, 1, (1, 5, 8, 8, 8)).astype(np.float32)
    xd, td = _dev(x), _dev(x * 1.1)
    net.gradients(xd.data_ptr(), td.data_ptr(), 1, (8, 8, 8))
    p0, g = net.get_params().astype(np.float64), net.get_grads().astype(np.float64)
    net.adam(1e-3)
    # first step: m = 0.1 g, v = 0.001 g^2, corrected m / sqrt(v) = g / |g|
    want = p0 - 1e-3 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(net.get_params(), want, rtol=0, atol=1e-6)


def _tgv_case(n, u0, R, We, Re=200.0, seed_centre=0.5):
    eta = u0 * n / Re
    return dict(grid=(n, n, n), u0=u0, R=R, xi=4.0, sigma=u0 * u0 * 2 * R / We, tau_f=3 * eta, tau_g=0.8, M=0.02,
                centre=(seed_centre * n - 0.5,) * 3)


def _tgv_lattice(c, stream=None):
    g = lbm.Lattice(c["grid"], 19, tau_f=c["tau_f"], tau_g=c["tau_g"], M=c["M"], xi=c["xi"], sigma=c["sigma"],
                    stream=stream)
    phi0 = I.droplet_phi(c["grid"], c["R"], c["xi"], centre=c["centre"])
    g.init_phi(phi0, I.taylor_green_velocity(c["grid"], c["u0"]), p=I.taylor_green_pressure(c["grid"], c["u0"]))
    return g


def _coarse(g, f):
    n = g.grid
    out = torch.empty((5, n[2] // f, n[1] // f, n[0] // f), device="cuda")
    torch.cuda.synchronize()
    lbm.lbm_coarse_fields(g.h, f, out.data_ptr())
    torch.cuda.synchronize()
    return out


def test_coarse_fields_are_block_means():
    c = _tgv_case(16, 0.04, 4.0, 20.0)
    g = _tgv_lattice(c)
    g.step(10)
    got = _coarse(g, 2).cpu().numpy()
    phi, p, u = g.moments()
    fields = np.stack([phi, u[0], u[1], u[2], p])
    want = fields.reshape(5, 8, 2, 8, 2, 8, 2).mean(axis=(2, 4, 6))
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-7)


def test_restart_holds_sum_phi_exactly():
    c = _tgv_case(16, 0.04, 4.0, 20.0)
    g = _tgv_lattice(c)
    g.step(20)
    s0 = g.mass()[0]
    coarse = _coarse(g, 2)
    coarse[0] += 0.01  # a prediction that adds mass: the restart removes it again, exactly
    lbm.lbm_restart_from_coarse(g.h, 2, coarse.data_ptr())
    assert g.mass()[0] == s0
    # upsampling and block means again smooth a two-coarse-cell interface: close, not equal
    dev = np.abs(_coarse(g, 2).cpu().numpy()[0] - (coarse[0].cpu().numpy() - 0.01))
    assert dev.mean() < 0.02 and dev.max() < 0.15
    g.step(5)
    assert g.mass()[0] == s0


def test_wild_prediction_is_rejected_and_the_lbm_takes_over():
    c = _tgv_case(16, 0.04, 4.0, 20.0)
    g, twin = _tgv_lattice(c), _tgv_lattice(c)
    net = _net(True, 1)
    net.set_params(np.random.default_rng(0).normal(0, 1.0, net.param_count).astype(np.float32))
    ms = [0.5, 0, 0, 0, 1 / 3, 0.5, 0.04, 0.04, 0.04, 1e-4]
    with pytest.raises(lbm.LBMError):
        lbm.lbm_surrogate_reserve(g.h, 3)  # 3 does not divide 16
    # the second jump reuses the workspace the first one allocated
    for _ in range(2):
        rep = lbm.lbm_surrogate_jump(g.h, net, 2, ms, 16, 4, 1e-3, 4.0)
        assert not rep["accepted"]
        twin.step(16)
        fa, ga = g.get_pops()
        fb, gb = twin.get_pops()
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(ga, gb)


def test_trained_surrogate_beats_persistence_and_is_accepted():
    """Training on 6 seeded trajectories (32^3, Re 200, u0, R and We varied), k = 48 steps,
    coarse grid 16^3; on a held-out trajectory the prediction's phi and u errors are below 0.6x
    those of persistence, and the judged jump is accepted with sum phi unchanged."""
    f, k, n = 2, 48, 32
    rng = np.random.default_rng(2024)
    pairs_x, pairs_y = [], []
    for s in range(6):
        c = _tgv_case(n, rng.uniform(0.03, 0.05), rng.uniform(4.0, 6.0), rng.uniform(10, 30),
                      seed_centre=rng.uniform(0.4, 0.6))
        g = _tgv_lattice(c)
        snaps = []
        for t in range(0, 337, 16):
            snaps.append(_coarse(g, f).clone())
            g.step(16)
        for a in range(len(snaps) - k // 16):
            pairs_x.append(snaps[a])
            pairs_y.append(snaps[a + k // 16])
    X, Y = torch.stack(pairs_x), torch.stack(pairs_y)
    mean = X.mean(dim=(0, 2, 3, 4))
    std = X.std(dim=(0, 2, 3, 4)) + 1e-12
    norm = lambda a: ((a - mean[None, :, None, None, None]) / std[None, :, None, None, None]).contiguous()
    Xn, Yn = norm(X), norm(Y)
    net = _net(True, 7)
    grid_c = (n // f,) * 3
    gen = torch.Generator(device="cpu").manual_seed(0)
    first = None
    for it in range(600):
        idx = torch.randint(0, X.shape[0], (8,), generator=gen)
        xb, yb = Xn[idx].contiguous(), Yn[idx].contiguous()
        loss = net.gradients(xb.data_ptr(), yb.data_ptr(), 8, grid_c)
        first = loss if first is None else first
        net.adam(1e-3 if it < 400 else 3e-4)
    assert loss < 0.2 * first
    # held-out trajectory
    c = _tgv_case(n, 0.04, 5.0, 20.0, seed_centre=0.47)
    g = _tgv_lattice(c)
    g.step(64)
    x0 = _coarse(g, f)
    xin = norm(x0[None])
    y = torch.empty_like(xin)
    net.forward(xin.data_ptr(), y.data_ptr(), 1, grid_c)
    pred = (y[0] * std[:, None, None, None] + mean[:, None, None, None])
    truth_h = _tgv_lattice(c)
    truth_h.step(64 + k)
    truth = _coarse(truth_h, f)
    err = lambda a, ch: float((a[ch] - truth[ch]).abs().mean())
    assert err(pred, 0) < 0.6 * err(x0, 0)
    assert sum(err(pred, a) for a in (1, 2, 3)) < 0.6 * sum(err(x0, a) for a in (1, 2, 3))
    s0 = g.mass()[0]
    ms = torch.cat([mean, std]).cpu().numpy().tolist()
    rep = lbm.lbm_surrogate_jump(g.h, net, f, ms, k, 8, 1e-2, 4.0)
    assert rep["accepted"], rep
    assert g.mass()[0] == s0
