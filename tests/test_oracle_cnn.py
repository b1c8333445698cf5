"""Pins of the surrogate's FP64 oracle (oracle/cnn.py): the convolution against brute-force
loops over the periodic grid, and every gradient against central finite differences."""
import numpy as np
import pytest

from oracle import cnn


def _brute_conv(h, W, b):
    cin, D, H, Wd = h.shape
    out = np.zeros((W.shape[0], D, H, Wd))
    for o in range(W.shape[0]):
        for z in range(D):
            for y in range(H):
                for x in range(Wd):
                    s = b[o]
                    for c in range(cin):
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    s += W[o, c, dz, dy, dx] * h[c, (z + dz - 1) % D, (y + dy - 1) % H, (x + dx - 1) % Wd]
                    out[o, z, y, x] = s
    return out


def _net(rng, chans, grid):
    weights = []
    for cin, cout in zip(chans[:-1], chans[1:]):
        weights.append((rng.normal(0, 0.3, (cout, cin, 3, 3, 3)), rng.normal(0, 0.1, cout)))
    x = rng.normal(0, 1, (chans[0],) + grid)
    t = x + rng.normal(0, 0.3, x.shape)
    return weights, x, t


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(1)
    h = rng.normal(size=(2, 3, 4, 5))
    W = rng.normal(size=(3, 2, 3, 3, 3))
    b = rng.normal(size=3)
    np.testing.assert_allclose(cnn.conv(h, W, b), _brute_conv(h, W, b), rtol=0, atol=1e-12)


def test_conv_of_a_delta_is_the_flipped_kernel():
    """A unit impulse at the origin returns the kernel, reversed, around it."""
    W = np.arange(27, dtype=float).reshape(1, 1, 3, 3, 3)
    h = np.zeros((1, 5, 5, 5))
    h[0, 0, 0, 0] = 1.0
    out = cnn.conv(h, W, np.zeros(1))
    for dz, dy, dx in cnn.TAPS:
        assert out[0, (1 - dz) % 5, (1 - dy) % 5, (1 - dx) % 5] == W[0, 0, dz, dy, dx]


@pytest.mark.parametrize("chans,cw", [((2, 3, 2), None), ((3, 4, 4, 3), None), ((3, 4, 3), (0.5, 2.0, 7.0))])
def test_gradients_match_finite_differences(chans, cw):
    rng = np.random.default_rng(7)
    grid = (3, 4, 3)
    weights, x, t = _net(rng, chans, grid)
    loss, grads = cnn.loss_and_gradients(x, t, weights, cw)
    eps = 1e-6
    for l, (W, b) in enumerate(weights):
        for idx in [(0, 0, 1, 1, 1), (W.shape[0] - 1, W.shape[1] - 1, 0, 2, 1), (0, W.shape[1] - 1, 2, 0, 0)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in weights]
            Wm = [(w.copy(), bb.copy()) for w, bb in weights]
            Wp[l][0][idx] += eps
            Wm[l][0][idx] -= eps
            fd = (cnn.loss_and_gradients(x, t, Wp, cw)[0] - cnn.loss_and_gradients(x, t, Wm, cw)[0]) / (2 * eps)
            assert grads[l][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        for o in range(b.shape[0]):
            Wp = [(w.copy(), bb.copy()) for w, bb in weights]
            Wm = [(w.copy(), bb.copy()) for w, bb in weights]
            Wp[l][1][o] += eps
            Wm[l][1][o] -= eps
            fd = (cnn.loss_and_gradients(x, t, Wp, cw)[0] - cnn.loss_and_gradients(x, t, Wm, cw)[0]) / (2 * eps)
            assert grads[l][1][o] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_input_gradient_of_conv_is_the_adjoint():
    """<conv(h) - b, g> = <h, conv_backward(h, W, g).gh>: the backward pass is the adjoint."""
    rng = np.random.default_rng(3)
    h = rng.normal(size=(3, 4, 5, 6))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    g = rng.normal(size=(2, 4, 5, 6))
    gh, _, _ = cnn.conv_backward(h, W, g)
    lhs = float((cnn.conv(h, W, np.zeros(2)) * g).sum())
    assert lhs == pytest.approx(float((h * gh).sum()), rel=1e-12)
