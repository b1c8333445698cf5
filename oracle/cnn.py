"""FP64 CPU oracle of the 3D convolutional surrogate (plain numpy).

TEST INFRASTRUCTURE, like the rest of this package: only the test suite and the benchmark's
CPU legs use it. The surrogate has no counterpart in the paper; this module restates the
network the CUDA library implements so that its forward pass and its gradients can be checked:

  input x: C0 channels on a periodic grid [C][D][H][W];
  layer l (l = 1..L): a_l = conv(h_{l-1}; W_l, b_l), h_l = relu(a_l) for l < L, h_L = a_L,
      conv(h; W, b)[o, z, y, x] = b[o] + sum_{c, dz, dy, dx} W[o, c, dz, dy, dx] h[c, z+dz-1, y+dy-1, x+dx-1]
      with indices taken modulo the grid (periodic padding), W of shape [Cout][Cin][3][3][3];
  prediction: x + h_L (a residual step);
  loss: mean over every element of w_c (prediction - target)^2, w_c the weight of the element's
  channel (1 unless given).

Everything is FP64; a library routine (numpy roll, tensordot) serves each convolution term.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in range(3) for dy in range(3) for dx in range(3)]


def shifted(h, dz, dy, dx):
    """h[c, z+dz-1, y+dy-1, x+dx-1] with periodic indices, for every (c, z, y, x)."""
    return np.roll(h, shift=(1 - dz, 1 - dy, 1 - dx), axis=(-3, -2, -1))


def conv(h, W, b):
    """Periodic 3x3x3 convolution of h [Cin][D][H][W] with W [Cout][Cin][3][3][3] and b [Cout]."""
    out = np.zeros((W.shape[0],) + h.shape[1:])
    for dz, dy, dx in TAPS:
        out += np.tensordot(W[:, :, dz, dy, dx], shifted(h, dz, dy, dx), axes=(1, 0))
    return out + b[:, None, None, None]


def conv_backward(h, W, gout):
    """Gradients of sum(gout * conv(h; W, b)) with respect to h, W and b."""
    gh = np.zeros_like(h)
    gW = np.zeros_like(W)
    for dz, dy, dx in TAPS:
        sh = shifted(h, dz, dy, dx)
        gW[:, :, dz, dy, dx] = np.tensordot(gout, sh, axes=([1, 2, 3], [1, 2, 3]))
        # the term W[:, :, tap] h[c, z + off] reaches h[c, q] from the output at q - off
        back = np.tensordot(W[:, :, dz, dy, dx], gout, axes=(0, 0))
        gh += np.roll(back, shift=(dz - 1, dy - 1, dx - 1), axis=(-3, -2, -1))
    gb = gout.sum(axis=(1, 2, 3))
    return gh, gW, gb


def forward(x, weights):
    """weights: list of (W, b). Returns the prediction and the per-layer pre-activations."""
    h = x
    pre = []
    for l, (W, b) in enumerate(weights):
        a = conv(h, W, b)
        pre.append(a)
        h = np.maximum(a, 0.0) if l < len(weights) - 1 else a
    return x + h, pre


def loss_and_gradients(x, target, weights, channel_weights=None):
    """Mean-squared loss of the prediction and its gradients [(gW, gb), ...] for one sample."""
    pred, pre = forward(x, weights)
    diff = pred - target
    w = np.ones(x.shape[0]) if channel_weights is None else np.asarray(channel_weights, dtype=np.float64)
    wd = w[:, None, None, None] * diff
    loss = float((wd * diff).mean())
    g = 2.0 * wd / diff.size            # d loss / d h_L (the residual adds x, which has no weights)
    grads = [None] * len(weights)
    for l in range(len(weights) - 1, -1, -1):
        h_in = x if l == 0 else np.maximum(pre[l - 1], 0.0)
        gh, gW, gb = conv_backward(h_in, weights[l][0], g)
        grads[l] = (gW, gb)
        if l > 0:
            g = gh * (pre[l - 1] > 0)
    return loss, grads
