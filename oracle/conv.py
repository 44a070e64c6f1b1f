"""FP64 3x3 convolution layers of the warm-start network, written plainly.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``).

The network is not in the paper (it is the learned warm start for the
conjugate-gradient reconstruction).  Its layers are 3x3 cross-correlations,
stride 1, zero padding 1, on NHWC tensors:

    y[b, h, w, o] = bias[o] + sum_{dy, dx, i} x[b, h + dy - 1, w + dx - 1, i] * W[o, dy, dx, i]

with x outside the image taken as 0, and the two gradients of that map:

    dx[b, h, w, i] = sum_{dy, dx, o} g[b, h - dy + 1, w - dx + 1, o] * W[o, dy, dx, i]
    dW[o, dy, dx, i] = sum_{b, h, w} g[b, h, w, o] * x[b, h + dy - 1, w + dx - 1, i]
    dbias[o] = sum_{b, h, w} g[b, h, w, o]

Each is the definition summed term by term over the nine taps.  With
dilation d the taps are (dy - 1) d, (dx - 1) d apart and the padding is d.
"""
from __future__ import annotations

import numpy as np


def _pad(x, d=1):
    return np.pad(np.asarray(x, dtype=np.float64), ((0, 0), (d, d), (d, d), (0, 0)))


def conv3x3(x, W, bias=None, d=1):
    """x [B,H,Wd,Ci], W [Co,3,3,Ci], bias [Co] or None -> y [B,H,Wd,Co]."""
    x = np.asarray(x, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    B, H, Wd, _ = x.shape
    xp = _pad(x, d)
    y = np.zeros((B, H, Wd, W.shape[0]))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("bhwi,oi->bhwo", xp[:, dy * d:dy * d + H, dx * d:dx * d + Wd, :], W[:, dy, dx, :])
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)
    return y


def conv3x3_grad_input(g, W, d=1):
    """g [B,H,Wd,Co], W [Co,3,3,Ci] -> dx [B,H,Wd,Ci]."""
    g = np.asarray(g, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    B, H, Wd, _ = g.shape
    gp = _pad(g, d)
    dx = np.zeros((B, H, Wd, W.shape[3]))
    for dy in range(3):
        for ddx in range(3):
            # dx[h, w] += g[h - (dy - 1) d, w - (ddx - 1) d] W[:, dy, ddx, :]
            oy, ox = (2 - dy) * d, (2 - ddx) * d
            dx += np.einsum("bhwo,oi->bhwi", gp[:, oy:oy + H, ox:ox + Wd, :], W[:, dy, ddx, :])
    return dx


def conv3x3_grad_weight(x, g, d=1):
    """x [B,H,Wd,Ci], g [B,H,Wd,Co] -> (dW [Co,3,3,Ci], dbias [Co])."""
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    B, H, Wd, _ = x.shape
    xp = _pad(x, d)
    dW = np.zeros((g.shape[3], 3, 3, x.shape[3]))
    for dy in range(3):
        for dx in range(3):
            dW[:, dy, dx, :] = np.einsum("bhwo,bhwi->oi", g, xp[:, dy * d:dy * d + H, dx * d:dx * d + Wd, :])
    return dW, g.sum(axis=(0, 1, 2))
