"""Pins of the oracle's 3x3 convolution layers against scipy's independent
2D correlation, the identity and shift kernels, and the adjoint relations
that define the two gradients (<conv(x), g> = <x, grad_input(g)> and
<conv(x), g> = <W, grad_weight(x, g)>)."""
import numpy as np
from scipy.signal import correlate2d

from oracle.conv import conv3x3, conv3x3_grad_input, conv3x3_grad_weight


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 9, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, i], W[o, :, :, i], mode="same", boundary="fill")
                             for i in range(3))
            assert np.allclose(y[n, :, :, o], ref, atol=1e-12)


def test_identity_and_shift_kernels():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 5, 6, 2))
    W = np.zeros((2, 3, 3, 2))
    W[0, 1, 1, 0] = W[1, 1, 1, 1] = 1.0
    assert np.allclose(conv3x3(x, W), x)
    S = np.zeros((1, 3, 3, 2))
    S[0, 1, 2, 1] = 1.0            # y[h, w] = x[h, w + 1, 1]
    y = conv3x3(x, S)[..., 0]
    assert np.allclose(y[0, :, :-1], x[0, :, 1:, 1])
    assert np.allclose(y[0, :, -1], 0.0)


def test_gradients_are_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 6, 5, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    g = rng.standard_normal((2, 6, 5, 4))
    y = conv3x3(x, W)
    lhs = float((y * g).sum())
    assert abs(lhs - float((x * conv3x3_grad_input(g, W)).sum())) < 1e-10 * abs(lhs)
    dW, db = conv3x3_grad_weight(x, g)
    assert abs(lhs - float((W * dW).sum())) < 1e-10 * abs(lhs)
    assert np.allclose(db, g.sum(axis=(0, 1, 2)))


def test_dilated_conv_is_correlation_with_spread_kernel():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 11, 13, 2))
    W = rng.standard_normal((3, 3, 3, 2))
    for d in (2, 3):
        y = conv3x3(x, W, d=d)
        for o in range(3):
            ref = 0.0
            for i in range(2):
                K = np.zeros((2 * d + 1, 2 * d + 1))
                K[::d, ::d] = W[o, :, :, i]
                ref = ref + correlate2d(x[0, :, :, i], K, mode="same", boundary="fill")
            assert np.allclose(y[0, :, :, o], ref, atol=1e-12)
        g = rng.standard_normal(y.shape)
        lhs = float((y * g).sum())
        assert abs(lhs - float((x * conv3x3_grad_input(g, W, d=d)).sum())) < 1e-10 * abs(lhs)
        assert abs(lhs - float((W * conv3x3_grad_weight(x, g, d=d)[0]).sum())) < 1e-10 * abs(lhs)
