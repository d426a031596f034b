"""Pins of the FP64 network reference (oracle/unet.py), CPU only.

* The forward convolution equals scipy's 2-D cross-correlation with zero
  padding ('same'), summed over input channels, plus the bias.
* Every adjoint (convolution, ReLU, pooling, upsampling, concatenation, the
  mean squared error) is pinned at once by central finite differences of the
  loss in the parameters on a small network: a dropped term, a wrong index or
  a transposed weight in any backward step changes some partial derivative.
* Pooling and upsampling satisfy <A x, y> = <x, A^T y> with their adjoints.
"""
import numpy as np
import pytest

from oracle import unet as U


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 9, 3))
    for K in (1, 3):
        w = rng.standard_normal((K, K, 3, 4))
        b = rng.standard_normal(4)
        y = U.conv(x, w, b)
        for n in range(2):
            for o in range(4):
                ref = b[o] + sum(signal.correlate2d(x[n, :, :, i], w[:, :, i, o], mode="same", boundary="fill") for i in range(3))
                assert np.allclose(y[n, :, :, o], ref, rtol=1e-13, atol=1e-13)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 8, 6, 3))
    y = rng.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.vdot(U.pool(x), y), np.vdot(x, U.pool_back(y)), rtol=1e-13)
    z = rng.standard_normal((2, 16, 12, 3))
    assert np.isclose(np.vdot(U.up(x), z), np.vdot(x, U.up_back(z)), rtol=1e-13)
    # pooling a constant keeps it, upsampling copies
    assert np.allclose(U.pool(np.ones((1, 4, 4, 1))), 1.0)
    assert np.array_equal(U.up(x)[:, ::2, ::2], x)


def test_parameter_count_and_layout():
    # levels 4, base 32: encoder (3>32, 32>32, 32>64, 64>64, 64>128, 128>128, 128>256, 256>256),
    # decoder per level (up 2c>c, first 2c>c, second c>c), output 1x1 32>2
    c = [32, 64, 128, 256]
    enc = [(3, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256)]
    dec = [(c[l + 1], c[l]) for l in (2, 1, 0) for _ in (0,)]
    n = sum(9 * i * o + o for i, o in enc)
    for l in (2, 1, 0):
        n += 9 * c[l + 1] * c[l] + c[l] + 9 * 2 * c[l] * c[l] + c[l] + 9 * c[l] * c[l] + c[l]
    n += 32 * 2 + 2
    assert U.num_params(4, 32) == n
    assert len(dec) == 3
    theta = np.arange(U.num_params(2, 2), dtype=float)
    P = U.unpack(theta, 2, 2)
    assert P[0][0].shape == (3, 3, 3, 2) and P[0][0][0, 0, 0, 1] == 1.0 and P[0][1][0] == 54.0
    assert P[-1][0].shape == (1, 1, 2, 2)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_gradient_matches_finite_differences(levels):
    base = 2
    rng = np.random.default_rng(10 + levels)
    theta = U.init(levels, base, seed=levels)
    H = 4 << levels
    x = rng.standard_normal((2, H, H, 3))
    t = rng.standard_normal((2, H, H, 2))
    loss, g = U.loss_and_grad(theta, x, t, levels, base)
    assert np.isfinite(loss) and g.shape == theta.shape
    # every parameter block, a few entries each
    idx = []
    off = 0
    for ci, co, K in U.conv_specs(levels, base):
        nw = K * K * ci * co
        idx += list(rng.choice(nw, size=min(nw, 6), replace=False) + off)
        idx += list(rng.choice(co, size=min(co, 2), replace=False) + off + nw)
        off += nw + co
    h = 1e-6
    for k in idx:
        tp = theta.copy()
        tp[k] += h
        tm = theta.copy()
        tm[k] -= h
        fd = (U.loss_and_grad(tp, x, t, levels, base)[0] - U.loss_and_grad(tm, x, t, levels, base)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * np.abs(g).max() + 1e-9, (k, fd, g[k])
