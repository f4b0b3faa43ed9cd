"""Pins of the surrogate oracle (FP64 numpy U-Net): the convolution against
its definition written as plain loops, every backward against central finite
differences, and the pooling / upsampling pair against adjointness."""

import itertools

import numpy as np
import pytest

from oracle import surrogate as S


def _brute_conv(x, w, b, k):
    B, n = x.shape[0], x.shape[1]
    r = k // 2
    taps = list(itertools.product(range(-r, r + 1), repeat=3))
    y = np.zeros((B, n, n, n, w.shape[1]))
    for bb, z, yy, xx, co in itertools.product(range(B), range(n), range(n), range(n), range(w.shape[1])):
        acc = b[co]
        for t, (dz, dy, dx) in enumerate(taps):
            sz, sy, sx = z + dz, yy + dy, xx + dx
            if 0 <= sz < n and 0 <= sy < n and 0 <= sx < n:
                acc += np.dot(x[bb, sz, sy, sx, :], w[t, co, :])
        y[bb, z, yy, xx, co] = acc
    return y


@pytest.mark.parametrize("k", [1, 3])
def test_conv3d_is_the_definition(k):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 4, 4, 3))
    w = rng.normal(size=(k ** 3, 5, 3))
    b = rng.normal(size=5)
    np.testing.assert_allclose(S.conv3d(x, w, b, k), _brute_conv(x, w, b, k), atol=1e-12)


def test_conv3d_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 4, 4, 4, 2))
    w = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=3)
    gy = rng.normal(size=(1, 4, 4, 4, 3))
    f = lambda xx, ww, bb: float(np.sum(S.conv3d(xx, ww, bb, 3) * gy))
    gx, gw, gb = S.conv3d_backward(x, w, gy, 3)
    eps = 1e-6
    for arr, g in ((x, gx), (w, gw), (b, gb)):
        for idx in list(np.ndindex(arr.shape))[::7]:
            old = arr[idx]
            arr[idx] = old + eps
            fp = f(x, w, b)
            arr[idx] = old - eps
            fm = f(x, w, b)
            arr[idx] = old
            assert abs((fp - fm) / (2 * eps) - g[idx]) < 1e-6


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 4, 4, 4, 3))
    y = rng.normal(size=(2, 2, 2, 2, 3))
    assert abs(np.sum(S.avgpool2(x) * y) - np.sum(x * S.avgpool2_backward(y))) < 1e-12
    assert abs(np.sum(S.up2(y) * x) - np.sum(y * S.up2_backward(x))) < 1e-12
    np.testing.assert_allclose(S.avgpool2(S.up2(y)), y, atol=1e-15)


def test_features_definition():
    f = S.features([1e3, 1e6], [1, 3], 8)
    assert f.shape == (2, 8, 8, 8, 8)
    assert np.allclose(f[0, ..., 0], -1.0) and np.allclose(f[1, ..., 0], 1.0)
    assert np.all(f[0, ..., 1] == 1) and np.all(f[0, ..., 2:4] == 0)
    assert np.all(f[1, ..., 3] == 1)
    # x runs along the last spatial axis, z along the first; 1/2 - Y along y
    assert f[0, 0, 0, 0, 4] == pytest.approx(-7 / 8) and f[0, 0, 0, 7, 4] == pytest.approx(7 / 8)
    assert f[0, 7, 0, 0, 6] == pytest.approx(7 / 8)
    assert f[0, 0, 0, 0, 7] == pytest.approx(0.5 - 1 / 16)
    assert f[0, 0, 7, 0, 7] == pytest.approx(0.5 - 15 / 16)


@pytest.mark.parametrize("depth,channels", [(1, (2, 3)), (2, (2, 2, 3))])
def test_unet_gradient_matches_finite_differences(depth, channels):
    n = 8
    net = S.UNet(n, depth, channels)
    rng = np.random.default_rng(4)
    p = rng.uniform(-0.5, 0.5, size=net.count)
    x = S.features([3e4, 2e5], [2, 1], n)
    t = rng.normal(size=(2, n, n, n, S.OUT))
    loss, g = net.loss_and_grad(p, x, t)
    eps = 1e-6
    idx = rng.choice(net.count, size=40, replace=False)
    for i in idx:
        old = p[i]
        p[i] = old + eps
        lp, _ = net.loss_and_grad(p, x, t)
        p[i] = old - eps
        lm, _ = net.loss_and_grad(p, x, t)
        p[i] = old
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    out, _ = net.forward(p, x)
    assert loss == pytest.approx(float(np.mean((out - t) ** 2)))


def test_parameter_count_of_the_config5_network():
    """c = (16, 32, 64, 128): 3^3-conv weights of the encoder pairs (8-16,
    16-16, 16-32, 32-32, 32-64, 64-64, 64-128, 128-128) and decoder pairs
    (128-64, 64-64, 64-32, 32-32, 32-16, 16-16), the 16-5 head, one bias per
    output channel: about 1.3 M parameters."""
    net = S.UNet(64, 3, (16, 32, 64, 128))
    pairs = [(8, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
             (128, 64), (64, 64), (64, 32), (32, 32), (32, 16), (16, 16)]
    expect = sum(27 * a * b + b for a, b in pairs) + 16 * 5 + 5
    assert net.count == expect == 1317525
