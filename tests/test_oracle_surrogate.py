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


# ------------------------------------------------------------------ warm-start mapping

def test_cell_centre_positions_by_hand():
    """Output centre k of an N-cell axis sits at (k + 1/2) m / N - 1/2 input
    cells; the values below are worked out by hand for m = 4."""
    np.testing.assert_allclose(S.source_positions(6, 4), [0.0, 0.5, 7 / 6, 11 / 6, 2.5, 3.0], atol=1e-15)
    np.testing.assert_allclose(S.source_positions(8, 4), [0.0, 0.25, 0.75, 1.25, 1.75, 2.25, 2.75, 3.0],
                               atol=1e-15)
    np.testing.assert_allclose(S.source_positions(2, 4), [0.5, 2.5], atol=1e-15)
    np.testing.assert_allclose(S.source_positions(5, 5), np.arange(5.0), atol=1e-15)


@pytest.mark.parametrize("m,N", [(4, 6), (4, 8), (6, 4), (5, 5), (3, 7)])
def test_trilinear_reproduces_linear_fields(m, N):
    """Linear interpolation reproduces a linear function, so a field linear in
    the input index coordinates comes out as the same function of the output
    cells' (clamped) source positions: exactly, everywhere, each axis with
    its own slope so that a swapped axis fails."""
    a, bx, by, bz = 0.3, 1.25, -0.5, 2.0
    i = np.arange(m, dtype=float)
    lin = a + bx * i[None, None, :] + by * i[None, :, None] + bz * i[:, None, None]
    pred = np.stack([lin, -2.0 * lin], axis=-1)
    p = S.source_positions(N, m)
    want = a + bx * p[None, None, :] + by * p[None, :, None] + bz * p[:, None, None]
    out = S.trilinear(pred, N)
    np.testing.assert_allclose(out[..., 0], want, atol=1e-12)
    np.testing.assert_allclose(out[..., 1], -2.0 * want, atol=1e-12)


def test_trilinear_of_a_separable_field_is_the_product_of_1d_interpolations():
    """For f = g(x) h(y) k(z) the tensor-product interpolation equals the
    product of the three 1-D linear interpolations (numpy.interp, which
    clamps at the ends like the resampling)."""
    rng = np.random.default_rng(7)
    m, N = 5, 9
    gx, hy, kz = rng.normal(size=m), rng.normal(size=m), rng.normal(size=m)
    f = kz[:, None, None] * hy[None, :, None] * gx[None, None, :]
    q = (np.arange(N) + 0.5) * m / N - 0.5
    i = np.arange(m)
    want = (np.interp(q, i, kz)[:, None, None] * np.interp(q, i, hy)[None, :, None]
            * np.interp(q, i, gx)[None, None, :])
    np.testing.assert_allclose(S.trilinear(f[..., None], N)[..., 0], want, atol=1e-12)


def test_identity_grid_and_channel_mapping():
    """N = m returns the input; the channels map to (u_x, u_y, u_z)/u_c, theta
    and (rho - 1)/(3 u_c^2)."""
    rng = np.random.default_rng(8)
    m, uc = 4, 0.05
    pred = rng.normal(size=(m, m, m, 5))
    np.testing.assert_allclose(S.trilinear(pred, m), pred, atol=1e-15)
    rho, u, th = S.warm_start_fields(pred.reshape(-1, 5), m, uc)
    np.testing.assert_allclose(u[0], uc * pred[..., 0], atol=1e-15)
    np.testing.assert_allclose(u[1], uc * pred[..., 1], atol=1e-15)
    np.testing.assert_allclose(u[2], uc * pred[..., 2], atol=1e-15)
    np.testing.assert_allclose(th, pred[..., 3], atol=1e-15)
    np.testing.assert_allclose(rho, 1.0 + 3 * uc * uc * pred[..., 4], atol=1e-15)
