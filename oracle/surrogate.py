"""FP64 numpy oracle of the warm-start surrogate network (forward and backward).

TEST INFRASTRUCTURE ONLY: the reference the CUDA surrogate's outputs and
gradients are checked against.  It shares no code with the CUDA path; it is
written from the network's definition (the U-Net described in include/dmrt.h:
encoder of conv3 + leaky ReLU pairs with 2x2x2 average pooling, decoder of
conv3 at the coarse level, nearest 2x upsampling plus the skip, conv3, and a
1x1x1 head; mean-squared-error loss), with the backward pass derived by hand
and pinned by finite differences in tests/test_oracle_surrogate.py.

Tensors are channels-last (batch, z, y, x, c); a k^3 convolution's weights are
(taps, cout, cin) with taps ordered (dz, dy, dx), dx fastest.

It also holds the warm start's mapping from a prediction to the initial
fields of a cavity (trilinear resampling between cell-centred grids on the
unit cube, then the channel scalings), written from its definition and pinned
in tests/test_oracle_surrogate.py by linear and separable fields and by hand
computed cell-centre positions.
"""

from __future__ import annotations

import numpy as np

SLOPE = 0.1
FEATURES = 8
OUT = 5


def features(ra, wall, n):
    """Per-voxel inputs (batch, n, n, n, 8): (log10 Ra - 4.5)/1.5, one-hot wall
    type (1..3), x, y, z in [-1, 1] at cell centres, and 1/2 - Y."""
    ra = np.atleast_1d(np.asarray(ra, dtype=np.float64))
    wall = np.atleast_1d(np.asarray(wall))
    c = (np.arange(n) + 0.5) / n
    out = np.zeros((len(ra), n, n, n, FEATURES))
    for b in range(len(ra)):
        out[b, ..., 0] = (np.log10(ra[b]) - 4.5) / 1.5
        out[b, ..., wall[b]] = 1.0
        out[b, ..., 4] = (2 * c - 1)[None, None, :]
        out[b, ..., 5] = (2 * c - 1)[None, :, None]
        out[b, ..., 6] = (2 * c - 1)[:, None, None]
        out[b, ..., 7] = (0.5 - c)[None, :, None]
    return out


def _taps(k):
    r = k // 2
    return [(dz, dy, dx) for dz in range(-r, r + 1) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def conv3d(x, w, b, k):
    """y[v, co] = sum over taps and ci of x[v + tap, ci] w[tap, co, ci] + b[co]
    (zero outside the grid)."""
    r = k // 2
    B, n = x.shape[0], x.shape[1]
    xp = np.pad(x, ((0, 0), (r, r), (r, r), (r, r), (0, 0)))
    y = np.zeros((B, n, n, n, w.shape[1]))
    for t, (dz, dy, dx) in enumerate(_taps(k)):
        xs = xp[:, r + dz:r + dz + n, r + dy:r + dy + n, r + dx:r + dx + n, :]
        y += np.einsum("bzyxc,oc->bzyxo", xs, w[t])
    if b is not None:
        y += b
    return y


def conv3d_backward(x, w, gy, k):
    """Gradients of conv3d: (dx, dw, db) for the output gradient gy."""
    r = k // 2
    B, n = x.shape[0], x.shape[1]
    xp = np.pad(x, ((0, 0), (r, r), (r, r), (r, r), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(_taps(k)):
        sl = (slice(None), slice(r + dz, r + dz + n), slice(r + dy, r + dy + n), slice(r + dx, r + dx + n))
        dw[t] = np.einsum("bzyxo,bzyxc->oc", gy, xp[sl])
        dxp[sl] += np.einsum("bzyxo,oc->bzyxc", gy, w[t])
    db = gy.sum(axis=(0, 1, 2, 3))
    return dxp[:, r:r + n, r:r + n, r:r + n, :], dw, db


def leaky(x):
    return np.where(x > 0, x, SLOPE * x)


def leaky_backward(y, gy):
    return np.where(y > 0, gy, SLOPE * gy)


def avgpool2(x):
    B, n, _, _, c = x.shape
    m = n // 2
    return x.reshape(B, m, 2, m, 2, m, 2, c).mean(axis=(2, 4, 6))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_backward(gy):
    B, n, _, _, c = gy.shape
    m = n // 2
    return gy.reshape(B, m, 2, m, 2, m, 2, c).sum(axis=(2, 4, 6))


class UNet:
    """The surrogate network with depth D and channels c_0..c_D."""

    def __init__(self, n, depth, channels):
        self.n, self.depth = n, depth
        self.ch = list(channels)[:depth + 1]
        # layer table: (cin, cout, k, act) in parameter order
        L = [(FEATURES, self.ch[0], 3, True), (self.ch[0], self.ch[0], 3, True)]
        for l in range(1, depth + 1):
            L += [(self.ch[l - 1], self.ch[l], 3, True), (self.ch[l], self.ch[l], 3, True)]
        for l in range(depth - 1, -1, -1):
            L += [(self.ch[l + 1], self.ch[l], 3, True), (self.ch[l], self.ch[l], 3, True)]
        L.append((self.ch[0], OUT, 1, False))
        self.layers = L
        self.offsets = []
        off = 0
        for cin, cout, k, _ in L:
            nw = k ** 3 * cout * cin
            self.offsets.append((off, off + nw))
            off += nw + cout
        self.count = off

    def unpack(self, p):
        out = []
        for (cin, cout, k, _), (wo, bo) in zip(self.layers, self.offsets):
            out.append((p[wo:bo].reshape(k ** 3, cout, cin), p[bo:bo + cout]))
        return out

    def _idx(self, kind, l):
        D = self.depth
        if kind == "a":
            return 2 * l
        if kind == "s":
            return 2 * l + 1
        if kind == "d":
            return 2 * (D + 1) + 2 * (D - 1 - l)
        if kind == "h":
            return 2 * (D + 1) + 2 * (D - 1 - l) + 1
        return len(self.layers) - 1

    def forward(self, p, x):
        P = self.unpack(p)
        D = self.depth
        c = {}

        def conv(kind, l, inp):
            i = self._idx(kind, l)
            w, b = P[i]
            k, act = self.layers[i][2], self.layers[i][3]
            y = conv3d(inp, w, b, k)
            return leaky(y) if act else y

        c["x"] = x
        c["a0"] = conv("a", 0, x)
        c["s0"] = conv("s", 0, c["a0"])
        for l in range(1, D + 1):
            c[f"p{l}"] = avgpool2(c[f"s{l - 1}"])
            c[f"a{l}"] = conv("a", l, c[f"p{l}"])
            c[f"s{l}"] = conv("s", l, c[f"a{l}"])
        c[f"h{D}"] = c[f"s{D}"]
        for l in range(D - 1, -1, -1):
            c[f"d{l}"] = conv("d", l, c[f"h{l + 1}"])
            c[f"m{l}"] = up2(c[f"d{l}"]) + c[f"s{l}"]
            c[f"h{l}"] = conv("h", l, c[f"m{l}"])
        c["out"] = conv("head", 0, c["h0"])
        return c["out"], c

    def loss_and_grad(self, p, x, target):
        """Mean squared error and its gradient with respect to p."""
        out, c = self.forward(p, x)
        P = self.unpack(p)
        D = self.depth
        diff = out - target
        loss = float(np.mean(diff * diff))
        grad = np.zeros_like(p)

        def back(kind, l, inp, outv, gy):
            i = self._idx(kind, l)
            w, _ = P[i]
            k, act = self.layers[i][2], self.layers[i][3]
            if act:
                gy = leaky_backward(outv, gy)
            gx, gw, gb = conv3d_backward(inp, w, gy, k)
            wo, bo = self.offsets[i]
            grad[wo:bo] = gw.ravel()
            grad[bo:bo + self.layers[i][1]] = gb
            return gx

        g = 2.0 * diff / diff.size
        gh = back("head", 0, c["h0"], c["out"], g)
        gs = {}
        for l in range(D):
            gm = back("h", l, c[f"m{l}"], c[f"h{l}"], gh)
            gs[l] = gm
            gd = up2_backward(gm)
            gh = back("d", l, c[f"h{l + 1}"], c[f"d{l}"], gd)
        gs[D] = gh
        for l in range(D, -1, -1):
            ga = back("s", l, c[f"a{l}"], c[f"s{l}"], gs[l])
            inp = c["x"] if l == 0 else c[f"p{l}"]
            gp = back("a", l, inp, c[f"a{l}"], ga)
            if l >= 1:
                gs[l - 1] = gs[l - 1] + avgpool2_backward(gp)
        return loss, grad


# ---------------------------------------------------------------- warm-start mapping

def source_positions(N, m):
    """Where the centres of N output cells fall on an m-cell input axis, in
    input cell units (0 = the first input centre).  Both grids divide the
    same unit interval into equal cells with values at the cell centres:
    output centre (k + 1/2)/N lies (k + 1/2) m / N - 1/2 input cells past the
    first input centre.  Positions outside [0, m - 1] are clamped, i.e. the
    field is held constant beyond the outermost input centres."""
    p = (np.arange(N) + 0.5) * m / N - 0.5
    return np.clip(p, 0.0, m - 1.0)


def _axis_weights(N, m):
    """Lower neighbour index and the weight of the upper one for each of N
    output positions (linear interpolation between input centres)."""
    p = source_positions(N, m)
    if m == 1:
        return np.zeros(N, dtype=int), np.zeros(N, dtype=int), np.zeros(N)
    i0 = np.minimum(np.floor(p).astype(int), m - 2)
    return i0, i0 + 1, p - i0


def trilinear(pred, N):
    """Trilinear resampling of a channels-last field pred (m, m, m, c) to
    (N, N, N, c): each output value is the sum over the 8 surrounding input
    centres of the value times the product of the three 1-D linear weights."""
    pred = np.asarray(pred, dtype=np.float64)
    m = pred.shape[0]
    x0, x1, fx = _axis_weights(N, m)
    y0, y1, fy = _axis_weights(N, m)
    z0, z1, fz = _axis_weights(N, m)
    out = np.zeros((N, N, N, pred.shape[-1]))
    for zi, zw in ((z0, 1.0 - fz), (z1, fz)):
        for yi, yw in ((y0, 1.0 - fy), (y1, fy)):
            for xi, xw in ((x0, 1.0 - fx), (x1, fx)):
                w = zw[:, None, None] * yw[None, :, None] * xw[None, None, :]
                out += w[..., None] * pred[np.ix_(zi, yi, xi)]
    return out


def warm_start_fields(pred, N, uc):
    """Initial fields of an N^3 cavity from one prediction (m^3, 5) or
    (m, m, m, 5) with channels (u_x, u_y, u_z)/u_c, theta and
    (rho - 1)/(3 u_c^2): resampled trilinearly, velocities times u_c, density
    1 + 3 u_c^2 times its channel.  Returns planar (rho (N,N,N),
    u (3,N,N,N), theta (N,N,N)) indexed [z][y][x]."""
    pred = np.asarray(pred, dtype=np.float64)
    m = round(pred.shape[0] ** (1.0 / 3.0)) if pred.ndim == 2 else pred.shape[0]
    pred = pred.reshape(m, m, m, OUT)
    f = trilinear(pred, N)
    u = np.stack([uc * f[..., 0], uc * f[..., 1], uc * f[..., 2]])
    theta = f[..., 3]
    rho = 1.0 + 3.0 * uc * uc * f[..., 4]
    return rho, u, theta
