"""CPU reference of the learned warm start's network (test infrastructure only).

ORACLE: imported only by tests/, __graft_entry__.smoke() and bench.py's CPU
legs; it shares no code with the CUDA path.

The paper has no learned component; this module restates, in plain numpy
(float64), the network the library trains on the GPU so that its kernels can
be checked: periodic ("circular") 3D cross-correlations of stride 1,
2x2x2 mean pooling, nearest-neighbour 2x upsampling, ReLU, additive skips, the
mean squared error, and the analytic gradients of all of them.  Pins (tests/
test_warmnet_oracle.py): brute-force loops, scipy.ndimage.correlate with
periodic wrap, adjoint identities, and central finite differences of the
forward pass.

Arrays are [batch][channel][n3][n2][n1]; weights [c_out][c_in][k][k][k].
"""
from __future__ import annotations

import numpy as np

# (name, c_in, c_out, kernel size, grid level) of the U-shaped network, in
# parameter order (each layer: weights then bias).
ARCH = [
    ("enc0", 2, 8, 3, 0),
    ("enc1a", 8, 16, 3, 1),
    ("enc1b", 16, 16, 3, 1),
    ("enc2a", 16, 32, 3, 2),
    ("enc2b", 32, 32, 3, 2),
    ("enc3a", 32, 64, 3, 3),
    ("enc3b", 64, 64, 3, 3),
    ("dec2", 64, 32, 3, 2),
    ("dec1", 32, 16, 3, 1),
    ("dec0", 16, 8, 1, 0),
    ("out", 8, 6, 3, 0),
]


def _taps(k):
    r = k // 2
    return [(dz, dy, dx) for dz in range(-r, r + 1) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def shifted(x, d):
    """x(v + d) on the periodic grid (last three axes z, y, x)."""
    dz, dy, dx = d
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv3d(x, w, b=None, skip=None, relu=False):
    """y[b,o](v) = b[o] + sum_i sum_d w[o,i,d] x[b,i](v + d) (+ skip), then ReLU if asked."""
    k = w.shape[-1]
    y = np.zeros((x.shape[0], w.shape[0]) + x.shape[2:])
    for t, d in enumerate(_taps(k)):
        kz, ky, kx = d[0] + k // 2, d[1] + k // 2, d[2] + k // 2
        y += np.einsum("oi,bi...->bo...", w[:, :, kz, ky, kx], shifted(x, d))
    if b is not None:
        y += b[None, :, None, None, None]
    if skip is not None:
        y += skip
    return np.maximum(y, 0.0) if relu else y


def conv3d_backward(x, w, gy):
    """Gradients of sum(gy * conv3d(x, w, b)) with respect to x, w and b."""
    k = w.shape[-1]
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for d in _taps(k):
        kz, ky, kx = d[0] + k // 2, d[1] + k // 2, d[2] + k // 2
        # x(v + d) feeds y(v): its gradient lands at v + d, i.e. gy(u - d) at u
        gx += np.einsum("oi,bo...->bi...", w[:, :, kz, ky, kx], shifted(gy, (-d[0], -d[1], -d[2])))
        gw[:, :, kz, ky, kx] = np.einsum("bozyx,bizyx->oi", gy, shifted(x, d))
    gb = gy.sum(axis=(0, 2, 3, 4))
    return gx, gw, gb


def pool2(x):
    s = x.shape
    return x.reshape(s[:-3] + (s[-3] // 2, 2, s[-2] // 2, 2, s[-1] // 2, 2)).mean(axis=(-5, -3, -1))


def pool2_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=-3), 2, axis=-2), 2, axis=-1) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=-3), 2, axis=-2), 2, axis=-1)


def up2_backward(g):
    s = g.shape
    return g.reshape(s[:-3] + (s[-3] // 2, 2, s[-2] // 2, 2, s[-1] // 2, 2)).sum(axis=(-5, -3, -1))


def forward(params, x):
    """Network output and the activations needed by `backward`.

    params: dict name -> (w, b).  x: [B][2][n3][n2][n1] (indicator of phase 1,
    log-contrast channel).  Encoder: per level, 3x3x3 conv + ReLU (two at levels
    1-3 after 2x mean pooling).  Decoder: nearest upsampling, conv, add the
    encoder output of the same level, ReLU; output: 3x3x3 conv to 6 channels.
    """
    a = {"x": x}
    c = lambda name, inp, **kw: conv3d(inp, params[name][0], params[name][1], **kw)
    a["e0"] = c("enc0", x, relu=True)
    a["p0"] = pool2(a["e0"])
    a["a1"] = c("enc1a", a["p0"], relu=True)
    a["e1"] = c("enc1b", a["a1"], relu=True)
    a["p1"] = pool2(a["e1"])
    a["a2"] = c("enc2a", a["p1"], relu=True)
    a["e2"] = c("enc2b", a["a2"], relu=True)
    a["p2"] = pool2(a["e2"])
    a["a3"] = c("enc3a", a["p2"], relu=True)
    a["e3"] = c("enc3b", a["a3"], relu=True)
    a["u2"] = up2(a["e3"])
    a["d2"] = c("dec2", a["u2"], skip=a["e2"], relu=True)
    a["u1"] = up2(a["d2"])
    a["d1"] = c("dec1", a["u1"], skip=a["e1"], relu=True)
    a["u0"] = up2(a["d1"])
    a["d0"] = c("dec0", a["u0"], skip=a["e0"], relu=True)
    a["y"] = c("out", a["d0"])
    return a["y"], a


def backward(params, a, gy):
    """Gradients of sum(gy * y) with respect to every (w, b)."""
    g = {}

    def layer(name, inp, gout):
        gx, gw, gb = conv3d_backward(inp, params[name][0], gout)
        g[name] = (gw, gb)
        return gx

    mask = lambda grad, act: grad * (act > 0)
    gd0 = mask(layer("out", a["d0"], gy), a["d0"])
    gu0 = layer("dec0", a["u0"], gd0)
    gd1 = mask(up2_backward(gu0), a["d1"])
    gu1 = layer("dec1", a["u1"], gd1)
    gd2 = mask(up2_backward(gu1), a["d2"])
    gu2 = layer("dec2", a["u2"], gd2)
    ge3 = mask(up2_backward(gu2), a["e3"])
    ga3 = mask(layer("enc3b", a["a3"], ge3), a["a3"])
    gp2 = layer("enc3a", a["p2"], ga3)
    ge2 = mask(gd2 + pool2_backward(gp2), a["e2"])
    ga2 = mask(layer("enc2b", a["a2"], ge2), a["a2"])
    gp1 = layer("enc2a", a["p1"], ga2)
    ge1 = mask(gd1 + pool2_backward(gp1), a["e1"])
    ga1 = mask(layer("enc1b", a["a1"], ge1), a["a1"])
    gp0 = layer("enc1a", a["p0"], ga1)
    ge0 = mask(gd0 + pool2_backward(gp0), a["e0"])
    layer("enc0", a["x"], ge0)
    return g


def mse(y, t):
    """Mean squared error and its gradient."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def random_params(seed=0, scale=1.0):
    """Random weights (He-like scale) for tests."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co, k, _ in ARCH:
        w = rng.standard_normal((co, ci, k, k, k)) * scale * np.sqrt(2.0 / (ci * k ** 3))
        b = rng.standard_normal(co) * 0.1 * scale
        p[name] = (w, b)
    return p
