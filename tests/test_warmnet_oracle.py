"""Pins of the warm-start network's CPU reference (oracle/warmnet_oracle.py).

* periodic 3D cross-correlation = brute-force loops with modular indices, and =
  scipy.ndimage.correlate with mode="wrap" (a library routine);
* pooling and upsampling backward passes are the adjoints of their forward
  passes, pooling a constant field keeps it;
* every analytic gradient (convolution, whole network) = central finite
  differences of the forward pass.
"""
import numpy as np
import pytest

from oracle import warmnet_oracle as W


def test_conv3d_brute_force():
    rng = np.random.default_rng(0)
    B, ci, co, n3, n2, n1 = 2, 2, 3, 3, 4, 5
    x = rng.standard_normal((B, ci, n3, n2, n1))
    w = rng.standard_normal((co, ci, 3, 3, 3))
    b = rng.standard_normal(co)
    y = W.conv3d(x, w, b)
    ref = np.zeros((B, co, n3, n2, n1))
    for bb in range(B):
        for o in range(co):
            for z in range(n3):
                for yy in range(n2):
                    for xx in range(n1):
                        s = b[o]
                        for i in range(ci):
                            for kz in range(3):
                                for ky in range(3):
                                    for kx in range(3):
                                        s += w[o, i, kz, ky, kx] * x[bb, i, (z + kz - 1) % n3, (yy + ky - 1) % n2,
                                                                    (xx + kx - 1) % n1]
                        ref[bb, o, z, yy, xx] = s
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_conv3d_matches_scipy_wrap():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 1, 6, 7, 8))
    w = rng.standard_normal((1, 1, 3, 3, 3))
    y = W.conv3d(x, w)
    ref = nd.correlate(x[0, 0], w[0, 0], mode="wrap")
    np.testing.assert_allclose(y[0, 0], ref, rtol=1e-12, atol=1e-12)
    # 1x1x1 kernels are channel mixing only
    w1 = rng.standard_normal((3, 1, 1, 1, 1))
    np.testing.assert_allclose(W.conv3d(x, w1)[0], w1[:, 0, 0, 0, 0, None, None, None] * x[0, 0], rtol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 4, 6, 8))
    g = rng.standard_normal((2, 3, 2, 3, 4))
    assert np.isclose(np.sum(W.pool2(x) * g), np.sum(x * W.pool2_backward(g)))
    xc = rng.standard_normal((2, 3, 2, 3, 4))
    gf = rng.standard_normal((2, 3, 4, 6, 8))
    assert np.isclose(np.sum(W.up2(xc) * gf), np.sum(xc * W.up2_backward(gf)))
    np.testing.assert_allclose(W.pool2(np.full((1, 1, 4, 4, 4), 2.5)), 2.5)
    np.testing.assert_allclose(W.pool2(W.up2(xc)), xc)


def _fd(f, arr, idx, h=1e-6):
    old = arr[idx]
    arr[idx] = old + h
    fp = f()
    arr[idx] = old - h
    fm = f()
    arr[idx] = old
    return (fp - fm) / (2 * h)


@pytest.mark.parametrize("k", [1, 3])
def test_conv3d_backward_finite_differences(k):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 3, 4, 5))
    w = rng.standard_normal((2, 3, k, k, k))
    b = rng.standard_normal(2)
    gy = rng.standard_normal((2, 2, 3, 4, 5))
    gx, gw, gb = W.conv3d_backward(x, w, gy)
    L = lambda: float(np.sum(gy * W.conv3d(x, w, b)))
    for idx in [(0, 0, 0, 0, 0), (1, 2, 2, 3, 4), (0, 1, 1, 2, 3)]:
        assert np.isclose(gx[idx], _fd(L, x, idx), rtol=1e-6, atol=1e-8)
    for idx in [(0, 0, 0, 0, 0), (1, 2, k - 1, k // 2, k - 1), (0, 1, k // 2, 0, k - 1)]:
        assert np.isclose(gw[idx], _fd(L, w, idx), rtol=1e-6, atol=1e-8)
    assert np.isclose(gb[1], _fd(L, b, (1,)), rtol=1e-6, atol=1e-8)


def test_network_backward_finite_differences():
    rng = np.random.default_rng(4)
    params = W.random_params(seed=5)
    x = rng.standard_normal((1, 2, 8, 8, 8))
    t = rng.standard_normal((1, 6, 8, 8, 8))
    y, acts = W.forward(params, x)
    assert y.shape == (1, 6, 8, 8, 8)
    loss, gy = W.mse(y, t)
    grads = W.backward(params, acts, gy)
    L = lambda: W.mse(W.forward(params, x)[0], t)[0]
    checked = 0
    for name, ci, co, k, _ in W.ARCH:
        w, b = params[name]
        for idx in [(0, 0) + (k // 2,) * 3, (co - 1, ci - 1) + (0, k - 1, k // 2)]:
            fd = _fd(L, w, idx)
            if abs(fd) > 1e-9:   # a ReLU can switch the path off exactly
                assert np.isclose(grads[name][0][idx], fd, rtol=1e-4, atol=1e-9), (name, idx)
                checked += 1
        fd = _fd(L, b, (0,))
        assert np.isclose(grads[name][1][0], fd, rtol=1e-4, atol=1e-9), name
    assert checked >= len(W.ARCH)


def test_parameter_count():
    n = sum(co * ci * k ** 3 + co for _, ci, co, k, _ in W.ARCH)
    assert 280_000 < n < 320_000
