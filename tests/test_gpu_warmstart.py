"""GPU: the learned warm start's kernels and network against the CPU reference,
and what the trained network gains over the solver started from eps_bar.

* every kernel of include/fftls_nn.h against oracle/warmnet_oracle.py (FP32 vs
  FP64: relative 1e-5 on outputs, 1e-4 on reductions);
* the whole network: output and every parameter gradient against the oracle's
  analytic backward (itself pinned by finite differences);
* a short training on solver-generated fields cuts the iterations to
  eta <= 1e-6 on held-out samples, the solver deciding convergence, without
  making the time to tolerance (tensor-core inference included) grow.
"""
import ctypes

import numpy as np
import pytest

from oracle import warmnet_oracle as W
from paper_1412_8398_gb300 import microstructure as MS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_8398_gb300 import build, fftls, warmstart
    build.build()
    return torch, fftls, warmstart, warmstart._lib()


def _dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _close(got, want, rtol):
    scale = max(np.abs(want).max(), 1e-30)
    assert np.abs(got - want).max() <= rtol * scale, (np.abs(got - want).max(), scale)


@pytest.mark.parametrize("k,ci,co,n", [(3, 5, 11, (6, 4, 5)), (1, 16, 8, (8, 8, 8)), (3, 64, 64, (4, 4, 4)),
                                       (3, 2, 8, (1, 3, 2))])
def test_conv3d_forward_and_backward(env, k, ci, co, n):
    torch, fftls, ws, lib = env
    rng = np.random.default_rng(k * 100 + ci)
    B = 2
    shape = (B, ci, n[2], n[1], n[0])
    x = rng.standard_normal(shape)
    w = rng.standard_normal((co, ci, k, k, k)) * 0.3
    b = rng.standard_normal(co)
    skip = rng.standard_normal((B, co, n[2], n[1], n[0]))
    gy = rng.standard_normal((B, co, n[2], n[1], n[0]))
    dx_, dw_, db_, dskip, dy_ = _dev(torch, x), _dev(torch, w), _dev(torch, b), _dev(torch, skip), _dev(torch, gy)
    y = torch.empty((B, co) + shape[2:], dtype=torch.float32, device="cuda")
    dims = ws._I3(*n)
    for relu in (0, 1):
        assert lib.fftls_nn_conv3d(_ptr(dx_), _ptr(dw_), _ptr(db_), _ptr(dskip), _ptr(y), B, ci, co, dims, k, relu,
                                   None) == 0
        _close(y.cpu().numpy(), W.conv3d(x, w, b, skip=skip, relu=bool(relu)), 1e-5)
    gx_ref, gw_ref, gb_ref = W.conv3d_backward(x, w, gy)
    gx = torch.full(shape, 0.5, dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_conv3d_backward_data(_ptr(dy_), _ptr(dw_), _ptr(gx), B, ci, co, dims, k, 1, None) == 0
    _close(gx.cpu().numpy(), gx_ref + 0.5, 1e-5)   # accumulate = 1
    assert lib.fftls_nn_conv3d_backward_data(_ptr(dy_), _ptr(dw_), _ptr(gx), B, ci, co, dims, k, 0, None) == 0
    _close(gx.cpu().numpy(), gx_ref, 1e-5)
    need = lib.fftls_nn_wgrad_scratch(B, ci, co, dims, k)
    scratch = torch.empty(int(need), dtype=torch.float32, device="cuda")
    gw = torch.empty_like(dw_)
    gb = torch.empty_like(db_)
    assert lib.fftls_nn_conv3d_backward_weights(_ptr(dx_), _ptr(dy_), _ptr(gw), _ptr(gb), B, ci, co, dims, k,
                                                _ptr(scratch), need, None) == 0
    _close(gw.cpu().numpy(), gw_ref, 1e-4)
    _close(gb.cpu().numpy(), gb_ref, 1e-4)
    # too little scratch is refused before any launch
    assert lib.fftls_nn_conv3d_backward_weights(_ptr(dx_), _ptr(dy_), _ptr(gw), _ptr(gb), B, ci, co, dims, k,
                                                _ptr(scratch), need - 1, None) == fftls.E_INVALID_ARG


def test_pool_upsample_relu_mse_adam(env):
    torch, fftls, ws, lib = env
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3, 4, 6, 8))      # 3 planes, n = (8, 6, 4)
    n = ws._I3(8, 6, 4)
    nc = ws._I3(4, 3, 2)
    dxv = _dev(torch, x)
    y = torch.empty((3, 2, 3, 4), dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_pool2(_ptr(dxv), _ptr(y), 3, n, None) == 0
    _close(y.cpu().numpy(), W.pool2(x), 1e-6)
    g = rng.standard_normal((3, 2, 3, 4))
    gx = torch.ones((3, 4, 6, 8), dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_pool2_backward(_ptr(_dev(torch, g)), _ptr(gx), 3, n, 1, None) == 0
    _close(gx.cpu().numpy(), W.pool2_backward(g) + 1.0, 1e-6)
    up = torch.empty((3, 4, 6, 8), dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_upsample2(_ptr(_dev(torch, g)), _ptr(up), 3, nc, None) == 0
    _close(up.cpu().numpy(), W.up2(g), 1e-7)
    gc = torch.empty((3, 2, 3, 4), dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_upsample2_backward(_ptr(dxv), _ptr(gc), 3, nc, None) == 0
    _close(gc.cpu().numpy(), W.up2_backward(x), 1e-6)
    # relu backward
    act = rng.standard_normal(100)
    gr = rng.standard_normal(100)
    gt = _dev(torch, gr)
    assert lib.fftls_nn_relu_backward(_ptr(gt), _ptr(_dev(torch, act)), 100, None) == 0
    _close(gt.cpu().numpy(), gr * (act.astype(np.float32) > 0), 1e-7)
    # mse
    yv, tv = rng.standard_normal(1000), rng.standard_normal(1000)
    dy = torch.empty(1000, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.fftls_nn_mse(_ptr(_dev(torch, yv)), _ptr(_dev(torch, tv)), _ptr(dy), _ptr(loss), 1000, None) == 0
    L, gref = W.mse(yv, tv)
    assert abs(float(loss) - L) < 1e-5 * L
    _close(dy.cpu().numpy(), gref, 1e-5)
    # adam, two steps against the textbook update
    p0, g0 = rng.standard_normal(50), rng.standard_normal(50)
    p, gg = _dev(torch, p0), _dev(torch, g0)
    m, v = torch.zeros(50, device="cuda"), torch.zeros(50, device="cuda")
    pr, mr, vr = p0.copy(), np.zeros(50), np.zeros(50)
    for step in (1, 2):
        assert lib.fftls_nn_adam(_ptr(p), _ptr(gg), _ptr(m), _ptr(v), 50, 1e-2, 0.9, 0.999, 1e-8, step, None) == 0
        mr = 0.9 * mr + 0.1 * g0
        vr = 0.999 * vr + 0.001 * g0 * g0
        pr = pr - 1e-2 * (mr / (1 - 0.9 ** step)) / (np.sqrt(vr / (1 - 0.999 ** step)) + 1e-8)
    _close(p.cpu().numpy(), pr, 1e-5)


def test_features_and_strain_init(env):
    torch, fftls, ws, lib = env
    ph, _ = MS.boolean_spheres((16, 8, 8), 2.0, 0.3, seed=2)
    dph = torch.from_numpy(ph).cuda()
    x = torch.empty((2, 8, 8, 16), dtype=torch.float32, device="cuda")
    n = ws._I3(16, 8, 8)
    assert lib.fftls_nn_features(_ptr(dph), _ptr(x), n, 0.25, None) == 0
    xv = x.cpu().numpy()
    assert np.array_equal(xv[0], (ph == 1).astype(np.float32)) and np.all(xv[1] == 0.25)
    rng = np.random.default_rng(3)
    y = rng.standard_normal((6, 8, 8, 16))
    eps = torch.empty((6, 8, 8, 16), dtype=torch.float64, device="cuda")
    scratch = torch.empty(ws.STRAIN_SCRATCH, dtype=torch.float64, device="cuda")
    eb = (ctypes.c_double * 6)(0.5, 0, 0, 0, 0, 0)
    assert lib.fftls_nn_strain_init(_ptr(_dev(torch, y)), _ptr(eps), n, eb, 0.5, _ptr(scratch), None) == 0
    yf = y.astype(np.float32).astype(np.float64)
    fluct = 0.5 * (yf - yf.mean(axis=(1, 2, 3), keepdims=True))
    got = eps.cpu().numpy() - np.array([0.5, 0, 0, 0, 0, 0])[:, None, None, None]
    _close(got, fluct, 4e-7)   # the fluctuation is formed in FP32: a few units of 2^-24 of its scale
    assert np.abs(got.mean(axis=(1, 2, 3))).max() < 1e-7
    t = torch.empty((6, 8, 8, 16), dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_strain_target(_ptr(eps), _ptr(t), n, eb, None) == 0
    _close(t.cpu().numpy(), eps.cpu().numpy() - np.array([0.5, 0, 0, 0, 0, 0])[:, None, None, None], 1e-6)


def test_network_forward_and_gradients_match_oracle(env):
    torch, fftls, ws, lib = env
    net = ws.WarmNet(seed=1)
    params = W.random_params(seed=11)
    net.load_arrays(params)
    ph, _ = MS.boolean_spheres((16, 16, 8), 2.5, 0.3, seed=5)
    dph = torch.from_numpy(ph).cuda()
    net._buffers((16, 16, 8), True)
    net.features(dph, 100.0 * 10 ** 0.3)
    y = net.forward().cpu().numpy().reshape(6, 8, 16, 16)
    x = np.stack([(ph == 1).astype(np.float64), np.full(ph.shape, 0.3)])[None]
    pf = {k: (v[0].astype(np.float32).astype(np.float64), v[1].astype(np.float32).astype(np.float64))
          for k, v in params.items()}
    yr, acts = W.forward(pf, x)
    _close(y, yr[0], 1e-4)
    rng = np.random.default_rng(6)
    target = rng.standard_normal((6, 8, 16, 16))
    net.loss_and_grad(_dev(torch, target))
    net.backward()
    loss, gy = W.mse(yr, target[None])
    assert abs(float(net.loss_buf) - loss) < 1e-4 * loss
    gref = W.backward(pf, acts, gy)
    got = net.layer_arrays(grad=True)
    for name, *_ in ws.LAYERS:
        _close(got[name][0], gref[name][0], 2e-3)
        _close(got[name][1], gref[name][1], 2e-3)


def test_batched_step_gradient_is_mean_of_samples(env):
    """A training step over a batch of two samples gives the mean of the two single-sample
    gradients (the loss is the mean over every output value of the batch)."""
    torch, fftls, ws, lib = env
    net = ws.WarmNet(seed=1)
    net.load_arrays(W.random_params(seed=21))
    rng = np.random.default_rng(9)
    samples = []
    for i in range(2):
        ph, _ = MS.boolean_spheres((16, 16, 8), 2.5, 0.3, seed=30 + i)
        samples.append({"phase": torch.from_numpy(ph).cuda(), "contrast": 10.0 ** (1 + i),
                        "target": _dev(torch, rng.standard_normal((6, 8, 16, 16)))})
    single = []
    for d in samples:
        net._buffers((16, 16, 8), True, 1)
        net.features(d["phase"], d["contrast"])
        net.forward()
        net.loss_and_grad(d["target"])
        net.backward()
        single.append(net.grads.clone())
    net._buffers((16, 16, 8), True, 2)
    for slot, d in enumerate(samples):
        net.features(d["phase"], d["contrast"], slot)
        net.target[slot * 6 * 2048:(slot + 1) * 6 * 2048].copy_(d["target"].reshape(-1))
    net.forward()
    net.loss_and_grad(net.target)
    net.backward()
    want = 0.5 * (single[0] + single[1])
    assert float((net.grads - want).abs().max()) <= 1e-4 * float(want.abs().max())


def _timed(torch, fn):
    import time
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t


def test_trained_network_gain_over_plain_start(env):
    """What a short training on 32^3 samples buys on held-out 256^3 samples, every solve through the
    FP32 -> FP64 ladder to eta <= 1e-6 (the solver decides convergence): the initial field's error
    against the converged solution drops well below that of eps_bar, the moduli agree with the
    plain start's, the iteration count does not grow, and neither does the time to tolerance with
    the tensor-core inference counted in (best of three runs of each; 3 % allowed for timing noise,
    about twice the inference's share of a solve at this size).
    The accelerated scheme's iteration count depends only logarithmically on the starting error
    (scaling the exact fluctuation by 0.5 saves about 5 % of the iterations), so the gain itself
    is small."""
    torch, fftls, ws, lib = env
    solver = fftls.Solver(0)
    eb = np.diag([1.0, 0.0, 0.0])
    kw = dict(tol=1e-6, max_iter=3000, precision="fp32_refine64", want_strain=False, want_stress=False)
    try:
        train, _ = ws.make_dataset(solver, 192, 32, first_seed=5000, concurrency=8)
        held, _ = ws.make_dataset(solver, 2, 256, first_seed=9000, concurrency=2)
        assert all(d["converged"] for d in train + held)
        net = ws.WarmNet(seed=0)
        losses = net.train(train, epochs=16)
        assert losses[-1] < 0.6 * losses[0]
        zero, warm, err_zero, err_warm, t_zero, t_warm = [], [], [], [], [], []
        for d in held:
            lam, mu = MS.young_poisson_phases([(1.0, 0.3), (d["contrast"], 0.3)])
            ph, c = d["phase"], d["contrast"]
            solve = lambda **extra: solver.solve(ph, lam, mu, eb, "R", "AS", **kw, **extra)
            solver.solve(ph, lam, mu, eb, "R", "AS", **dict(kw, max_iter=3), raise_on_error=False)   # tile schedules
            e0 = net.initial_strain(ph, c)
            fluct = e0.float() - torch.tensor([1.0, 0, 0, 0, 0, 0], device="cuda").view(6, 1, 1, 1)
            err_warm.append(float(((fluct - d["target"].view(fluct.shape)) ** 2).mean()))
            err_zero.append(float((d["target"] ** 2).mean()))
            del e0, fluct
            r0, r1 = None, None
            best0 = best1 = float("inf")
            for _ in range(3):
                r0, t = _timed(torch, lambda: solve())
                best0 = min(best0, t)
                r1, t = _timed(torch, lambda: solve(eps_init=net.initial_strain(ph, c)))
                best1 = min(best1, t)
            assert r0.converged and r1.converged
            assert np.abs(r1.mean_stress - r0.mean_stress).max() < 1e-5 * np.abs(r0.mean_stress).max()
            zero.append(r0.iterations)
            warm.append(r1.iterations)
            t_zero.append(best0)
            t_warm.append(best1)
    finally:
        solver.close()
    assert np.mean(err_warm) < 0.7 * np.mean(err_zero)
    assert sum(warm) <= sum(zero)
    assert sum(t_warm) <= 1.03 * sum(t_zero), (t_warm, t_zero, warm, zero)
