"""GPU: the tensor-core path of the learned warm start (fftls_nn_tc_* of include/fftls_nn.h)
against oracle/warmnet_oracle.py.

The kernels round their operands to BF16 and accumulate in FP32.  The oracle is
given the same BF16-rounded inputs and weights (rounded here, on the host, to
the nearest BF16 with ties to even) and computes in FP64, so an FP32 output
differs from it only by FP32 accumulation: relative 1e-5 of the output's
largest magnitude.  A BF16 output adds its own rounding: half a BF16 unit,
2^-9 of the value, allowed as 2^-8 |value| on top.  Cases cover several tiles
with ragged edges, grids smaller than one tile, every stored channel count
(8, 16, 32, 64), both kernel sizes, the three input modes (same grid, upsampled
coarse grid, pooled fine grid), skips, ReLU, accumulation, and the transposed
packing of the input gradient.
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


def _bf16(a):
    """Nearest BF16 (ties to even) of float32(a), as float32 values."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def _stored(c):
    return 8 if c <= 8 else 16 if c <= 16 else 32 if c <= 32 else 64


def _to_cl(torch, a):
    """Planar (B, C, n3, n2, n1) -> channels-last BF16 device tensor (B, n3, n2, n1, stored(C))."""
    B, C = a.shape[:2]
    cl = np.zeros((B,) + a.shape[2:] + (_stored(C),), dtype=np.float32)
    cl[..., :C] = np.moveaxis(_bf16(a), 1, -1)
    bits = (cl.view(np.uint32) >> 16).astype(np.uint16)
    return torch.from_numpy(bits.view(np.int16)).to("cuda").view(torch.bfloat16)


def _from_cl(t, C):
    a = np.moveaxis(t.float().cpu().numpy(), -1, 1)
    return a[:, :C], a[:, C:]


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _close(got, want, rtol, vrel=0.0):
    scale = max(np.abs(want).max(), 1e-30)
    err = np.abs(got - want) - vrel * np.abs(want)
    assert err.max() <= rtol * scale, (err.max(), scale)


def _pack(torch, lib, w, ci, co, k, transposed):
    nbytes = int(lib.fftls_nn_tc_packed_bytes(ci, co, k, transposed))
    assert nbytes > 0
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    wd = torch.tensor(np.ascontiguousarray(w, dtype=np.float32), device="cuda")
    assert lib.fftls_nn_tc_pack(_p(wd), _p(buf), ci, co, k, transposed, None) == 0
    return buf


CASES = [
    # k, c_in, c_out, output grid (n1, n2, n3), input mode, batch
    (3, 16, 16, (40, 12, 10), 0, 1),     # two x tiles, the second ragged
    (3, 8, 6, (8, 8, 8), 0, 2),          # 8 stored channels (two taps per k step), 6 -> 8 stored outputs
    (3, 64, 32, (8, 8, 8), 0, 1),
    (3, 32, 64, (6, 4, 5), 0, 1),        # grid smaller than one tile
    (3, 16, 32, (8, 8, 8), 2, 1),        # input: mean pooling of a 16^3 grid
    (3, 64, 32, (8, 8, 4), 1, 1),        # input: upsampling of a 4 x 4 x 2 grid
    (3, 32, 16, (16, 16, 8), 1, 1),
    (1, 16, 8, (16, 8, 8), 1, 1),        # the 1x1x1 decoder layer
    (3, 8, 16, (8, 8, 8), 2, 1),
    (3, 2, 8, (1, 3, 2), 0, 1),          # 2 input channels padded to 8, tiny periodic grid
]


@pytest.mark.parametrize("k,ci,co,n,mode,B", CASES)
def test_tc_conv3d_matches_oracle(env, k, ci, co, n, mode, B):
    torch, fftls, ws, lib = env
    rng = np.random.default_rng(k * 1000 + ci * 10 + co + mode)
    n1, n2, n3 = n
    f = {0: 1.0, 1: 0.5, 2: 2.0}[mode]
    m = (int(n3 * f), int(n2 * f), int(n1 * f))
    x = _bf16(rng.standard_normal((B, ci) + m)).astype(np.float64)
    w = rng.standard_normal((co, ci, k, k, k)) * 0.3
    wb = _bf16(w).astype(np.float64)
    b = rng.standard_normal(co).astype(np.float32)
    skip = _bf16(rng.standard_normal((B, co, n3, n2, n1))).astype(np.float64)
    xin = x if mode == 0 else W.up2(x) if mode == 1 else _bf16(W.pool2(x)).astype(np.float64)
    xd, sd = _to_cl(torch, x), _to_cl(torch, skip)
    bd = torch.tensor(b, device="cuda")
    packed = _pack(torch, lib, w, ci, co, k, 0)
    dims = ws._I3(*n)
    # FP32 planar output, with and without ReLU and skip
    yp = torch.empty((B, co, n3, n2, n1), dtype=torch.float32, device="cuda")
    for relu, use_skip in ((0, False), (1, True)):
        assert lib.fftls_nn_tc_conv3d(_p(xd), _p(packed), _p(bd), _p(sd) if use_skip else None, _p(yp), B, ci, co,
                                      dims, k, mode, relu, 1, 0, None) == 0
        want = W.conv3d(xin, wb, b.astype(np.float64), skip=skip if use_skip else None, relu=bool(relu))
        _close(yp.cpu().numpy(), want, 1e-5)
    # channels-last BF16 output: padding channels zero; accumulate adds to it
    yc = torch.empty((B, n3, n2, n1, _stored(co)), dtype=torch.bfloat16, device="cuda")
    assert lib.fftls_nn_tc_conv3d(_p(xd), _p(packed), _p(bd), _p(sd), _p(yc), B, ci, co, dims, k, mode, 1, 0, 0,
                                  None) == 0
    got, pad = _from_cl(yc, co)
    want = W.conv3d(xin, wb, b.astype(np.float64), skip=skip, relu=True)
    _close(got, want, 1e-5, vrel=2.0 ** -8)
    assert not pad.any()
    prev = got.copy()
    assert lib.fftls_nn_tc_conv3d(_p(xd), _p(packed), None, None, _p(yc), B, ci, co, dims, k, mode, 0, 0, 1,
                                  None) == 0
    got, _ = _from_cl(yc, co)
    _close(got, prev + W.conv3d(xin, wb), 2e-5, vrel=2.0 ** -8)


@pytest.mark.parametrize("k,ci,co,n", [(3, 8, 6, (8, 8, 8)), (3, 32, 16, (16, 8, 8)), (3, 32, 64, (8, 8, 8)),
                                       (1, 16, 8, (8, 8, 16))])
def test_tc_input_gradient_matches_oracle(env, k, ci, co, n):
    """Transposed packing: dx = conv^T(dy, w), the input gradient of the layer w [co][ci][k^3]."""
    torch, fftls, ws, lib = env
    rng = np.random.default_rng(k + ci + co)
    shape = (1, co, n[2], n[1], n[0])
    gy = _bf16(rng.standard_normal(shape)).astype(np.float64)
    w = rng.standard_normal((co, ci, k, k, k)) * 0.3
    xdummy = np.zeros((1, ci) + shape[2:])
    gx_ref, _, _ = W.conv3d_backward(xdummy, _bf16(w).astype(np.float64), gy)
    packed = _pack(torch, lib, w, ci, co, k, 1)
    gx = torch.empty((1, ci) + shape[2:], dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_tc_conv3d(_p(_to_cl(torch, gy)), _p(packed), None, None, _p(gx), 1, co, ci, ws._I3(*n), k, 0,
                                  0, 1, 0, None) == 0
    _close(gx.cpu().numpy(), gx_ref, 1e-5)


@pytest.mark.parametrize("n", [(32, 8, 8), (40, 12, 6), (8, 8, 8)])
def test_tc_conv_phase_matches_oracle(env, n):
    """First layer from the phase bytes: the oracle convolves the two feature channels."""
    torch, fftls, ws, lib = env
    ph, _ = MS.boolean_spheres(n, 2.0, 0.3, seed=sum(n))
    ph[0, 0, :3] = 2          # a third phase id: not phase 1, so indicator 0
    rng = np.random.default_rng(4)
    w = (rng.standard_normal((8, 2, 3, 3, 3)) * 0.3).astype(np.float32)
    b = rng.standard_normal(8).astype(np.float32)
    lc = 0.75
    x = np.stack([(ph == 1).astype(np.float64), np.full(ph.shape, lc)])[None]
    want = W.conv3d(x, w.astype(np.float64), b.astype(np.float64), relu=True)
    y = torch.empty(ph.shape + (8,), dtype=torch.bfloat16, device="cuda")
    assert lib.fftls_nn_tc_conv_phase(_p(torch.from_numpy(ph).cuda()), _p(torch.tensor(w, device="cuda")),
                                      _p(torch.tensor(b, device="cuda")), _p(y), ws._I3(*n), 8, lc, 1, None) == 0
    got, _ = _from_cl(y[None], 8)
    _close(got, want, 1e-5, vrel=2.0 ** -8)


def test_tc_argument_checks(env):
    torch, fftls, ws, lib = env
    assert lib.fftls_nn_tc_packed_bytes(65, 8, 3, 0) == 0
    assert lib.fftls_nn_tc_packed_bytes(8, 8, 2, 0) == 0
    buf = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    x = torch.zeros((8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    dims = ws._I3(8, 8, 8)
    assert lib.fftls_nn_tc_conv3d(_p(x), _p(buf), None, None, _p(x), 1, 16, 16, dims, 3, 0, 0, 0, 0, None) \
        == fftls.E_INVALID_ARG                                   # y aliases x
    assert lib.fftls_nn_tc_conv3d(_p(x), _p(buf), None, None, _p(y), 1, 16, 16, dims, 3, 3, 0, 0, 0, None) \
        == fftls.E_INVALID_ARG                                   # no input mode 3
    assert lib.fftls_nn_tc_conv3d(_p(x), _p(buf), None, None, _p(y), 1, 16, 16, ws._I3(7, 8, 8), 3, 1, 0, 0, 0,
                                  None) == fftls.E_INVALID_ARG      # upsampling needs even sizes
    assert lib.fftls_nn_tc_conv3d(ctypes.c_void_p(x.data_ptr() + 2), _p(buf), None, None, _p(y), 1, 16, 16, dims,
                                  3, 0, 0, 0, 0, None) == fftls.E_INVALID_ARG   # 16-byte alignment
    assert lib.fftls_nn_tc_conv_phase(None, _p(buf), None, _p(y), dims, 8, 0.0, 1, None) == fftls.E_INVALID_ARG


def test_tc_network_matches_fp32_network(env):
    """The whole network on the tensor cores against the FP32 network with the same parameters.
    Every layer rounds its input and weights to BF16 (relative 2^-9 each); over eleven layers the
    output's relative L2 error stays at the percent level: bound 3e-2."""
    torch, fftls, ws, lib = env
    net = ws.WarmNet(seed=3)
    net.load_arrays(W.random_params(seed=12))
    for n in ((32, 32, 16), (48, 16, 24)):
        ph, _ = MS.boolean_spheres(n, 3.0, 0.25, seed=n[0])
        dph = torch.from_numpy(ph).cuda()
        net._buffers(n, False)
        net.features(dph, 50.0)
        ref = net.forward().clone().cpu().numpy()
        got = net.forward_tc(dph, 50.0).cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < 3e-2, rel
        # the packed weights follow parameter changes
        net.load_arrays(W.random_params(seed=13))
        net.features(dph, 50.0)
        ref2 = net.forward().clone().cpu().numpy()
        got2 = net.forward_tc(dph, 50.0).cpu().numpy()
        assert np.linalg.norm(got2 - ref2) / np.linalg.norm(ref2) < 3e-2
        net.load_arrays(W.random_params(seed=12))


WGRAD_CASES = [
    # k, c_in, c_out, output grid (n1, n2, n3), input mode, batch
    (3, 16, 16, (40, 12, 10), 0, 1),
    (3, 8, 6, (8, 8, 8), 0, 2),
    (3, 64, 32, (8, 8, 4), 1, 1),
    (3, 16, 32, (8, 8, 8), 2, 1),
    (1, 16, 8, (16, 8, 8), 1, 1),
    (3, 32, 64, (6, 4, 5), 0, 1),
    (3, 8, 16, (8, 8, 8), 2, 2),
    (3, 64, 64, (8, 8, 8), 0, 1),
]


@pytest.mark.parametrize("k,ci,co,n,mode,B", WGRAD_CASES)
def test_tc_weight_gradient_matches_oracle(env, k, ci, co, n, mode, B):
    """dW and db on the tensor cores against the oracle's weight gradient of the same BF16-rounded input
    and output gradient (FP32 accumulation per voxel tile: 2e-5 of the largest magnitude)."""
    torch, fftls, ws, lib = env
    rng = np.random.default_rng(k * 977 + ci * 13 + co + mode)
    n1, n2, n3 = n
    f = {0: 1.0, 1: 0.5, 2: 2.0}[mode]
    m = (int(n3 * f), int(n2 * f), int(n1 * f))
    x = _bf16(rng.standard_normal((B, ci) + m)).astype(np.float64)
    gy = _bf16(rng.standard_normal((B, co, n3, n2, n1))).astype(np.float64)
    xin = x if mode == 0 else W.up2(x) if mode == 1 else _bf16(W.pool2(x)).astype(np.float64)
    _, gw_ref, gb_ref = W.conv3d_backward(xin, np.zeros((co, ci, k, k, k)), gy)
    dims = ws._I3(*n)
    need = int(lib.fftls_nn_tc_wgrad_scratch(B, ci, co, dims, k))
    assert need > 0
    scratch = torch.empty(need, dtype=torch.float32, device="cuda")
    gw = torch.full((co, ci, k, k, k), 7.0, dtype=torch.float32, device="cuda")
    gb = torch.full((co,), 7.0, dtype=torch.float32, device="cuda")
    for _ in range(2):   # written, not accumulated: a second call gives the same result
        assert lib.fftls_nn_tc_conv3d_backward_weights(_p(_to_cl(torch, x)), _p(_to_cl(torch, gy)), _p(gw), _p(gb), B,
                                                       ci, co, dims, k, mode, _p(scratch), need, None) == 0
        _close(gw.cpu().numpy(), gw_ref, 2e-5)
        _close(gb.cpu().numpy(), gb_ref, 2e-5)
    assert lib.fftls_nn_tc_conv3d_backward_weights(_p(_to_cl(torch, x)), _p(_to_cl(torch, gy)), _p(gw), _p(gb), B,
                                                   ci, co, dims, k, mode, _p(scratch), need - 1, None) \
        == fftls.E_INVALID_ARG


@pytest.mark.parametrize("n", [(32, 8, 4), (40, 12, 6)])
def test_tc_phase_weight_gradient_matches_oracle(env, n):
    """The first layer's weight gradient from the phase bytes against the oracle's gradient with respect
    to the two-channel input's weights (indicator, constant log-contrast)."""
    torch, fftls, ws, lib = env
    ph, _ = MS.boolean_spheres(n, 2.0, 0.3, seed=sum(n) + 1)
    rng = np.random.default_rng(5)
    gy = _bf16(rng.standard_normal((1, 8) + ph.shape)).astype(np.float64)
    lc = -0.6
    x = np.stack([(ph == 1).astype(np.float64), np.full(ph.shape, np.float64(np.float32(lc)))])[None]
    _, gw_ref, gb_ref = W.conv3d_backward(x, np.zeros((8, 2, 3, 3, 3)), gy)
    dims = ws._I3(*n)
    need = int(lib.fftls_nn_tc_phase_wgrad_scratch(dims))
    scratch = torch.empty(need, dtype=torch.float32, device="cuda")
    gw = torch.empty((8, 2, 3, 3, 3), dtype=torch.float32, device="cuda")
    gb = torch.empty(8, dtype=torch.float32, device="cuda")
    assert lib.fftls_nn_tc_conv_phase_backward_weights(_p(torch.from_numpy(ph).cuda()), _p(_to_cl(torch, gy)), _p(gw),
                                                       _p(gb), dims, 8, lc, _p(scratch), need, None) == 0
    _close(gw.cpu().numpy(), gw_ref, 2e-5)
    _close(gb.cpu().numpy(), gb_ref, 2e-5)


def test_tc_elementwise_backward(env):
    """Layout change, ReLU backward, addition and the adjoints of upsampling and pooling on
    channels-last BF16, against numpy on the same BF16 values (one rounding of the result)."""
    torch, fftls, ws, lib = env
    rng = np.random.default_rng(8)
    B, c, nc = 2, 12, (4, 3, 2)        # coarse grid (n1, n2, n3); 12 channels stored as 16
    fine = (B, c, 2 * nc[2], 2 * nc[1], 2 * nc[0])
    coarse = (B, c, nc[2], nc[1], nc[0])
    # planar FP32 -> channels-last BF16
    xp = rng.standard_normal((B, 6, 4, 4, 8)).astype(np.float32)
    y = torch.empty((B, 4, 4, 8, 8), dtype=torch.bfloat16, device="cuda")
    assert lib.fftls_nn_tc_from_planar(_p(torch.tensor(xp, device="cuda")), _p(y), B, 6, 128, None) == 0
    got, pad = _from_cl(y, 6)
    assert np.array_equal(got, _bf16(xp)) and not pad.any()
    # relu backward and add
    g = _bf16(rng.standard_normal(fine))
    act = _bf16(rng.standard_normal(fine))
    gd, ad = _to_cl(torch, g), _to_cl(torch, act)
    assert lib.fftls_nn_tc_relu_backward(_p(gd), _p(ad), gd.numel(), None) == 0
    assert np.array_equal(_from_cl(gd, c)[0], g * (act > 0))
    h = _bf16(rng.standard_normal(fine))
    hd = _to_cl(torch, h)
    assert lib.fftls_nn_tc_add(_p(hd), _p(gd), hd.numel(), None) == 0
    _close(_from_cl(hd, c)[0], h + g * (act > 0), 0.0, vrel=2.0 ** -8)
    # adjoint of upsampling: coarse = sum over each 2x2x2 block
    up = torch.empty((B,) + coarse[2:] + (16,), dtype=torch.bfloat16, device="cuda")
    assert lib.fftls_nn_tc_upsample2_backward(_p(_to_cl(torch, h)), _p(up), B, c, ws._I3(*nc), None) == 0
    _close(_from_cl(up, c)[0], W.up2_backward(h.astype(np.float64)), 1e-6, vrel=2.0 ** -8)
    # adjoint of pooling, written and accumulated
    q = _bf16(rng.standard_normal(coarse))
    fd = torch.empty((B,) + fine[2:] + (16,), dtype=torch.bfloat16, device="cuda")
    assert lib.fftls_nn_tc_pool2_backward(_p(_to_cl(torch, q)), _p(fd), B, c, ws._I3(*nc), 0, None) == 0
    assert np.array_equal(_from_cl(fd, c)[0], W.pool2_backward(q.astype(np.float64)).astype(np.float32))
    base = _bf16(rng.standard_normal(fine))
    fd = _to_cl(torch, base)
    assert lib.fftls_nn_tc_pool2_backward(_p(_to_cl(torch, q)), _p(fd), B, c, ws._I3(*nc), 1, None) == 0
    _close(_from_cl(fd, c)[0], base + W.pool2_backward(q.astype(np.float64)), 1e-6, vrel=2.0 ** -8)


def test_tc_network_gradients_close_to_fp32(env):
    """Every parameter gradient of the tensor-core backward against the FP32 network's on the same batch
    of two 32 x 32 x 16 samples; the loss within 1 %, each layer's gradient within 10 % (relative L2):
    a gradient passes about twenty BF16 roundings of activations and gradients (2^-9 relative each),
    ReLU units near zero switch, and the deepest level sums over only 64 voxels."""
    torch, fftls, ws, lib = env
    net = ws.WarmNet(seed=2)
    net.load_arrays(W.random_params(seed=31))
    rng = np.random.default_rng(10)
    group = []
    for i in range(2):
        ph, _ = MS.boolean_spheres((32, 32, 16), 2.5, 0.3, seed=40 + i)
        group.append({"phase": torch.from_numpy(ph).cuda(), "contrast": 20.0 * (i + 1),
                      "target": torch.tensor(rng.standard_normal((6, 16, 32, 32)), dtype=torch.float32,
                                             device="cuda")})
    # FP32 reference gradient of the batch
    net._buffers((32, 32, 16), True, 2)
    for slot, d in enumerate(group):
        net.features(d["phase"], d["contrast"], slot)
        net.target[slot * 6 * 16384:(slot + 1) * 6 * 16384].copy_(d["target"].reshape(-1))
    net.forward()
    net.loss_and_grad(net.target)
    net.backward()
    ref = net.layer_arrays(grad=True)
    loss_ref = float(net.loss_buf)
    # tensor cores
    phases = [d["phase"] for d in group]
    contrasts = [d["contrast"] for d in group]
    net.forward_tc_batch(phases, contrasts, train=True)
    for slot, d in enumerate(group):
        net.tc_target[slot * 6 * 16384:(slot + 1) * 6 * 16384].copy_(d["target"].reshape(-1))
    assert lib.fftls_nn_mse(_p(net.tc["y"]), _p(net.tc_target), _p(net.tc_gy), _p(net.tc_loss),
                            net.tc["y"].numel(), None) == 0
    net.grads.zero_()
    net.backward_tc(phases, contrasts)
    got = net.layer_arrays(grad=True)
    assert abs(float(net.tc_loss) - loss_ref) < 1e-2 * loss_ref
    for name, *_ in ws.LAYERS:
        for j in (0, 1):
            r = np.linalg.norm(got[name][j] - ref[name][j]) / np.linalg.norm(ref[name][j])
            assert r < 0.1, (name, j, r)


def test_tc_training_reduces_loss(env):
    """A short training on the tensor cores lowers the loss on solver-generated fields."""
    torch, fftls, ws, lib = env
    solver = fftls.Solver(0)
    try:
        data, _ = ws.make_dataset(solver, 32, 32, first_seed=7000, concurrency=8)
    finally:
        solver.close()
    net = ws.WarmNet(seed=0)
    losses = net.train(data, epochs=8, batch=4, lr=1e-3, lr_final=1e-4, tensor_cores=True)
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0]
