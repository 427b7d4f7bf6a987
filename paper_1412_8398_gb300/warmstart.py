"""Learned warm start of the FFT Lippmann-Schwinger iteration (C ABI: include/fftls_nn.h).

A U-shaped 3D convolutional network (about 289k parameters, periodic padding)
maps the indicator of phase 1 and the log-contrast of a two-phase
microstructure to the strain fluctuation of the unit load eps_bar = e1 (x) e1.
The solver then starts from eps^0 = eps_bar + s (prediction - its mean) for the
load s e1 (x) e1 (the problem is linear), and its own equilibrium criterion
decides convergence: the network can only change the number of iterations.
The training targets are fields the solver itself produces.

Every step of the network (convolutions and their gradients, pooling,
upsampling, loss, Adam) runs in the library's CUDA kernels; torch only holds
device memory.  The paper has no learned component.

Layout: activations [channel][n3][n2][n1] (batch 1), FP32; parameters are one
flat FP32 vector, layer by layer in LAYERS order, weights [c_out][c_in][k^3]
then bias [c_out].

Inference also runs on the tensor cores (``predict_tc``): BF16 weights and
channels-last BF16 activations, FP32 accumulation, the pooling and upsampling
folded into the next convolution's input staging and the first layer computed
from the phase bytes.  Training stays in FP32.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np

from . import fftls
from . import microstructure as MS

# (name, c_in, c_out, kernel size, grid level: the grid is n / 2^level)
LAYERS = [
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
LEVELS = 3  # grid lengths must be divisible by 2^LEVELS

# activations: name -> (channels, level)
_ACTS = {
    "x": (2, 0), "e0": (8, 0), "p0": (8, 1), "a1": (16, 1), "e1": (16, 1), "p1": (16, 2), "a2": (32, 2),
    "e2": (32, 2), "p2": (32, 3), "a3": (64, 3), "e3": (64, 3), "u2": (64, 2), "d2": (32, 2), "u1": (32, 1),
    "d1": (16, 1), "u0": (16, 0), "d0": (8, 0), "y": (6, 0),
}
# channels-last BF16 activations of the tensor-core forward: name -> (stored channels, level)
_TC_ACTS = {
    "e0": (8, 0), "a1": (16, 1), "e1": (16, 1), "a2": (32, 2), "e2": (32, 2), "a3": (64, 3), "e3": (64, 3),
    "d2": (32, 2), "d1": (16, 1), "d0": (8, 0),
}
# tensor-core forward: (layer, input, input mode (0 same grid, 1 upsampled coarse, 2 pooled fine), skip)
_TC_PLAN = [
    ("enc1a", "e0", 2, None), ("enc1b", "a1", 0, None), ("enc2a", "e1", 2, None), ("enc2b", "a2", 0, None),
    ("enc3a", "e2", 2, None), ("enc3b", "a3", 0, None), ("dec2", "e3", 1, "e2"), ("dec1", "d2", 1, "e1"),
    ("dec0", "d1", 1, "e0"),
]
_TC_OUT = {"enc1a": "a1", "enc1b": "e1", "enc2a": "a2", "enc2b": "e2", "enc3a": "a3", "enc3b": "e3",
           "dec2": "d2", "dec1": "d1", "dec0": "d0"}

# channels-last BF16 gradients of the tensor-core backward: name -> (channels, level)
_TC_GRADS = {
    "gy": (6, 0), "gd0": (8, 0), "gu0": (16, 0), "gd1": (16, 1), "gu1": (32, 1), "gd2": (32, 2), "gu2": (64, 2),
    "ge3": (64, 3), "ga3": (64, 3), "gp2": (32, 3), "ga2": (32, 2), "gp1": (16, 2), "ga1": (16, 1), "gp0": (8, 1),
}


def _stored(c):
    """Stored channels of a channels-last activation with c channels."""
    return 8 if c <= 8 else 16 if c <= 16 else 32 if c <= 32 else 64


# gradient buffers: name -> (channels, level)
_GRADS = {
    "gy": (6, 0), "gd0": (8, 0), "gu0": (16, 0), "gd1": (16, 1), "gu1": (32, 1), "gd2": (32, 2), "gu2": (64, 2),
    "ge3": (64, 3), "ga3": (64, 3), "gp2": (32, 3), "ga2": (32, 2), "gp1": (16, 2), "ga1": (16, 1),
    "gp0": (8, 1),
}

_P = ctypes.c_void_p
_I3 = ctypes.c_int * 3
_NN_SIGNATURES = {
    "fftls_nn_conv3d": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I3,
                                       ctypes.c_int, ctypes.c_int, _P]),
    "fftls_nn_conv3d_backward_data": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I3,
                                                     ctypes.c_int, ctypes.c_int, _P]),
    "fftls_nn_conv3d_backward_weights": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                        _I3, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "fftls_nn_wgrad_scratch": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I3, ctypes.c_int]),
    "fftls_nn_relu_backward": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "fftls_nn_pool2": (ctypes.c_int, [_P, _P, ctypes.c_int, _I3, _P]),
    "fftls_nn_pool2_backward": (ctypes.c_int, [_P, _P, ctypes.c_int, _I3, ctypes.c_int, _P]),
    "fftls_nn_upsample2": (ctypes.c_int, [_P, _P, ctypes.c_int, _I3, _P]),
    "fftls_nn_upsample2_backward": (ctypes.c_int, [_P, _P, ctypes.c_int, _I3, _P]),
    "fftls_nn_add": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "fftls_nn_mse": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_longlong, _P]),
    "fftls_nn_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_longlong, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_int, _P]),
    "fftls_nn_features": (ctypes.c_int, [_P, _P, _I3, ctypes.c_float, _P]),
    "fftls_nn_strain_init": (ctypes.c_int, [_P, _P, _I3, ctypes.POINTER(ctypes.c_double), ctypes.c_double, _P, _P]),
    "fftls_nn_strain_target": (ctypes.c_int, [_P, _P, _I3, ctypes.POINTER(ctypes.c_double), _P]),
    "fftls_nn_tc_packed_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "fftls_nn_tc_pack": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "fftls_nn_tc_conv3d": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I3,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "fftls_nn_tc_conv_phase": (ctypes.c_int, [_P, _P, _P, _P, _I3, ctypes.c_int, ctypes.c_float, ctypes.c_int, _P]),
    "fftls_nn_tc_wgrad_scratch": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I3, ctypes.c_int]),
    "fftls_nn_tc_conv3d_backward_weights": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                           _I3, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "fftls_nn_tc_phase_wgrad_scratch": (ctypes.c_size_t, [_I3]),
    "fftls_nn_tc_conv_phase_backward_weights": (ctypes.c_int, [_P, _P, _P, _P, _I3, ctypes.c_int, ctypes.c_float, _P,
                                                               ctypes.c_size_t, _P]),
    "fftls_nn_tc_from_planar": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _P]),
    "fftls_nn_tc_relu_backward": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "fftls_nn_tc_add": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "fftls_nn_tc_upsample2_backward": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _I3, _P]),
    "fftls_nn_tc_pool2_backward": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _I3, ctypes.c_int, _P]),
}
STRAIN_SCRATCH = 1536  # FFTLS_NN_STRAIN_SCRATCH

_LIB = None


def _lib():
    """The library with the warm-start signatures applied (raises if it is missing)."""
    global _LIB
    if _LIB is None:
        lib = fftls.load_library()
        for name, (res, args) in _NN_SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def parameter_count() -> int:
    return sum(co * ci * k ** 3 + co for _, ci, co, k, _ in LAYERS)


def _check(st, what):
    if st != fftls.OK:
        raise fftls.FftlsError(st, what)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def log_contrast(contrast: float) -> float:
    """Second input channel: log10 of E_incl / E_matrix, centred on a contrast of 100."""
    return math.log10(contrast) - 2.0


class WarmNet:
    """The network, its parameters, Adam state and per-grid activation buffers."""

    def __init__(self, device: int = 0, seed: int = 0, stream=None):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.lib = _lib()
        self.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", 0) or 0)) if stream is not None else None
        self.offsets = {}
        off = 0
        for name, ci, co, k, _ in LAYERS:
            nw = co * ci * k ** 3
            self.offsets[name] = (off, nw, off + nw, co)
            off += nw + co
        self.count = off
        rng = np.random.default_rng(seed)
        host = np.zeros(off, dtype=np.float32)
        for name, ci, co, k, _ in LAYERS:
            o, nw, _, _ = self.offsets[name]
            std = math.sqrt(2.0 / (ci * k ** 3)) * (0.1 if name == "out" else 1.0)
            host[o:o + nw] = rng.standard_normal(nw).astype(np.float32) * std
        self.params = torch.tensor(host, device=self.dev)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.steps = 0
        self._grid = None
        self.losses = []
        self.version = 0          # bumped whenever the parameters change
        self._tc_packed = None    # (version, {layer: packed BF16 weights})
        self._tc_packed_t = None  # the same, transposed for the input gradient
        self._tc_grid = None

    # -- parameters ------------------------------------------------------
    def _w(self, name, grad=False):
        o, _, _, _ = self.offsets[name]
        t = self.grads if grad else self.params
        return ctypes.c_void_p(t.data_ptr() + 4 * o)

    def _b(self, name, grad=False):
        _, _, ob, _ = self.offsets[name]
        t = self.grads if grad else self.params
        return ctypes.c_void_p(t.data_ptr() + 4 * ob)

    def layer_arrays(self, grad=False):
        """Host copies {name: (w, b)} of the parameters (or gradients)."""
        src = (self.grads if grad else self.params).cpu().numpy()
        out = {}
        for name, ci, co, k, _ in LAYERS:
            o, nw, ob, nb = self.offsets[name]
            out[name] = (src[o:o + nw].reshape(co, ci, k, k, k).copy(), src[ob:ob + nb].copy())
        return out

    def load_arrays(self, arrays):
        host = np.zeros(self.count, dtype=np.float32)
        for name, ci, co, k, _ in LAYERS:
            o, nw, ob, nb = self.offsets[name]
            host[o:o + nw] = np.asarray(arrays[name][0], dtype=np.float32).reshape(-1)
            host[ob:ob + nb] = np.asarray(arrays[name][1], dtype=np.float32).reshape(-1)
        self.params.copy_(self.torch.from_numpy(host).to(self.dev))
        self.version += 1

    def save(self, path):
        np.savez(path, params=self.params.cpu().numpy(), layers=np.array([str(l) for l in LAYERS]))

    def load(self, path):
        z = np.load(path)
        if z["params"].size != self.count:
            raise ValueError("parameter file does not match this network")
        self.params.copy_(self.torch.from_numpy(z["params"].astype(np.float32)).to(self.dev))
        self.version += 1

    # -- buffers ----------------------------------------------------------
    def _buffers(self, n, train, batch=1):
        n = tuple(int(v) for v in n)
        if any(v % (1 << LEVELS) for v in n):
            raise ValueError(f"grid lengths must be multiples of {1 << LEVELS}")
        key = (n, train, batch)
        if self._grid == key:
            return
        torch = self.torch
        vox = lambda lvl: batch * (n[0] >> lvl) * (n[1] >> lvl) * (n[2] >> lvl)
        self.a = {k: torch.empty(c * vox(l), dtype=torch.float32, device=self.dev) for k, (c, l) in _ACTS.items()}
        self.g = {}
        self.scratch = None
        if train:
            self.g = {k: torch.empty(c * vox(l), dtype=torch.float32, device=self.dev) for k, (c, l) in _GRADS.items()}
            self.target = torch.empty(6 * vox(0), dtype=torch.float32, device=self.dev)
            need = max(self.lib.fftls_nn_wgrad_scratch(batch, ci, co, self._dims(n, lvl), k)
                       for _, ci, co, k, lvl in LAYERS)
            self.scratch = torch.empty(int(need), dtype=torch.float32, device=self.dev)
            self.loss_buf = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.mean_scratch = torch.empty(STRAIN_SCRATCH, dtype=torch.float64, device=self.dev)
        self.n = n
        self.batch = batch
        self._grid = key

    @staticmethod
    def _dims(n, lvl):
        return _I3(n[0] >> lvl, n[1] >> lvl, n[2] >> lvl)

    # -- network ----------------------------------------------------------
    def _conv(self, name, src, dst, skip=None, relu=True):
        _, ci, co, k, lvl = next(l for l in LAYERS if l[0] == name)
        st = self.lib.fftls_nn_conv3d(_p(self.a[src]), self._w(name), self._b(name),
                                      _p(self.a[skip]) if skip else None, _p(self.a[dst]), self.batch, ci, co,
                                      self._dims(self.n, lvl), k, 1 if relu else 0, self.stream)
        _check(st, f"conv {name}")

    def _pool(self, src, dst, channels, lvl):
        _check(self.lib.fftls_nn_pool2(_p(self.a[src]), _p(self.a[dst]), self.batch * channels, self._dims(self.n, lvl),
                                       self.stream), "pool")

    def _up(self, src, dst, channels, lvl_coarse):
        _check(self.lib.fftls_nn_upsample2(_p(self.a[src]), _p(self.a[dst]), self.batch * channels,
                                           self._dims(self.n, lvl_coarse), self.stream), "upsample")

    def features(self, phase, contrast, slot=0):
        """Fill the input channels of batch entry `slot` from a device phase image (uint8, (n3, n2, n1))."""
        n = (phase.shape[2], phase.shape[1], phase.shape[0])
        if self._grid is None or self._grid[0] != n:
            self._buffers(n, False)
        if not 0 <= slot < self.batch:
            raise ValueError("batch entry out of range")
        x = ctypes.c_void_p(self.a["x"].data_ptr() + 4 * 2 * n[0] * n[1] * n[2] * slot)
        _check(self.lib.fftls_nn_features(_p(phase), x, _I3(*n), float(log_contrast(contrast)), self.stream),
               "features")

    def forward(self):
        c = self._conv
        c("enc0", "x", "e0")
        self._pool("e0", "p0", 8, 0)
        c("enc1a", "p0", "a1")
        c("enc1b", "a1", "e1")
        self._pool("e1", "p1", 16, 1)
        c("enc2a", "p1", "a2")
        c("enc2b", "a2", "e2")
        self._pool("e2", "p2", 32, 2)
        c("enc3a", "p2", "a3")
        c("enc3b", "a3", "e3")
        self._up("e3", "u2", 64, 3)
        c("dec2", "u2", "d2", skip="e2")
        self._up("d2", "u1", 32, 2)
        c("dec1", "u1", "d1", skip="e1")
        self._up("d1", "u0", 16, 1)
        c("dec0", "u0", "d0", skip="e0")
        c("out", "d0", "y", relu=False)
        return self.a["y"]

    def backward(self):
        """Parameter gradients of the loss whose output gradient is in self.g['gy']."""
        lib, s, n, B = self.lib, self.stream, self.n, self.batch
        a, g = self.a, self.g
        scratch = _p(self.scratch)
        ns = self.scratch.numel()

        def wgrad(name, src, gout):
            _, ci, co, k, lvl = next(l for l in LAYERS if l[0] == name)
            _check(lib.fftls_nn_conv3d_backward_weights(_p(a[src]), _p(g[gout]), self._w(name, True),
                                                        self._b(name, True), B, ci, co, self._dims(n, lvl), k,
                                                        scratch, ns, s), f"wgrad {name}")

        def dgrad(name, gout, gin):
            _, ci, co, k, lvl = next(l for l in LAYERS if l[0] == name)
            _check(lib.fftls_nn_conv3d_backward_data(_p(g[gout]), self._w(name), _p(g[gin]), B, ci, co,
                                                     self._dims(n, lvl), k, 0, s), f"dgrad {name}")

        def relu(gname, act):
            _check(lib.fftls_nn_relu_backward(_p(g[gname]), _p(a[act]), a[act].numel(), s), "relu")

        def up_bwd(gsrc, gdst, ch, lvl_coarse):
            _check(lib.fftls_nn_upsample2_backward(_p(g[gsrc]), _p(g[gdst]), B * ch, self._dims(n, lvl_coarse), s),
                   "upsample backward")

        def pool_bwd_acc(gsrc, gdst, ch, lvl_fine):
            _check(lib.fftls_nn_pool2_backward(_p(g[gsrc]), _p(g[gdst]), B * ch, self._dims(n, lvl_fine), 1, s),
                   "pool backward")

        wgrad("out", "d0", "gy")
        dgrad("out", "gy", "gd0")
        relu("gd0", "d0")
        wgrad("dec0", "u0", "gd0")
        dgrad("dec0", "gd0", "gu0")
        up_bwd("gu0", "gd1", 16, 1)
        relu("gd1", "d1")
        wgrad("dec1", "u1", "gd1")
        dgrad("dec1", "gd1", "gu1")
        up_bwd("gu1", "gd2", 32, 2)
        relu("gd2", "d2")
        wgrad("dec2", "u2", "gd2")
        dgrad("dec2", "gd2", "gu2")
        up_bwd("gu2", "ge3", 64, 3)
        relu("ge3", "e3")
        wgrad("enc3b", "a3", "ge3")
        dgrad("enc3b", "ge3", "ga3")
        relu("ga3", "a3")
        wgrad("enc3a", "p2", "ga3")
        dgrad("enc3a", "ga3", "gp2")
        pool_bwd_acc("gp2", "gd2", 32, 2)   # gd2 now holds the gradient of e2
        relu("gd2", "e2")
        wgrad("enc2b", "a2", "gd2")
        dgrad("enc2b", "gd2", "ga2")
        relu("ga2", "a2")
        wgrad("enc2a", "p1", "ga2")
        dgrad("enc2a", "ga2", "gp1")
        pool_bwd_acc("gp1", "gd1", 16, 1)   # gradient of e1
        relu("gd1", "e1")
        wgrad("enc1b", "a1", "gd1")
        dgrad("enc1b", "gd1", "ga1")
        relu("ga1", "a1")
        wgrad("enc1a", "p0", "ga1")
        dgrad("enc1a", "ga1", "gp0")
        pool_bwd_acc("gp0", "gd0", 8, 0)    # gradient of e0
        relu("gd0", "e0")
        wgrad("enc0", "x", "gd0")

    def loss_and_grad(self, target):
        """MSE of the output against target ([6][N] FP32 device) into the loss buffer; output gradient in gy."""
        _check(self.lib.fftls_nn_mse(_p(self.a["y"]), _p(target), _p(self.g["gy"]), _p(self.loss_buf),
                                     self.a["y"].numel(), self.stream), "mse")

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.steps += 1
        self.version += 1
        _check(self.lib.fftls_nn_adam(_p(self.params), _p(self.grads), _p(self.m), _p(self.v), self.count,
                                      float(lr), beta1, beta2, eps, self.steps, self.stream), "adam")

    # -- tensor-core inference -------------------------------------------
    def _tc_weights(self, transposed=False):
        """Packed BF16 weights of every layer after the first (transposed: for the input gradient),
        repacked when the parameters changed."""
        cache = self._tc_packed_t if transposed else self._tc_packed
        if cache is not None and cache[0] == self.version:
            return cache[1]
        torch = self.torch
        packed = {}
        for name, ci, co, k, _ in LAYERS[1:]:
            nbytes = int(self.lib.fftls_nn_tc_packed_bytes(ci, co, k, int(transposed)))
            buf = torch.empty(nbytes, dtype=torch.uint8, device=self.dev)
            _check(self.lib.fftls_nn_tc_pack(self._w(name), _p(buf), ci, co, k, int(transposed), self.stream),
                   f"pack {name}")
            packed[name] = buf
        if transposed:
            self._tc_packed_t = (self.version, packed)
        else:
            self._tc_packed = (self.version, packed)
        return packed

    def _tc_buffers(self, n, batch=1, train=False):
        n = tuple(int(v) for v in n)
        if any(v % (1 << LEVELS) for v in n):
            raise ValueError(f"grid lengths must be multiples of {1 << LEVELS}")
        key = (n, batch, train)
        if self._tc_grid == key:
            return
        torch = self.torch
        vox = lambda lvl: batch * (n[0] >> lvl) * (n[1] >> lvl) * (n[2] >> lvl)
        self.tc = {k: torch.empty(c * vox(l), dtype=torch.bfloat16, device=self.dev) for k, (c, l) in _TC_ACTS.items()}
        self.tc["y"] = torch.empty(6 * vox(0), dtype=torch.float32, device=self.dev)
        self.tc_mean_scratch = torch.empty(STRAIN_SCRATCH, dtype=torch.float64, device=self.dev)
        self.tcg = {}
        if train:
            self.tcg = {k: torch.empty(_stored(c) * vox(l), dtype=torch.bfloat16, device=self.dev)
                        for k, (c, l) in _TC_GRADS.items()}
            self.tc_gy = torch.empty(6 * vox(0), dtype=torch.float32, device=self.dev)
            self.tc_target = torch.empty(6 * vox(0), dtype=torch.float32, device=self.dev)
            self.tc_loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
            need = max(self.lib.fftls_nn_tc_wgrad_scratch(batch, ci, co, self._dims(n, lvl), k)
                       for _, ci, co, k, lvl in LAYERS[1:])
            need = max(int(need), int(self.lib.fftls_nn_tc_phase_wgrad_scratch(self._dims(n, 0))))
            self.tc_scratch = torch.empty(need, dtype=torch.float32, device=self.dev)
            self.tc_dw0 = torch.empty(self.offsets["enc0"][1] + 8, dtype=torch.float32, device=self.dev)
        self.tc_batch = batch
        self._tc_grid = key

    def forward_tc(self, phase, contrast):
        """The network on the tensor cores for a device phase image (uint8, (n3, n2, n1)); returns the
        FP32 output [6][N]."""
        return self.forward_tc_batch([phase], [contrast])

    def forward_tc_batch(self, phases, contrasts, train=False):
        """The network on the tensor cores for a batch of phase images of one grid; returns the FP32
        output [batch][6][N]."""
        n = (phases[0].shape[2], phases[0].shape[1], phases[0].shape[0])
        B = len(phases)
        if self._tc_grid is None or self._tc_grid[0] != n or self._tc_grid[1] != B or (train and not self._tc_grid[2]):
            self._tc_buffers(n, B, train)
        packed = self._tc_weights()
        lib, s, t = self.lib, self.stream, self.tc
        N = n[0] * n[1] * n[2]
        for b, (ph, c) in enumerate(zip(phases, contrasts)):
            if tuple(ph.shape) != tuple(phases[0].shape):
                raise ValueError("the samples of a batch must share one grid")
            e0 = ctypes.c_void_p(t["e0"].data_ptr() + 2 * 8 * N * b)
            _check(lib.fftls_nn_tc_conv_phase(_p(ph), self._w("enc0"), self._b("enc0"), e0, _I3(*n), 8,
                                              float(log_contrast(c)), 1, s), "conv enc0")
        layer = {l[0]: l for l in LAYERS}
        for name, src, mode, skip in _TC_PLAN:
            _, ci, co, k, lvl = layer[name]
            _check(lib.fftls_nn_tc_conv3d(_p(t[src]), _p(packed[name]), self._b(name), _p(t[skip]) if skip else None,
                                          _p(t[_TC_OUT[name]]), B, ci, co, self._dims(n, lvl), k, mode, 1, 0, 0, s),
                   f"conv {name}")
        _, ci, co, k, lvl = layer["out"]
        _check(lib.fftls_nn_tc_conv3d(_p(t["d0"]), _p(packed["out"]), self._b("out"), None, _p(t["y"]), B, ci, co,
                                      self._dims(n, 0), k, 0, 0, 1, 0, s), "conv out")
        return t["y"]

    def backward_tc(self, phases, contrasts):
        """Parameter gradients (into self.grads) of the loss whose output gradient is in self.tc_gy, after
        forward_tc_batch(..., train=True) on the same batch: the forward's chain backwards on the
        tensor cores (BF16 channels-last gradients, FP32 weight gradients)."""
        lib, s, t, g = self.lib, self.stream, self.tc, self.tcg
        n = self._tc_grid[0]
        B = self.tc_batch
        N = n[0] * n[1] * n[2]
        packed_t = self._tc_weights(transposed=True)
        layer = {l[0]: l for l in LAYERS}
        scratch, ns = _p(self.tc_scratch), self.tc_scratch.numel()
        vox = lambda lvl: B * (n[0] >> lvl) * (n[1] >> lvl) * (n[2] >> lvl)

        def wgrad(name, src, gout, mode):
            _, ci, co, k, lvl = layer[name]
            _check(lib.fftls_nn_tc_conv3d_backward_weights(_p(src), _p(g[gout]), self._w(name, True),
                                                           self._b(name, True), B, ci, co, self._dims(n, lvl), k, mode,
                                                           scratch, ns, s), f"wgrad {name}")

        def dgrad(name, gout, gin):
            _, ci, co, k, lvl = layer[name]
            _check(lib.fftls_nn_tc_conv3d(_p(g[gout]), _p(packed_t[name]), None, None, _p(g[gin]), B, co, ci,
                                          self._dims(n, lvl), k, 0, 0, 0, 0, s), f"dgrad {name}")

        def relu(gname, act):
            _check(lib.fftls_nn_tc_relu_backward(_p(g[gname]), _p(t[act]), t[act].numel(), s), "relu")

        def up_bwd(gsrc, gdst, ch, lvl_coarse):
            _check(lib.fftls_nn_tc_upsample2_backward(_p(g[gsrc]), _p(g[gdst]), B, ch, self._dims(n, lvl_coarse), s),
                   "upsample backward")

        def pool_bwd_acc(gsrc, gdst, ch, lvl_coarse):
            _check(lib.fftls_nn_tc_pool2_backward(_p(g[gsrc]), _p(g[gdst]), B, ch, self._dims(n, lvl_coarse), 1, s),
                   "pool backward")

        _check(lib.fftls_nn_tc_from_planar(_p(self.tc_gy), _p(g["gy"]), B, 6, N, s), "gradient layout")
        wgrad("out", t["d0"], "gy", 0)
        dgrad("out", "gy", "gd0")
        relu("gd0", "d0")
        wgrad("dec0", t["d1"], "gd0", 1)
        dgrad("dec0", "gd0", "gu0")
        up_bwd("gu0", "gd1", 16, 1)
        relu("gd1", "d1")
        wgrad("dec1", t["d2"], "gd1", 1)
        dgrad("dec1", "gd1", "gu1")
        up_bwd("gu1", "gd2", 32, 2)
        relu("gd2", "d2")
        wgrad("dec2", t["e3"], "gd2", 1)
        dgrad("dec2", "gd2", "gu2")
        up_bwd("gu2", "ge3", 64, 3)
        relu("ge3", "e3")
        wgrad("enc3b", t["a3"], "ge3", 0)
        dgrad("enc3b", "ge3", "ga3")
        relu("ga3", "a3")
        wgrad("enc3a", t["e2"], "ga3", 2)
        dgrad("enc3a", "ga3", "gp2")
        pool_bwd_acc("gp2", "gd2", 32, 3)   # gd2 now holds the gradient of e2
        relu("gd2", "e2")
        wgrad("enc2b", t["a2"], "gd2", 0)
        dgrad("enc2b", "gd2", "ga2")
        relu("ga2", "a2")
        wgrad("enc2a", t["e1"], "ga2", 2)
        dgrad("enc2a", "ga2", "gp1")
        pool_bwd_acc("gp1", "gd1", 16, 2)   # gradient of e1
        relu("gd1", "e1")
        wgrad("enc1b", t["a1"], "gd1", 0)
        dgrad("enc1b", "gd1", "ga1")
        relu("ga1", "a1")
        wgrad("enc1a", t["e0"], "ga1", 2)
        dgrad("enc1a", "ga1", "gp0")
        pool_bwd_acc("gp0", "gd0", 8, 1)    # gradient of e0
        relu("gd0", "e0")
        # first layer, one sample at a time (each has its own log-contrast channel)
        nw0 = self.offsets["enc0"][1]
        for b, (ph, c) in enumerate(zip(phases, contrasts)):
            dy = ctypes.c_void_p(g["gd0"].data_ptr() + 2 * 8 * N * b)
            dw = self._w("enc0", True) if b == 0 else _p(self.tc_dw0)
            db = self._b("enc0", True) if b == 0 else ctypes.c_void_p(self.tc_dw0.data_ptr() + 4 * nw0)
            _check(lib.fftls_nn_tc_conv_phase_backward_weights(_p(ph), dy, dw, db, _I3(*n), 8, float(log_contrast(c)),
                                                               scratch, ns, s), "wgrad enc0")
            if b > 0:
                _check(lib.fftls_nn_add(self._w("enc0", True), _p(self.tc_dw0), nw0, s), "wgrad enc0 sum")
                _check(lib.fftls_nn_add(self._b("enc0", True), ctypes.c_void_p(self.tc_dw0.data_ptr() + 4 * nw0), 8,
                                        s), "bias grad enc0 sum")

    # -- training and prediction -----------------------------------------
    def _train_step_tc(self, group, rate, loss_out):
        """One Adam step on a batch on the tensor cores; the batch's loss into loss_out (device)."""
        phases = [d["phase"] for d in group]
        contrasts = [d["contrast"] for d in group]
        self.forward_tc_batch(phases, contrasts, train=True)
        n = self._tc_grid[0]
        N6 = 6 * n[0] * n[1] * n[2]
        for slot, d in enumerate(group):
            self.tc_target[slot * N6:(slot + 1) * N6].copy_(d["target"].reshape(-1))
        _check(self.lib.fftls_nn_mse(_p(self.tc["y"]), _p(self.tc_target), _p(self.tc_gy), _p(self.tc_loss),
                                     self.tc["y"].numel(), self.stream), "mse")
        loss_out.copy_(self.tc_loss)
        self.backward_tc(phases, contrasts)
        self.adam(rate)

    def train(self, data, epochs: int, lr: float = 5e-4, lr_final: float = 5e-5, seed: int = 0, batch: int = 1,
              tensor_cores: bool = False):
        """Adam on the MSE between prediction and solver fluctuation, `batch` samples (of one grid
        size) per step in a seeded random order (each epoch leaves out the len(data) % batch samples
        its permutation puts last); the learning rate decays geometrically from lr to lr_final (at
        2e-3 the ReLU units of this network die within the first epoch).  tensor_cores: forward and
        backward on the tensor cores (BF16 activations and gradients, FP32 weights and Adam).
        Returns the mean loss of each epoch."""
        torch = self.torch
        rng = np.random.default_rng(seed)
        per = len(data) // batch
        if per < 1:
            raise ValueError("fewer samples than one batch")
        total = epochs * per
        per_epoch = []
        step = 0
        for _ in range(epochs):
            losses = torch.zeros(per, dtype=torch.float64, device=self.dev)
            order = rng.permutation(len(data))
            for j in range(per):
                group = [data[i] for i in order[j * batch:(j + 1) * batch]]
                n = (group[0]["phase"].shape[2], group[0]["phase"].shape[1], group[0]["phase"].shape[0])
                if tensor_cores:
                    self._train_step_tc(group, lr * (lr_final / lr) ** (step / max(1, total - 1)), losses[j:j + 1])
                    step += 1
                    continue
                self._buffers(n, True, batch)
                N6 = 6 * n[0] * n[1] * n[2]
                for slot, d in enumerate(group):
                    if d["phase"].shape != group[0]["phase"].shape:
                        raise ValueError("the samples of a batch must share one grid")
                    self.features(d["phase"], d["contrast"], slot)
                    if batch > 1:
                        self.target[slot * N6:(slot + 1) * N6].copy_(d["target"].reshape(-1))
                self.forward()
                self.loss_and_grad(self.target if batch > 1 else group[0]["target"])
                losses[j:j + 1].copy_(self.loss_buf)
                self.backward()
                rate = lr * (lr_final / lr) ** (step / max(1, total - 1))
                self.adam(rate)
                step += 1
            per_epoch.append(float(losses.mean()))
        self.losses += per_epoch
        return per_epoch

    def initial_strain(self, phase, contrast: float, eps11: float = 1.0, tensor_cores: bool = True):
        """eps^0 (FP64 device tensor [6][n3][n2][n1]) for the load eps11 e1 (x) e1, from the
        tensor-core forward (BF16) or the FP32 one."""
        torch = self.torch
        n = (phase.shape[2], phase.shape[1], phase.shape[0])
        if tensor_cores:
            y = self.forward_tc(phase, contrast)
            scratch = self.tc_mean_scratch
        else:
            self._buffers(n, self._grid[1] if self._grid and self._grid[0] == n else False)
            self.features(phase, contrast)
            y = self.forward()
            scratch = self.mean_scratch
        eps = torch.empty((6,) + tuple(phase.shape), dtype=torch.float64, device=self.dev)
        eb = (ctypes.c_double * 6)(eps11, 0, 0, 0, 0, 0)
        _check(self.lib.fftls_nn_strain_init(_p(y), _p(eps), _I3(*n), eb, float(eps11), _p(scratch), self.stream),
               "strain init")
        # the solver reads eps_init on its own stream
        torch.cuda.synchronize(self.dev)
        return eps


def make_dataset(solver, count: int, L: int, first_seed: int, tol: float = 1e-6, chunk: int = 64,
                 concurrency: int = 8):
    """Solver-generated training samples: the batched recipe at grid L^3 (radius 3-8, fraction
    0.1-0.4, contrast 10-1000), eps_bar = e1 (x) e1, AS with G^R to eta <= tol; target = eps - eps_bar
    (FP32 device tensor [6][N]).  Returns (samples, seconds)."""
    import torch
    lib = _lib()
    specs = MS.batch_recipe(count, first_seed, lengths=(L,))
    out = []
    t0 = time.perf_counter()
    eb = np.diag([1.0, 0.0, 0.0])
    ebv = (ctypes.c_double * 6)(1, 0, 0, 0, 0, 0)
    for c0 in range(0, count, chunk):
        batch = []
        for spec in specs[c0:c0 + chunk]:
            ph, lam, mu, info = MS.batch_sample(spec)
            batch.append({"phase": torch.from_numpy(ph).cuda(solver.device), "lam": lam, "mu": mu, "eps_bar": eb,
                          "contrast": spec["contrast"], "iterations": 0})
        res, st = solver.solve_batched(batch, tol=tol, precision="fp32_refine64", want_strain=True,
                                       device_outputs=True, concurrency=concurrency)
        for b, r in zip(batch, res):
            t = torch.empty((6, L, L, L), dtype=torch.float32, device=b["phase"].device)
            _check(lib.fftls_nn_strain_target(_p(r.strain), _p(t), _I3(L, L, L), ebv, None), "strain target")
            out.append({"phase": b["phase"], "contrast": b["contrast"], "target": t, "iterations": r.iterations,
                        "converged": r.converged})
        torch.cuda.synchronize()
    return out, time.perf_counter() - t0
