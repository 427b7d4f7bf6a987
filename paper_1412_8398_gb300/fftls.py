"""Python binding of the C ABI in ``include/fftls.h`` (ctypes, marshalling only).

Every step of the solve runs in the CUDA library ``_build/libfftls.so``; this
module only converts arrays to pointers.  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.

Array conventions (same as the C ABI):
  * phase images are ``uint8`` with numpy shape (n3, n2, n1) in 3D or
    (n2, n1) in 2D (x1 fastest);
  * strain / stress fields have shape (n_c,) + phase.shape with components
    (11, 22, 33, 23, 13, 12) in 3D or (11, 22, 12) in 2D, tensor (not
    engineering) shear.
Host inputs may be numpy arrays; device inputs may be torch CUDA tensors
(torch is used only to hold device memory and streams).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import build as _build

GREEN = {"MS": 0, "C": 1, "W": 2, "R": 3}
SCHEME = {"DS": 0, "AS": 1}
PRECISION = {"fp64": 0, "fp32_refine64": 1, "fp32": 2}
STOP = {"eta": 0, "maxdelta": 1}

OK, E_INVALID_ARG, E_UNSUPPORTED_SIZE, E_OOM, E_CUDA, E_NOT_CONVERGED, E_DIVERGED, E_TIMEOUT = range(8)


# Fields of one tile-schedule row (fftls_tile_plans / fftls_set_tile_plans), FFTLS_PLAN_FIELDS of them.
PLAN_KEYS = ("precision", "n1", "n2", "n3", "green", "x1_lines", "x1_vb", "x5_lines", "y_w", "z_w", "e_planes",
             "tuned", "y_threads", "z_threads", "x5_vb")


class FftlsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("phase", ctypes.c_void_p),
        ("phase_on_device", ctypes.c_int),
        ("n_phases", ctypes.c_int),
        ("lambda_", ctypes.POINTER(ctypes.c_double)),
        ("mu", ctypes.POINTER(ctypes.c_double)),
        ("lambda0", ctypes.c_double),
        ("mu0", ctypes.c_double),
        ("green", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("eps_bar", ctypes.c_double * 6),
    ]


class _Options(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("stop", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("refine_switch", ctypes.c_double),
        ("eps_init", ctypes.c_void_p),
        ("eps_init_on_device", ctypes.c_int),
        ("fields_on_device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("use_graphs", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("eta_only", ctypes.c_int),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("strain", ctypes.c_void_p),
        ("stress", ctypes.c_void_p),
        ("mean_stress", ctypes.c_double * 6),
        ("mean_strain", ctypes.c_double * 6),
        ("iterations", ctypes.c_int),
        ("iterations_fp32", ctypes.c_int),
        ("final_eta", ctypes.c_double),
        ("final_delta", ctypes.c_double),
        ("eta_history", ctypes.POINTER(ctypes.c_double)),
        ("mean_stress_history", ctypes.POINTER(ctypes.c_double)),
        ("history_capacity", ctypes.c_int),
        ("history_len", ctypes.c_int),
    ]


# Every function declared in include/fftls.h, with its ctypes signature.
_SIGNATURES = {
    "fftls_default_options": (None, [ctypes.POINTER(_Options)]),
    "fftls_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "fftls_destroy": (None, [ctypes.c_void_p]),
    "fftls_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Problem), ctypes.POINTER(_Options),
                                   ctypes.POINTER(_Result)]),
    "fftls_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.POINTER(_Options),
                                           ctypes.POINTER(_Result)]),
    "fftls_effective_stiffness": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Problem),
                                                 ctypes.POINTER(_Options), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_int)]),
    "fftls_reference_medium": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
    "fftls_supported_length": (ctypes.c_int, [ctypes.c_int]),
    "fftls_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_char_p),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
    "fftls_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "fftls_tile_plans": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "fftls_set_tile_plans": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "fftls_solve_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Problem), ctypes.c_int,
                                           ctypes.POINTER(_Options), ctypes.POINTER(_Result),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "fftls_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fftls_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libfftls.so (raises if absent: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def status_name(s: int) -> str:
    names = ["FFTLS_OK", "FFTLS_E_INVALID_ARG", "FFTLS_E_UNSUPPORTED_SIZE", "FFTLS_E_OOM", "FFTLS_E_CUDA",
             "FFTLS_E_NOT_CONVERGED", "FFTLS_E_DIVERGED", "FFTLS_E_TIMEOUT"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


@dataclass
class SolveResult:
    status: int
    strain: object
    stress: object
    mean_stress: np.ndarray
    mean_strain: np.ndarray
    iterations: int
    iterations_fp32: int
    final_eta: float
    final_delta: float
    eta_history: np.ndarray
    mean_stress_history: np.ndarray
    message: str = ""

    @property
    def converged(self) -> bool:
        return self.status == OK


def _key(table, v, what):
    if isinstance(v, str):
        try:
            return table[v]
        except KeyError:
            raise ValueError(f"unknown {what} {v!r}; expected one of {sorted(table)}")
    return int(v)


class Solver:
    """One library context on one CUDA device (owns device workspaces)."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.fftls_create(ctypes.byref(h), int(device))
        if st != OK:
            raise FftlsError(st, f"cannot create a context on CUDA device {device}")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fftls_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self.lib.fftls_last_error(self.handle).decode()

    # ------------------------------------------------------------------
    def _problem(self, phase, lam, mu, eps_bar, green, scheme, lam0, mu0):
        shape = tuple(phase.shape)
        dim = len(shape)
        if dim not in (2, 3):
            raise ValueError("phase must be 2D (n2, n1) or 3D (n3, n2, n1)")
        p = _Problem()
        p.dim = dim
        n = list(reversed(shape)) + [1] * (3 - dim)
        p.n[:] = n
        on_dev = _is_torch(phase) and phase.is_cuda
        if _is_torch(phase):
            if not phase.is_contiguous() or str(phase.dtype) != "torch.uint8":
                raise ValueError("phase tensor must be contiguous uint8")
        else:
            phase = np.ascontiguousarray(phase, dtype=np.uint8)
        p.phase = _ptr(phase).value
        p.phase_on_device = 1 if on_dev else 0
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
        if lam.size != mu.size:
            raise ValueError("lambda and mu need one entry per phase")
        p.n_phases = lam.size
        p.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.mu = mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.lambda0 = math.nan if lam0 is None else float(lam0)
        p.mu0 = math.nan if mu0 is None else float(mu0)
        p.green = _key(GREEN, green, "green")
        p.scheme = _key(SCHEME, scheme, "scheme")
        eb = _eps_bar_vector(eps_bar, dim)
        p.eps_bar[:] = list(eb) + [0.0] * (6 - eb.size)
        keep = (phase, lam, mu)
        return p, keep, on_dev

    def _options(self, tol, max_iter, precision, stop, refine_switch, eps_init, fields_on_device, stream,
                 use_graphs, profile, autotune=True, eta_only=False):
        o = _Options()
        self.lib.fftls_default_options(ctypes.byref(o))
        o.tol = float(tol)
        o.max_iter = int(max_iter)
        o.precision = _key(PRECISION, precision, "precision")
        o.stop = _key(STOP, stop, "stop rule")
        o.refine_switch = float(refine_switch)
        o.fields_on_device = 1 if fields_on_device else 0
        o.use_graphs = 1 if use_graphs else 0
        o.profile = 1 if profile else 0
        o.autotune = 1 if autotune else 0
        o.eta_only = 1 if eta_only else 0
        keep = None
        if eps_init is not None:
            if _is_torch(eps_init):
                if str(eps_init.dtype) != "torch.float64" or not eps_init.is_contiguous():
                    raise ValueError("eps_init tensor must be contiguous float64")
                o.eps_init_on_device = 1 if eps_init.is_cuda else 0
                keep = eps_init
            else:
                keep = np.ascontiguousarray(eps_init, dtype=np.float64)
                o.eps_init_on_device = 0
            o.eps_init = _ptr(keep).value
        if stream is not None:
            o.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        return o, keep

    def solve(self, phase, lam, mu, eps_bar, green="R", scheme="AS", lam0=None, mu0=None, tol=1e-8,
              max_iter=1000, precision="fp64", stop="eta", refine_switch=0.0, eps_init=None,
              want_strain=True, want_stress=True, history=True, device_outputs=None, stream=None,
              use_graphs=True, profile=False, autotune=True, eta_only=False, raise_on_error=True) -> SolveResult:
        """Solve one load case; see fftls_solve in include/fftls.h."""
        p, keep_p, on_dev = self._problem(phase, lam, mu, eps_bar, green, scheme, lam0, mu0)
        if device_outputs is None:
            device_outputs = on_dev
        o, keep_o = self._options(tol, max_iter, precision, stop, refine_switch, eps_init, device_outputs,
                                  stream, use_graphs, profile, autotune, eta_only)
        r, out = self._outputs(p, phase.shape, want_strain, want_stress, history, max_iter, device_outputs)
        st = self.lib.fftls_solve(self.handle, ctypes.byref(p), ctypes.byref(o), ctypes.byref(r))
        msg = self.last_error()
        if st not in (OK, E_NOT_CONVERGED, E_DIVERGED):
            raise FftlsError(st, msg)
        if raise_on_error and st == E_DIVERGED:
            raise FftlsError(st, msg)
        del keep_p, keep_o
        return self._collect(st, r, out, msg)

    def _outputs(self, p, grid_shape, want_strain, want_stress, history, max_iter, device_outputs, r=None):
        """Caller-owned result buffers of one solve (numpy, or torch on the device)."""
        nc = 6 if p.dim == 3 else 3
        shape = (nc,) + tuple(grid_shape)
        if r is None:
            r = _Result()
        strain = stress = None
        if device_outputs:
            import torch
            dev = torch.device("cuda", self.device)
            if want_strain:
                strain = torch.empty(shape, dtype=torch.float64, device=dev)
            if want_stress:
                stress = torch.empty(shape, dtype=torch.float64, device=dev)
        else:
            if want_strain:
                strain = np.empty(shape, dtype=np.float64)
            if want_stress:
                stress = np.empty(shape, dtype=np.float64)
        r.strain = _ptr(strain).value if strain is not None else None
        r.stress = _ptr(stress).value if stress is not None else None
        cap = int(max_iter) if history else 0
        eh = np.zeros(cap, dtype=np.float64)
        mh = np.zeros((cap, nc), dtype=np.float64)
        if cap:
            r.eta_history = eh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            r.mean_stress_history = mh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.history_capacity = cap
        return r, (strain, stress, eh, mh, nc)

    @staticmethod
    def _collect(st, r, out, msg):
        strain, stress, eh, mh, nc = out
        n = r.history_len
        return SolveResult(
            status=st, strain=strain, stress=stress,
            mean_stress=np.array(r.mean_stress[:nc]), mean_strain=np.array(r.mean_strain[:nc]),
            iterations=r.iterations, iterations_fp32=r.iterations_fp32, final_eta=r.final_eta,
            final_delta=r.final_delta, eta_history=eh[:n].copy(), mean_stress_history=mh[:n].copy(),
            message=msg)

    def solve_batched(self, samples, green="R", scheme="AS", tol=1e-6, max_iter=3000, precision="fp32_refine64",
                      stop="eta", refine_switch=0.0, concurrency=0, want_strain=False, want_stress=False,
                      history=False, device_outputs=False, use_graphs=True, autotune=True):
        """Solve independent problems concurrently (fftls_solve_batched in include/fftls.h).

        samples: sequence of dicts with keys phase, lam, mu, eps_bar and optionally lam0, mu0,
        green, scheme (overriding the shared arguments).  Returns (list of SolveResult, status).
        """
        count = len(samples)
        probs = (_Problem * max(count, 1))()
        results = (_Result * max(count, 1))()
        statuses = (ctypes.c_int * max(count, 1))()
        keeps, outs = [], []
        for i, smp in enumerate(samples):
            p, keep, on_dev = self._problem(smp["phase"], smp["lam"], smp["mu"], smp["eps_bar"],
                                            smp.get("green", green), smp.get("scheme", scheme),
                                            smp.get("lam0"), smp.get("mu0"))
            probs[i] = p
            keeps.append((keep, smp["phase"]))
            _, out = self._outputs(p, smp["phase"].shape, want_strain, want_stress, history, max_iter,
                                   device_outputs, r=results[i])
            outs.append(out)
        o, keep_o = self._options(tol, max_iter, precision, stop, refine_switch, None, device_outputs, None,
                                  use_graphs, False, autotune)
        st = self.lib.fftls_solve_batched(self.handle, probs, count, ctypes.byref(o), results, statuses,
                                          int(concurrency))
        msg = self.last_error()
        if st not in (OK, E_NOT_CONVERGED, E_DIVERGED):
            raise FftlsError(st, msg)
        res = [self._collect(statuses[i], results[i], outs[i], "") for i in range(count)]
        del keeps, keep_o
        return res, st

    def effective_stiffness(self, phase, lam, mu, green="R", scheme="AS", lam0=None, mu0=None, tol=1e-8,
                            max_iter=1000, precision="fp64", stop="eta", refine_switch=0.0):
        """Mandel C~ (n_c x n_c) and the iteration count of each unit load."""
        p, keep_p, _ = self._problem(phase, lam, mu, np.zeros(6), green, scheme, lam0, mu0)
        o, keep_o = self._options(tol, max_iter, precision, stop, refine_switch, None, False, None, True, False)
        nc = 6 if p.dim == 3 else 3
        C = np.zeros(36, dtype=np.float64)
        its = np.zeros(6, dtype=np.int32)
        st = self.lib.fftls_effective_stiffness(self.handle, ctypes.byref(p), ctypes.byref(o),
                                                C.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                its.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if st not in (OK, E_NOT_CONVERGED):
            raise FftlsError(st, self.last_error())
        return C[: nc * nc].reshape(nc, nc), its[:nc].copy(), st

    def counters(self):
        """(kernels launched, CUDA graphs launched) on this context so far."""
        k = ctypes.c_longlong()
        g = ctypes.c_longlong()
        self.lib.fftls_counters(self.handle, ctypes.byref(k), ctypes.byref(g))
        return k.value, g.value

    def tile_plans(self) -> list:
        """Tile schedules held by this context (see fftls_tile_plans), one dict per grid and precision."""
        n = ctypes.c_int(0)
        self.lib.fftls_tile_plans(self.handle, None, ctypes.byref(n))
        keys = PLAN_KEYS
        w = len(keys)
        rows = (ctypes.c_int * (w * max(n.value, 1)))()
        self.lib.fftls_tile_plans(self.handle, rows, ctypes.byref(n))
        return [dict(zip(keys, rows[w * i:w * i + w])) for i in range(n.value)]

    def set_tile_plans(self, plans: list) -> None:
        """Import schedules (dicts as returned by tile_plans) for later solves (see fftls_set_tile_plans)."""
        keys = PLAN_KEYS
        w = len(keys)
        rows = (ctypes.c_int * (w * max(len(plans), 1)))()
        for i, p in enumerate(plans):
            for j, k in enumerate(keys):
                rows[w * i + j] = int(p.get(k, 1 if k == "x5_vb" else 0))
        st = self.lib.fftls_set_tile_plans(self.handle, rows, len(plans))
        if st:
            raise FftlsError(st, self.last_error())

    def profile(self) -> dict:
        """Per-kernel (total ms, launches) of the last solve run with profile=True."""
        cap = ctypes.c_int(32)
        names = (ctypes.c_char_p * 32)()
        ms = (ctypes.c_double * 32)()
        cnt = (ctypes.c_int * 32)()
        self.lib.fftls_profile(self.handle, names, ms, cnt, ctypes.byref(cap))
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(cap.value)}


def _eps_bar_vector(eps_bar, dim):
    e = np.asarray(eps_bar, dtype=np.float64)
    if e.ndim == 2:
        if dim == 3:
            return np.array([e[0, 0], e[1, 1], e[2, 2], e[1, 2], e[0, 2], e[0, 1]])
        return np.array([e[0, 0], e[1, 1], e[0, 1]])
    nc = 6 if dim == 3 else 3
    if e.size < nc:
        raise ValueError(f"eps_bar needs {nc} components")
    return e[:nc].copy()


def reference_medium(lam, mu, dim, scheme="AS"):
    """Default (lambda0, mu0) from the library (eq. refAcc / eq. ref)."""
    lib = load_library()
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    p = _Problem()
    p.dim = dim
    p.n_phases = lam.size
    p.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.mu = mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.scheme = _key(SCHEME, scheme, "scheme")
    l0 = ctypes.c_double()
    m0 = ctypes.c_double()
    st = lib.fftls_reference_medium(ctypes.byref(p), ctypes.byref(l0), ctypes.byref(m0))
    if st != OK:
        raise FftlsError(st, "default reference medium degenerates")
    return l0.value, m0.value


def supported_length(L: int) -> bool:
    return load_library().fftls_supported_length(int(L)) == OK


def components_to_tensor(field_nc, dim):
    """(n_c, grid) component field -> (d, d, grid) full tensor field (numpy)."""
    f = np.asarray(field_nc)
    grid = f.shape[1:]
    t = np.zeros((dim, dim) + grid, dtype=f.dtype)
    if dim == 3:
        t[0, 0], t[1, 1], t[2, 2] = f[0], f[1], f[2]
        t[1, 2] = t[2, 1] = f[3]
        t[0, 2] = t[2, 0] = f[4]
        t[0, 1] = t[1, 0] = f[5]
    else:
        t[0, 0], t[1, 1] = f[0], f[1]
        t[0, 1] = t[1, 0] = f[2]
    return t
