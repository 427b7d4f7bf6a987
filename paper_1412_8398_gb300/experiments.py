"""Drivers of the paper's numerical experiments on top of the solver (Sec. 6).

Each driver only chooses inputs and collects outputs of ``fftls.Solver``; the
iteration itself is the library's.  Workloads are synthetic (Boolean models,
periodic spheres) built by ``microstructure``.

* ``iterations_vs_reference``: N(E0), the iterations to eta <= tol as the
  reference Young's modulus E0 varies at fixed nu0 (Sec. 6.2, the curves whose
  minimum defines the optimal reference medium).
* ``optimal_reference``: the E0 minimising N(E0), found by a golden-section
  search on log E0 (the paper minimises N(E0) numerically; the search method is
  this library's reading).
* ``iterations_vs_contrast``: iterations to eta <= tol against the contrast chi
  with the default reference media (Sec. 6.3: AS iterations grow like sqrt(chi)
  for chi >> 1, DS like chi).
* ``modulus_history``: the apparent modulus <sigma_11> / eps_bar_11 after each
  iteration (Sec. 6.4, convergence of C~_1111 with the iterations).
* ``effective_stiffness``: the full C~ from the six unit loads (eq. a2).
"""
from __future__ import annotations

import math

import numpy as np

from . import microstructure as MS


def lame(E: float, nu: float):
    return MS.lame_from_young(E, nu)


def iterations_vs_reference(solver, phase, lam, mu, E0_values, nu0=0.25, green="R", scheme="AS", tol=1e-8,
                            max_iter=5000, precision="fp64", eps_bar=None):
    """[(E0, iterations, converged)] for each reference Young's modulus E0 (nu0 fixed)."""
    d = phase.ndim
    eb = np.diag([1.0] + [0.0] * (d - 1)) if eps_bar is None else eps_bar
    out = []
    for E0 in E0_values:
        l0, m0 = lame(float(E0), nu0)
        r = solver.solve(phase, lam, mu, eb, green, scheme, lam0=l0, mu0=m0, tol=tol, max_iter=max_iter,
                         precision=precision, want_strain=False, want_stress=False, history=False,
                         raise_on_error=False)
        out.append((float(E0), int(r.iterations), bool(r.converged)))
    return out


def optimal_reference(solver, phase, lam, mu, E0_lo, E0_hi, nu0=0.25, green="R", scheme="AS", tol=1e-8,
                      max_iter=5000, precision="fp64", evaluations=12):
    """(E0*, N(E0*), evaluations) by golden-section search on log E0 in [E0_lo, E0_hi]."""
    cache = {}

    def N(logE):
        if logE not in cache:
            (_, its, conv), = iterations_vs_reference(solver, phase, lam, mu, [math.exp(logE)], nu0, green, scheme,
                                                      tol, max_iter, precision)
            cache[logE] = its if conv else max_iter + 1
        return cache[logE]

    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = math.log(E0_lo), math.log(E0_hi)
    c, e = b - g * (b - a), a + g * (b - a)
    for _ in range(max(1, evaluations - 2)):
        if N(c) <= N(e):
            b, e = e, c
            c = b - g * (b - a)
        else:
            a, c = c, e
            e = a + g * (b - a)
    best = min(cache, key=lambda k: (cache[k], k))
    return math.exp(best), cache[best], sorted((math.exp(k), v) for k, v in cache.items())


def iterations_vs_contrast(solver, phase, chis, nu=0.25, green="R", scheme="AS", tol=1e-8, max_iter=20000,
                           precision="fp64"):
    """[(chi, iterations, converged)]: matrix E = 1, inclusions E = chi, same nu, default C0."""
    d = phase.ndim
    eb = np.diag([1.0] + [0.0] * (d - 1))
    out = []
    for chi in chis:
        lam, mu = MS.young_poisson_phases([(1.0, nu), (float(chi), nu)])
        r = solver.solve(phase, lam, mu, eb, green, scheme, tol=tol, max_iter=max_iter, precision=precision,
                         want_strain=False, want_stress=False, history=False, raise_on_error=False)
        out.append((float(chi), int(r.iterations), bool(r.converged)))
    return out


def modulus_history(solver, phase, lam, mu, green="R", scheme="AS", iterations=50, precision="fp64", **kw):
    """<sigma_11> after each eta evaluation for eps_bar = e1 (x) e1 (the apparent C~_1111)."""
    d = phase.ndim
    eb = np.diag([1.0] + [0.0] * (d - 1))
    r = solver.solve(phase, lam, mu, eb, green, scheme, tol=0.0, max_iter=iterations, precision=precision,
                     want_strain=False, want_stress=False, raise_on_error=False, **kw)
    return r.mean_stress_history[:, 0].copy()


def effective_stiffness(solver, phase, lam, mu, green="R", scheme="AS", tol=1e-8, precision="fp64"):
    """Mandel C~ from the six (2D: three) unit loads."""
    C, its, _ = solver.effective_stiffness(phase, lam, mu, green=green, scheme=scheme, tol=tol, precision=precision)
    return C, its
