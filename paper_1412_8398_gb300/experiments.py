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
* ``four_cell``: the 2D quasi-rigid square inclusion of Sec. 5.1 (chi = 1e3, eq. load2d),
  sigma_12 around the inclusion corners.
* ``four_cell_delta_floor``: the FP64 round-off floor of Sec. 5.1's max-delta stop rule against L.
* ``periodic_sphere_modulus``: C~_1111 of one periodic spherical pore-like inclusion
  (f = 20 %, chi = 1e-4) of Sec. 5.3 at grid length L.
* ``boolean_reference_study``: N(E0) and its minimum on the 64^3 Boolean model of Sec. 6
  (743 spheres of diameter 5, f = 17 %).
* ``accelerated_rate_study``: the initial eta, decades and asymptotic eta ratio of the accelerated
  scheme per operator on that model (where its iterations go);
* ``modulus_rate_study``: Sec. 6.4, the apparent C~_1111 after each iteration of AS with each
  operator (each at its optimal E0 on the 64^3 model) on the Sec. 6 Boolean model refined to
  L^3, and the iterations after which it stays within 1 % of its converged value.
* ``eight_cube``: the 3D analogue of the four-cell (Sec. 5.2): a centred cube inclusion of side
  L/2 (f = 12.5 %, chi = 1e3) under eps_bar_12 = eps_bar_21 = 1/2, sigma_12 on the section
  x3 = -0.2461 close to the inclusion's face: mirror asymmetry, corner peaks, ripple inside the
  inclusion, and the fraction of voxels above 8.5.

The paper's phases (Sec. 2): nu = 0.25 in both phases; matrix kappa = 1, mu = 0.6
(lambda = 0.4 in 2D, 0.6 in 3D); the inclusion's moduli are chi times the matrix's.
``python -m paper_1412_8398_gb300.experiments [--study NAME ...]`` runs the studies (all five by
default) and prints one JSON summary per case.
"""
from __future__ import annotations

import math

import numpy as np

from . import microstructure as MS


def lame(E: float, nu: float):
    return MS.lame_from_young(E, nu)


def iterations_vs_reference(solver, phase, lam, mu, E0_values, nu0=0.25, green="R", scheme="AS", tol=1e-8,
                            max_iter=5000, precision="fp64", eps_bar=None, eta_only=False):
    """[(E0, iterations, converged)] for each reference Young's modulus E0 (nu0 fixed).
    eta_only: stop on eta alone, the paper's criterion (see fftls_options.eta_only)."""
    d = phase.ndim
    eb = np.diag([1.0] + [0.0] * (d - 1)) if eps_bar is None else eps_bar
    out = []
    for E0 in E0_values:
        l0, m0 = lame(float(E0), nu0)
        r = solver.solve(phase, lam, mu, eb, green, scheme, lam0=l0, mu0=m0, tol=tol, max_iter=max_iter,
                         precision=precision, want_strain=False, want_stress=False, history=False,
                         raise_on_error=False, eta_only=eta_only)
        out.append((float(E0), int(r.iterations), bool(r.converged)))
    return out


def optimal_reference(solver, phase, lam, mu, E0_lo, E0_hi, nu0=0.25, green="R", scheme="AS", tol=1e-8,
                      max_iter=5000, precision="fp64", evaluations=12, eta_only=False):
    """(E0*, N(E0*), evaluations) by golden-section search on log E0 in [E0_lo, E0_hi]."""
    cache = {}

    def N(logE):
        if logE not in cache:
            (_, its, conv), = iterations_vs_reference(solver, phase, lam, mu, [math.exp(logE)], nu0, green, scheme,
                                                      tol, max_iter, precision, eta_only=eta_only)
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


def paper_phases(chi: float, dim: int):
    """(lambda, mu) of the matrix and of the inclusions in the paper's convention (Sec. 2)."""
    lam1 = 0.4 if dim == 2 else 0.6
    return np.array([lam1, chi * lam1]), np.array([0.6, chi * 0.6])


def four_cell(solver, L=512, green="R", chi=1e3, tol=None, max_iter=20000, window=0.04, threshold=3.5):
    """Sec. 5.1: centred square inclusion of side L/2 (the simplified four-cell), eps_bar_12 =
    eps_bar_21 = 1/2 (eq. load2d), AS, stop when no strain or stress value moves by more than tol
    between iterations.  Returns sigma_12 statistics in the squares of half-width `window` (in
    cell lengths) around the four inclusion corners.  tol defaults to the paper's 2e-13 up to
    L = 512 and to 1e-12 above: the FP64 round-off floor of the largest change per iteration is
    2.4-9e-13 at L = 512..2048 (four_cell_delta_floor), so 2e-13 is met only on a favourable
    fluctuation of the round-off."""
    if tol is None:
        tol = 2e-13 if L <= 512 else 1e-12
    ph = MS.square_inclusion(L, 2)
    lam, mu = paper_phases(chi, 2)
    eb = np.array([[0.0, 0.5], [0.5, 0.0]])
    r = solver.solve(ph, lam, mu, eb, green, "AS", tol=tol, max_iter=max_iter, precision="fp64", stop="maxdelta",
                     want_strain=False, history=False, raise_on_error=False)
    s12 = np.asarray(r.stress[2])
    h = int(round(window * L))
    c_lo, c_hi = L // 4, L // 4 + L // 2
    stats = []
    for cy in (c_lo, c_hi):
        for cx in (c_lo, c_hi):
            w = s12[cy - h:cy + h, cx - h:cx + h]
            stats.append({"corner": [cx, cy], "max": float(w.max()), "min": float(w.min()),
                          "frac_above": float(np.mean(w > threshold))})
    return {"L": L, "green": green, "iterations": int(r.iterations), "converged": bool(r.converged),
            "max_sigma12_near_corners": max(q["max"] for q in stats),
            "frac_above_threshold_near_corners": float(np.mean([q["frac_above"] for q in stats])),
            "frac_above_threshold_whole_cell": float(np.mean(s12 > threshold)),
            "mean_sigma12": float(s12.mean()), "corners": stats}


def four_cell_delta_floor(solver, L=1024, green="R", chi=1e3, chunk=2000, chunks=10):
    """Sec. 5.1's stop rule at large L: the largest change of a strain or stress value between two
    iterations (the max-delta rule, 2e-13 in the paper) after every `chunk` accelerated iterations
    of the four-cell, up to chunk * chunks iterations (each chunk continues from the previous field:
    the accelerated scheme carries no other state).  Where the sequence stops decreasing it has
    reached its FP64 round-off floor; returns the sequence, that floor (the smallest value seen) and
    the corner statistics of the final field."""
    ph = MS.square_inclusion(L, 2)
    lam, mu = paper_phases(chi, 2)
    eb = np.array([[0.0, 0.5], [0.5, 0.0]])
    deltas, eps, its = [], None, 0
    for _ in range(chunks):
        r = solver.solve(ph, lam, mu, eb, green, "AS", tol=0.0, max_iter=chunk, precision="fp64", stop="maxdelta",
                         want_stress=False, history=False, raise_on_error=False, eps_init=eps)
        eps = np.asarray(r.strain).copy()
        its += int(r.iterations)
        deltas.append(float(r.final_delta))
        if len(deltas) >= 3 and deltas[-1] >= 0.9 * min(deltas[:-1]):
            break  # no longer decreasing: the round-off floor
    return {"L": L, "green": green, "iterations": its, "max_delta_per_chunk": deltas, "floor": min(deltas),
            "reaches_2e-13": min(deltas) < 2e-13}


def periodic_sphere_modulus(solver, L, green="R", f=0.2, chi=1e-4, tol=2e-10, max_iter=200000):
    """Sec. 5.3: C~_1111 = <sigma_11> under eps_bar = e1 (x) e1 for one periodic sphere of volume
    fraction f and contrast chi, AS, max-delta stop at tol (FP64)."""
    ph = MS.periodic_sphere(L, f)
    lam, mu = paper_phases(chi, 3)
    r = solver.solve(ph, lam, mu, np.diag([1.0, 0.0, 0.0]), green, "AS", tol=tol, max_iter=max_iter,
                     precision="fp64", stop="maxdelta", want_strain=False, want_stress=False, history=False,
                     raise_on_error=False)
    return {"L": L, "green": green, "C1111": float(r.mean_stress[0]), "iterations": int(r.iterations),
            "converged": bool(r.converged), "fraction": float(ph.mean())}


def boolean_reference_study(solver, chi=1e-5, green="R", scheme="AS", tol=1e-8, seed=39, eta_only=True,
                            E0_grid=(0.02, 0.04, 0.06, 0.09, 0.13, 0.2, 0.3, 0.5)):
    """Sec. 6: a 64^3 Boolean model of spheres of diameter 5 (seed 39: 746 spheres, f = 16.9 %, an
    instance like the paper's 743 spheres and 17 %), N(E0) on a grid and the golden-section optimum
    (nu0 = 0.25), iterations to eta <= tol (eta_only: the paper's criterion)."""
    ph, info = MS.boolean_spheres((64, 64, 64), 2.5, 0.17, seed=seed)
    lam, mu = paper_phases(chi, 3)
    sweep = iterations_vs_reference(solver, ph, lam, mu, E0_grid, 0.25, green, scheme, tol, eta_only=eta_only)
    E0, N, seen = optimal_reference(solver, ph, lam, mu, E0_grid[0], E0_grid[-1], 0.25, green, scheme, tol,
                                    evaluations=14, eta_only=eta_only)
    return {"chi": chi, "green": green, "scheme": scheme, "eta_only": eta_only, "spheres": int(info["n_centers"]),
            "fraction": float(info["fraction"]), "sweep": sweep, "optimal_E0": E0, "optimal_iterations": N}


def accelerated_rate_study(solver, chi=1e-5, greens=("R", "C", "W", "MS"), E0_grid=(0.03, 0.05, 0.07, 0.09, 0.12),
                           tol=1e-8, max_iter=1500, seed=39, looser=(256.0, 512.0)):
    """Where the accelerated scheme's iterations go on the Sec. 6 instance (64^3, 17 %, chi): per
    operator and reference Young's modulus E0 (nu0 = 0.25, FP64, the paper's eta-only criterion), the
    initial eta, the decades from it to tol, the asymptotic eta ratio per iteration (geometric mean
    over the last 100 iterations), the iterations to tol, and the iterations to thresholds `looser`
    times tol (a test of readings of eta's normalisation)."""
    ph, info = MS.boolean_spheres((64, 64, 64), 2.5, 0.17, seed=seed)
    lam, mu = paper_phases(chi, 3)
    eb = np.diag([1.0, 0.0, 0.0])
    rows = []
    for g in greens:
        for E0 in E0_grid:
            l0, m0 = lame(float(E0), 0.25)
            r = solver.solve(ph, lam, mu, eb, g, "AS", lam0=l0, mu0=m0, tol=tol, max_iter=max_iter, precision="fp64",
                             want_strain=False, want_stress=False, history=True, raise_on_error=False, eta_only=True)
            eta = np.asarray(r.eta_history, dtype=np.float64)
            n = eta.size
            k0 = max(0, n - 101)
            ratio = float((eta[-1] / eta[k0]) ** (1.0 / (n - 1 - k0))) if n - 1 > k0 and eta[k0] > 0 else float("nan")
            to = {f"x{int(f)}": int(np.argmax(eta <= f * tol)) + 1 if (eta <= f * tol).any() else None for f in looser}
            rows.append({"green": g, "E0": float(E0), "iterations": int(r.iterations), "converged": bool(r.converged),
                         "eta0": float(eta[0]), "decades": float(np.log10(eta[0] / tol)), "ratio": ratio,
                         "iterations_to_looser": to})
    return {"chi": chi, "tol": tol, "spheres": int(info["n_centers"]), "fraction": float(info["fraction"]),
            "rows": rows}


def boolean_model(L: int, seed: int = 39):
    """The Sec. 6 Boolean model (spheres of diameter 5 on 64^3, f = 17 %) at L^3: the generator draws
    the same number of centres at the same relative positions for any L when the radius scales with
    L (seed 39: 746 spheres), so L = 256 and 512 are refinements of the same microstructure."""
    return MS.boolean_spheres((L, L, L), 2.5 * L / 64.0, 0.17, seed=seed)


def settle_iteration(history, final, rel=1e-2):
    """First iteration k after which every estimate stays within rel of `final` (len(history) if none)."""
    bad = np.nonzero(np.abs(np.asarray(history) - final) > rel * abs(final))[0]
    return int(bad[-1]) + 1 if bad.size else 0


def modulus_rate_study(solver, L, chi, greens=("MS", "C", "W", "R"), nu0=0.25, tol=1e-6, max_iter=20000,
                       E0=None, search_evaluations=12, rel=1e-2):
    """Sec. 6.4: C~_1111 = <sigma_11> after each iteration for eps_bar = e1 (x) e1, AS, on the Boolean
    model at L^3.  The reference Young's modulus of each operator is its golden-section optimum on the
    64^3 model at the same contrast (eta <= 1e-8, eta alone), unless E0 = {green: E0} is given; the
    search brackets are the matrix's and the inclusions' moduli.  Each run iterates to eta <= tol
    (FP32 bulk, FP64 certification) and reports the iterations after which the estimate stays within
    rel of its converged value, and the largest relative deviation after iteration 5."""
    lam, mu = paper_phases(chi, 3)
    E = [9 * (l + 2 * m / 3) * m / (3 * (l + 2 * m / 3) + m) for l, m in zip(lam, mu)]
    lo, hi = min(E), max(E)
    ph, info = boolean_model(L)
    out = {"L": L, "chi": chi, "fraction": float(info["fraction"]), "spheres": int(info["n_centers"]), "schemes": {}}
    ph64 = boolean_model(64)[0] if E0 is None else None
    for g in greens:
        if E0 is not None and g in E0:
            e0 = float(E0[g])
        else:
            e0, _, _ = optimal_reference(solver, ph64, lam, mu, lo, hi, nu0, g, "AS", 1e-8,
                                         evaluations=search_evaluations, eta_only=True)
        l0, m0 = lame(e0, nu0)
        r = solver.solve(ph, lam, mu, np.diag([1.0, 0.0, 0.0]), g, "AS", lam0=l0, mu0=m0, tol=tol,
                         max_iter=max_iter, precision="fp32_refine64", want_strain=False, want_stress=False,
                         history=True, raise_on_error=False)
        h = r.mean_stress_history[:, 0]
        final = float(r.mean_stress[0])
        dev = np.abs(h[5:] - final) / abs(final) if h.size > 5 else np.zeros(1)
        out["schemes"][g] = {"E0": e0, "iterations": int(r.iterations), "converged": bool(r.converged),
                             "C1111": final, "settle_1pct": settle_iteration(h, final, rel),
                             "max_dev_after_5": float(dev.max()), "first_10": [float(v) for v in h[:10]]}
    return out


def section_index(L: int, x3: float = -0.2461) -> int:
    """Voxel plane nearest to the section x3 (cell [-1/2, 1/2)^3, voxel i at x = -1/2 + i / L;
    x3 = -0.2461 is the second voxel plane of the inclusion at L = 256, 512, 1024)."""
    return int(round((0.5 + x3) * L))


def mirror_asymmetry(s12):
    """max |sigma_12 - M sigma_12| / max |sigma_12| over the cube's mirrors x_i -> -x_i and the
    swap x1 <-> x2 (index i -> L - 1 - i about the cube's centre); sigma_12 is invariant under
    each for the load eps_bar_12 (a reflection flips the sign of eps_bar_12 and of sigma_12)."""
    m = np.abs(s12).max()
    maps = [s12[:, :, ::-1], s12[:, ::-1, :], s12[::-1, :, :], np.swapaxes(s12, 1, 2)] if s12.ndim == 3 else \
        [s12[:, ::-1], s12[::-1, :], s12.T]
    return max(float(np.abs(s12 - t).max()) for t in maps) / m


def eight_cube(solver, L=128, green="R", chi=1e3, tol=1e-12, max_iter=100000, x3=-0.2461, threshold=8.5,
               window=0.04, precision="fp64"):
    """Sec. 5.2: the centred cube inclusion of side L/2, eps_bar_12 = eps_bar_21 = 1/2, AS, iterated
    until no strain or stress value moves by more than tol (FP64: round-off).  Returns statistics of
    sigma_12: on the section plane (its maximum, its mirror asymmetry, the peaks in squares of
    half-width `window` around the four corners of the inclusion's cross-section and their spread,
    the ripple inside the inclusion = mean |second difference along x1| / mean |sigma_12| away from
    the interface) and over the volume (mirror asymmetry, fraction of voxels above `threshold`)."""
    ph = MS.square_inclusion(L, 3)
    lam, mu = paper_phases(chi, 3)
    eb = np.zeros((3, 3))
    eb[0, 1] = eb[1, 0] = 0.5
    r = solver.solve(ph, lam, mu, eb, green, "AS", tol=tol, max_iter=max_iter, precision=precision,
                     stop="maxdelta", want_strain=False, history=False, raise_on_error=False)
    s12 = np.asarray(r.stress[5])  # [x3][x2][x1]
    z = section_index(L, x3)
    sec = s12[z]
    lo, hi = L // 4, L // 4 + L // 2
    h = max(1, int(round(window * L)))
    peaks = [float(sec[cy - h:cy + h, cx - h:cx + h].max()) for cy in (lo, hi) for cx in (lo, hi)]
    inner = sec[lo + 2:hi - 2, lo + 2:hi - 2]
    ripple = float(np.abs(np.diff(inner, 2, axis=1)).mean() / np.abs(inner).mean())
    return {"L": L, "green": green, "iterations": int(r.iterations), "converged": bool(r.converged),
            "section_plane": z, "max_sigma12_section": float(sec.max()),
            "mirror_asymmetry_section": mirror_asymmetry(sec), "mirror_asymmetry_volume": mirror_asymmetry(s12),
            "corner_peaks": peaks, "corner_spread": (max(peaks) - min(peaks)) / max(peaks),
            "ripple_inside": ripple, "frac_above_threshold": float(np.mean(s12 > threshold)),
            "mean_sigma12": float(s12.mean())}


def main(argv=None):
    import argparse
    import json

    from . import fftls
    ap = argparse.ArgumentParser(description="the paper's studies on the GPU path, one JSON line per case")
    ap.add_argument("--study", action="append",
                    choices=["four_cell", "four_cell_floor", "periodic_sphere", "eight_cube", "boolean_reference",
                             "modulus_rate", "accelerated_rate"],
                    help="run only these studies (repeatable; default: all)")
    ap.add_argument("--cube-sizes", default="128,256", help="grid lengths of the eight-cube study")
    ap.add_argument("--cell-sizes", default="512", help="grid lengths of the four-cell study (up to 2048)")
    args = ap.parse_args(argv)
    studies = args.study or ["four_cell", "periodic_sphere", "eight_cube", "boolean_reference", "modulus_rate"]
    s = fftls.Solver(0)
    try:
        if "four_cell" in studies:
            for L in (int(v) for v in args.cell_sizes.split(",")):
                for g in ("MS", "C", "W", "R"):
                    print(json.dumps({"study": "four_cell", **{k: v for k, v in four_cell(s, L, g).items()
                                                                  if k != "corners"}}), flush=True)
        if "four_cell_floor" in studies and args.study:  # run on request only (minutes at L = 2048)
            for L in (int(v) for v in args.cell_sizes.split(",")):
                for g in ("MS", "C", "W", "R"):
                    print(json.dumps({"study": "four_cell_floor", **four_cell_delta_floor(s, L, g)}), flush=True)
        if "periodic_sphere" in studies:
            for L in (64, 128, 256):
                print(json.dumps({"study": "periodic_sphere", **periodic_sphere_modulus(s, L)}), flush=True)
        if "eight_cube" in studies:
            for L in (int(v) for v in args.cube_sizes.split(",")):
                for g in ("MS", "C", "W", "R"):
                    print(json.dumps({"study": "eight_cube", **eight_cube(s, L, g)}), flush=True)
        if "modulus_rate" in studies:  # quasi-porous at 512^3, quasi-rigid at 256^3 (Figs. itPorous, itRigid)
            for L, chi in ((512, 1e-4), (256, 1e4)):
                print(json.dumps({"study": "modulus_rate", **modulus_rate_study(s, L, chi)}), flush=True)
        if "accelerated_rate" in studies and args.study:  # on request only
            print(json.dumps({"study": "accelerated_rate", **accelerated_rate_study(s)}), flush=True)
        if "boolean_reference" in studies:
            for g in ("R", "W", "C"):
                for eta_only in (True, False):
                    print(json.dumps({"study": "boolean_reference",
                                      **boolean_reference_study(s, green=g, eta_only=eta_only)}), flush=True)
    finally:
        s.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
