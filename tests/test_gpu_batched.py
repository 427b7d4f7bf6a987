"""GPU: fftls_solve_batched (independent problems of uneven sizes, concurrent workers).

* With the built-in tile schedules a batched sample gives bit for bit what
  fftls_solve gives (same kernels, same schedule, fixed reduction order),
  whatever the mix of grids, operators and schemes in the batch.
* Batched ladder solves reach eta <= tol (re-checked by the oracle from the
  returned field) with moduli within 1e-6 of the FP64 solve.
* Argument errors are reported, not run.
"""
import numpy as np
import pytest

from oracle import fftls_oracle as O
from paper_1412_8398_gb300 import microstructure as MS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fftls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_8398_gb300 import build, fftls as F
    build.build()
    return F


def _tensor(f):
    if f.shape[0] == 6:
        t = np.zeros((3, 3) + f.shape[1:])
        t[0, 0], t[1, 1], t[2, 2] = f[0], f[1], f[2]
        t[1, 2] = t[2, 1] = f[3]
        t[0, 2] = t[2, 0] = f[4]
        t[0, 1] = t[1, 0] = f[5]
    else:
        t = np.zeros((2, 2) + f.shape[1:])
        t[0, 0], t[1, 1] = f[0], f[1]
        t[0, 1] = t[1, 0] = f[2]
    return t


def _mixed_batch():
    shapes = [(16, 16, 16), (12, 10, 9), (8, 8, 8), (20, 16), (9, 5, 15), (24, 20, 18), (5, 5, 5), (32, 24)]
    greens = ["R", "W", "C", "MS", "R", "C", "W", "R"]
    schemes = ["AS", "DS", "AS", "AS", "DS", "AS", "AS", "DS"]
    out = []
    for i, shp in enumerate(shapes):
        ph, _ = MS.boolean_spheres(shp, 2.0, 0.3, seed=40 + i)
        lam, mu = MS.young_poisson_phases([(1.0, 0.3), (5.0 + 10 * i, 0.25)])
        d = len(shp)
        eb = np.eye(d) * (0.5 + 0.1 * i)
        eb[0, d - 1] = eb[d - 1, 0] = 0.2
        out.append({"phase": ph, "lam": lam, "mu": mu, "eps_bar": eb, "green": greens[i], "scheme": schemes[i]})
    return out


def test_batched_equals_individual_solves(fftls):
    batch = _mixed_batch()
    s = fftls.Solver(0)
    try:
        res, st = s.solve_batched(batch, tol=1e-9, max_iter=400, precision="fp64", concurrency=3,
                                  want_strain=True, history=True, autotune=False)
        single = [s.solve(b["phase"], b["lam"], b["mu"], b["eps_bar"], b["green"], b["scheme"], tol=1e-9,
                          max_iter=400, precision="fp64", autotune=False) for b in batch]
    finally:
        s.close()
    assert st in (fftls.OK, fftls.E_NOT_CONVERGED)
    assert sum(r.status == fftls.OK for r in res) >= 5
    for r, q in zip(res, single):
        assert r.status == q.status
        assert r.iterations == q.iterations
        assert np.array_equal(r.strain, q.strain)
        assert np.array_equal(r.eta_history, q.eta_history)
        assert np.array_equal(r.mean_stress, q.mean_stress)


def test_batched_matches_oracle_fixed_iterations(fftls):
    batch = _mixed_batch()[:5]
    s = fftls.Solver(0)
    try:
        res, _ = s.solve_batched(batch, tol=0.0, max_iter=3, precision="fp64", concurrency=2, want_strain=True)
    finally:
        s.close()
    gmap = {"MS": O.MS, "C": O.CENTERED, "W": O.WILLOT, "R": O.ROTATED}
    for b, r in zip(batch, res):
        ref = O.solve(b["phase"], b["lam"], b["mu"], b["eps_bar"], gmap[b["green"]],
                      O.ACCELERATED if b["scheme"] == "AS" else O.DIRECT, tol=0.0, max_iter=3)
        assert np.abs(_tensor(r.strain) - ref["strain"]).max() < 1e-9


def test_batched_ladder_reaches_tolerance(fftls):
    specs = MS.batch_recipe(6, lengths=(16, 24, 32))
    batch = []
    for spec in specs:
        ph, lam, mu, _ = MS.batch_sample(spec)
        batch.append({"phase": ph, "lam": lam, "mu": mu, "eps_bar": np.diag([1.0, 0.0, 0.0])})
    s = fftls.Solver(0)
    try:
        res, st = s.solve_batched(batch, tol=1e-6, max_iter=3000, precision="fp32_refine64", concurrency=4,
                                  want_strain=True)
        r64 = [s.solve(b["phase"], b["lam"], b["mu"], b["eps_bar"], "R", "AS", tol=1e-6, max_iter=3000,
                       precision="fp64", want_strain=False, want_stress=False) for b in batch]
        plans = s.tile_plans()
    finally:
        s.close()
    assert st == fftls.OK
    assert {(p["n1"], p["precision"]) for p in plans} >= {(L, 0) for L in {sp["L"] for sp in specs}}
    for b, r, q in zip(batch, res, r64):
        assert r.converged and q.converged
        k = O.wave_vector(O.grid_shape_xyz(b["phase"]), O.ROTATED)
        Cs = [O.stiffness_tensor(b["lam"][a], b["mu"][a], 3) for a in range(2)]
        sig = O._contract(Cs, b["phase"], _tensor(np.asarray(r.strain)))
        assert O.equilibrium_eta(sig, k)[0] <= 1e-6 * 1.0001
        assert np.abs(r.mean_stress - q.mean_stress).max() < 1e-6 * np.abs(q.mean_stress).max()


def test_batched_argument_errors(fftls):
    s = fftls.Solver(0)
    try:
        res, st = s.solve_batched([], concurrency=2)
        assert res == [] and st == fftls.OK
        b = _mixed_batch()[:1]
        with pytest.raises(fftls.FftlsError):
            s.solve_batched(b, concurrency=65)
        bad = dict(b[0], lam=np.array([1.0, -5.0]))
        with pytest.raises(fftls.FftlsError) as e:
            s.solve_batched([b[0], bad], concurrency=2)
        assert "sample 1" in str(e.value)
    finally:
        s.close()


def _grouped_batch():
    """Samples sharing grids, operators and schemes (grouped launches), with different phases,
    moduli, reference media and loads, interleaved with a 2D and an odd-sized sample."""
    out = []
    specs = [((16, 16, 16), "R", "AS")] * 5 + [((12, 10, 9), "W", "DS")] * 3 + [((20, 16), "C", "AS"),
                                                                             ((9, 5, 15), "MS", "AS")]
    for i, (shp, g, sch) in enumerate(specs):
        ph, _ = MS.boolean_spheres(shp, 2.0, 0.2 + 0.03 * i, seed=70 + i)
        lam, mu = MS.young_poisson_phases([(1.0, 0.3), (3.0 + 7 * i, 0.2 + 0.01 * i)])
        d = len(shp)
        eb = np.eye(d) * (0.3 + 0.1 * i)
        eb[0, d - 1] = eb[d - 1, 0] = 0.1 * (i % 3)
        item = {"phase": ph, "lam": lam, "mu": mu, "eps_bar": eb, "green": g, "scheme": sch}
        if i == 2:
            item["lam0"], item["mu0"] = 2.0, 1.5   # an explicit reference medium inside a group
        out.append(item)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine64", "fp32"])
def test_grouped_launch_equals_individual_solves(fftls, precision):
    """Samples of one 3D grid, operator and scheme run as one grouped launch per kernel; each gives
    what fftls_solve gives alone, including samples that stop at max_iter while others of the group
    go on: the same statuses and iteration counts and bit for bit the same fields (same schedule,
    same per-sample partial sums).  The eta and <sigma> histories agree to one unit in the last place:
    the reduction kernel's grouped instantiation is compiled on its own and may contract its FP64
    multiply-adds differently."""
    batch = _grouped_batch()
    s = fftls.Solver(0)
    kw = dict(tol=1e-7 if precision == "fp32" else 1e-9, max_iter=160, precision=precision)
    try:
        res, st = s.solve_batched(batch, concurrency=3, want_strain=True, want_stress=True, history=True,
                                  autotune=False, **kw)
        single = [s.solve(b["phase"], b["lam"], b["mu"], b["eps_bar"], b["green"], b["scheme"],
                          lam0=b.get("lam0"), mu0=b.get("mu0"), autotune=False, raise_on_error=False, **kw)
                  for b in batch]
    finally:
        s.close()
    statuses = {r.status for r in res}
    assert fftls.OK in statuses
    for r, q in zip(res, single):
        assert r.status == q.status
        assert r.iterations == q.iterations and r.iterations_fp32 == q.iterations_fp32
        assert np.array_equal(r.strain, q.strain)
        assert np.array_equal(r.stress, q.stress)
        np.testing.assert_allclose(r.eta_history, q.eta_history, rtol=1e-15, atol=0)
        np.testing.assert_allclose(r.mean_stress_history, q.mean_stress_history, rtol=1e-15, atol=1e-300)
        np.testing.assert_allclose(r.mean_stress, q.mean_stress, rtol=1e-15, atol=1e-300)
