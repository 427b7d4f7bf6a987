"""GPU: the tile-schedule autotuner changes no result.

Every schedule the tuner may pick computes the same per-line and per-mode
arithmetic; only the grouping of the FP64 partial sums of eta and <sigma>
changes.  So a tuned and an untuned solve agree to rounding, and both agree
with the oracle.
"""
import numpy as np
import pytest

from oracle import fftls_oracle as O
from paper_1412_8398_gb300 import microstructure as MS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_8398_gb300 import build as B, fftls
    B.build()
    return fftls


@pytest.mark.parametrize("green,scheme,shape", [("R", "AS", (24, 20, 18)), ("W", "DS", (16, 12, 10)),
                                                ("C", "AS", (12, 10, 9)), ("MS", "AS", (16, 16, 8)),
                                                ("R", "DS", (32, 24))])
def test_tuned_schedule_matches_default(build, green, scheme, shape):
    fftls = build
    ph, _ = MS.boolean_spheres(tuple(shape), 2.5, 0.3, seed=9)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (50.0, 0.25)])
    d = ph.ndim
    eb = np.eye(d)
    eb[0, 1] = eb[1, 0] = 0.3
    s_def, s_tun = fftls.Solver(0), fftls.Solver(0)
    try:
        r0 = s_def.solve(ph, lam, mu, eb, green, scheme, tol=0.0, max_iter=4, autotune=False)
        r1 = s_tun.solve(ph, lam, mu, eb, green, scheme, tol=0.0, max_iter=4, autotune=True)
        plans0, plans1 = s_def.tile_plans(), s_tun.tile_plans()
    finally:
        s_def.close()
        s_tun.close()
    assert [p["tuned"] for p in plans0] == [0] and [p["tuned"] for p in plans1] == [1]
    p = plans1[0]
    assert p["x1_lines"] in (1, 2, 4, 8) and p["x5_lines"] in (1, 2, 4, 8) and p["x1_vb"] in (0, 1, 2, 4)
    assert p["x5_vb"] in (0, 1)
    assert p["y_w"] in (1, 2, 4, 8, 16) and p["z_w"] in (1, 2, 4, 8, 16)
    assert np.abs(r1.strain - r0.strain).max() < 1e-12
    np.testing.assert_allclose(r1.eta_history, r0.eta_history, rtol=1e-12)
    g = {"MS": O.MS, "C": O.CENTERED, "W": O.WILLOT, "R": O.ROTATED}[green]
    ref = O.solve(ph, lam, mu, eb, g, O.ACCELERATED if scheme == "AS" else O.DIRECT, tol=0.0, max_iter=4)
    comps = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)] if d == 3 else [(0, 0), (1, 1), (0, 1)]
    want = np.stack([ref["strain"][i, j] for i, j in comps])
    assert np.abs(r1.strain - want).max() < 1e-9


def test_plan_cached_per_grid_and_precision(build):
    fftls = build
    ph, _ = MS.boolean_spheres((16, 16, 16), 2.0, 0.3, seed=3)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (10.0, 0.3)])
    s = fftls.Solver(0)
    try:
        k0, _ = s.counters()
        s.solve(ph, lam, mu, np.diag([1.0, 0, 0]), "R", "AS", tol=1e-6, precision="fp32_refine64")
        k1, _ = s.counters()
        s.solve(ph, lam, mu, np.diag([0, 1.0, 0]), "R", "AS", tol=1e-6, precision="fp32_refine64")
        k2, _ = s.counters()
        plans = s.tile_plans()
    finally:
        s.close()
    assert sorted(p["precision"] for p in plans) == [0, 1] and all(p["tuned"] for p in plans)
    # the second solve of the same grid does not tune again: far fewer launches than the first
    assert (k2 - k1) < (k1 - k0)


@pytest.mark.parametrize("green,shape", [("R", (64, 24, 20)), ("MS", (32, 16, 12)), ("R", (48, 40))])
def test_imported_schedules_same_bits(build, green, shape):
    """Schedules imported with set_tile_plans are used as they are: every variant of the x1
    passes (eps loaded by the threads, 1, 2 or 4 voxels at a time, or each batch staged in shared
    memory by bulk copies) at one batch size gives the same FP32 fields bit for bit (the same voxels per thread, in the
    same order); eta, normalised by FP32 partial sums of <sigma>, agrees to their rounding."""
    fftls = build
    ph, _ = MS.boolean_spheres(tuple(shape), 2.5, 0.3, seed=12)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (30.0, 0.25)])
    d = ph.ndim
    eb = np.eye(d)
    eb[0, 1] = eb[1, 0] = 0.2
    n = tuple(reversed(ph.shape)) + (1,) * (3 - d)  # (n1, n2, n3) of the solve
    gcode = {"MS": 0, "C": 1, "W": 2, "R": 3}[green]
    runs = {}
    for lines, vb, vb5 in [(1, 4, 1), (1, 0, 0), (2, 1, 1), (2, 0, 1), (4, 4, 1), (4, 0, 0), (4, 4, 0)]:
        plan = {"precision": 0, "n1": n[0], "n2": n[1], "n3": n[2], "green": gcode, "x1_lines": lines,
                "x1_vb": vb, "x5_lines": 2, "y_w": 2, "z_w": 2, "e_planes": 4 if (d == 3 and green != "MS") else 0,
                "x5_vb": vb5}
        s = fftls.Solver(0)
        try:
            s.set_tile_plans([plan])
            r = s.solve(ph, lam, mu, eb, green, "AS", tol=0.0, max_iter=5, precision="fp32")
            held = [p for p in s.tile_plans() if p["precision"] == 0]
        finally:
            s.close()
        assert len(held) == 1 and held[0]["tuned"] == 1
        assert (held[0]["x1_lines"], held[0]["x1_vb"], held[0]["x5_vb"]) == (lines, vb, vb5)
        runs[(lines, vb, vb5)] = r
    for a, b in [((1, 4, 1), (1, 0, 0)), ((2, 1, 1), (2, 0, 1)), ((4, 4, 1), (4, 0, 0)), ((4, 4, 1), (4, 4, 0))]:
        assert np.array_equal(runs[a].strain, runs[b].strain)
    # eta's normalisation <sigma> comes from FP32 partial sums, which the compiler may contract
    # differently per variant and other batch sizes group differently: equal to FP32 rounding
    ref = runs[(1, 4, 1)]
    for r in runs.values():
        assert np.abs(r.strain - ref.strain).max() <= 1e-6 * np.abs(ref.strain).max()
        np.testing.assert_allclose(r.eta_history, ref.eta_history, rtol=1e-6)


def test_set_tile_plans_rejects_invalid_rows(build):
    fftls = build
    s = fftls.Solver(0)
    try:
        good = {"precision": 0, "n1": 32, "n2": 32, "n3": 32, "green": 3, "x1_lines": 2, "x1_vb": 4,
                "x5_lines": 2, "y_w": 4, "z_w": 4, "e_planes": 8}
        for bad in [{"x1_lines": 9}, {"x1_vb": 3}, {"precision": 1, "x1_vb": 0}, {"n1": 40, "x1_vb": 0}, {"y_w": 3},
                    {"e_planes": 33}, {"y_threads": 64}, {"x5_vb": 2}, {"precision": 1, "x1_vb": 1, "x5_vb": 0}]:
            with pytest.raises(fftls.FftlsError):
                s.set_tile_plans([dict(good, **bad)])
        assert s.tile_plans() == []
        s.set_tile_plans([good])
        assert [p["x1_lines"] for p in s.tile_plans()] == [2]
    finally:
        s.close()
