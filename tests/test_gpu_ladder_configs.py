"""GPU: the FP32 -> FP64 precision ladder, the configuration shapes and
full-size properties, against the FP64 oracle or against what holds exactly.

* Ladder: the returned field's eta is recomputed by the oracle (FP64, from the
  field alone) and must be <= tol; moduli agree with the FP64 solve to 1e-6.
* 2D 128^2 centred disc: parity with the oracle (fields 1e-9 max-abs, <sigma>
  1e-10 relative).
* 3D 128^3 Boolean spheres at three contrasts: every operator under both
  schemes for two FP64 iterations against the oracle (fields 1e-9 max-abs, eta
  1e-9 relative), and every operator under the ladder (oracle eta of the
  returned field <= tol, <sigma> within 1e-6 of FP64); operator G's two-field
  x1 tile at 64^3.
* 512^3, the benchmark's launch configuration: a homogeneous medium converges
  in one iteration to eps_bar exactly; a laminate reproduces the exact
  piecewise-constant solution (G^R and G^W are exact for any layer widths).
"""
import numpy as np
import pytest

from oracle import fftls_oracle as O
import _oracle_jobs as _jobs
from paper_1412_8398_gb300 import microstructure as MS

pytestmark = pytest.mark.gpu
FIELD_TOL = 1e-9


@pytest.fixture(scope="module")
def solver():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_8398_gb300 import build, fftls
    build.build()
    s = fftls.Solver(0)
    yield s
    s.close()


def comps(t):
    d = t.shape[0]
    if d == 3:
        return np.stack([t[0, 0], t[1, 1], t[2, 2], t[1, 2], t[0, 2], t[0, 1]])
    return np.stack([t[0, 0], t[1, 1], t[0, 1]])


def tensor(f):
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


def oracle_eta(ph, lam, mu, strain, green):
    """eta of eq. criterion recomputed by the oracle from a strain field."""
    d = ph.ndim
    eps = tensor(np.asarray(strain))
    Cs = [O.stiffness_tensor(lam[a], mu[a], d) for a in range(len(lam))]
    sig = O._contract(Cs, ph, eps)
    k = O.wave_vector(O.grid_shape_xyz(ph), green)
    return O.equilibrium_eta(sig, k)[0]


GREENS = ["MS", "C", "W", "R"]


@pytest.mark.parametrize("green", range(4))
@pytest.mark.parametrize("scheme", ["AS", "DS"])
def test_ladder_reaches_tolerance_and_matches_fp64(solver, green, scheme):
    ph, _ = MS.boolean_spheres((32, 32, 32), 3.0, 0.3, seed=21)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)] if scheme == "AS" else [(1.0, 0.3), (20.0, 0.3)])
    eb = np.diag([1.0, 0.0, 0.0])
    tol = 1e-6
    mix = solver.solve(ph, lam, mu, eb, GREENS[green], scheme, tol=tol, max_iter=5000, precision="fp32_refine64")
    f64 = solver.solve(ph, lam, mu, eb, GREENS[green], scheme, tol=tol, max_iter=5000, precision="fp64")
    assert mix.converged and f64.converged
    assert mix.iterations_fp32 >= mix.iterations - 4      # the bulk of the work runs in FP32
    assert oracle_eta(ph, lam, mu, mix.strain, green) <= tol * 1.0001
    rel = np.abs(mix.mean_stress - f64.mean_stress).max() / np.abs(f64.mean_stress).max()
    assert rel < 1e-6
    assert abs(mix.mean_strain[0] - 1.0) < tol


def test_fp32_only_floor(solver):
    """Plain FP32 stalls above a tight tolerance (its rounding floor); the ladder does not."""
    ph, _ = MS.boolean_spheres((32, 32, 32), 3.0, 0.3, seed=22)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)])
    r32 = solver.solve(ph, lam, mu, np.diag([1.0, 0, 0]), "R", "AS", tol=1e-9, max_iter=1500, precision="fp32")
    rmix = solver.solve(ph, lam, mu, np.diag([1.0, 0, 0]), "R", "AS", tol=1e-9, max_iter=1500,
                        precision="fp32_refine64")
    assert not r32.converged
    assert rmix.converged


def test_config_2d_disc(solver):
    """128^2 centred disc, f = 0.25, E 1 / 100, nu 0.3, eps_bar_12 = 1, G^R direct scheme (FP64)."""
    ph = MS.centered_disc(128, 0.25)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (100.0, 0.3)])
    eb = np.array([[0.0, 1.0], [1.0, 0.0]])
    ref = O.solve(ph, lam, mu, eb, O.ROTATED, O.DIRECT, tol=1e-8, max_iter=5000)
    got = solver.solve(ph, lam, mu, eb, "R", "DS", tol=1e-8, max_iter=5000)
    assert ref["converged"] and got.converged and got.iterations == ref["iterations"]
    assert np.abs(got.strain - comps(ref["strain"])).max() < FIELD_TOL
    ms = np.array([ref["mean_stress"][0, 0], ref["mean_stress"][1, 1], ref["mean_stress"][0, 1]])
    assert np.abs(got.mean_stress - ms).max() < 1e-10 * np.abs(ms).max()
    # the symmetric discretisations keep the disc's symmetry, G^W does not (Sec. 4.1)
    for green, sym in [("MS", True), ("C", True), ("W", False)]:
        r = solver.solve(ph, lam, mu, eb, green, "AS", tol=1e-8, max_iter=5000)
        s12 = r.stress[2]
        asym = max(np.abs(s12 - s12[::-1, ::-1]).max(), np.abs(s12 - s12.T).max())
        assert (asym < 1e-6) if sym else (asym > 1e-3)


C2_CHIS = [0.01, 10.0, 1000.0]
C2_CASES = [(128, 6.0, 0.3, 1, chi, g, sch, 2) for chi in C2_CHIS for g in range(4) for sch in (O.DIRECT, O.ACCELERATED)]
# operator G with the accelerated scheme at a second compile-time length: its x1 pass carries tau and sigma
C2_CASES.append((64, 3.0, 0.3, 2, 1000.0, O.MS, O.ACCELERATED, 2))


@pytest.fixture(scope="module")
def c2_oracle():
    """The oracle on every case of the 128^3 matrix, in spawned worker processes (the parent has a CUDA
    context; spawn starts clean interpreters)."""
    import multiprocessing as mp
    import os
    workers = max(1, min(8, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        out = {case: (comp, eta) for case, comp, eta in pool.imap_unordered(_jobs.boolean_case, C2_CASES)}
    return out


@pytest.mark.parametrize("contrast", C2_CHIS)
def test_config_128_boolean_parity(solver, c2_oracle, contrast):
    """128^3 Boolean spheres (radius 6, f = 0.3, seed 1), contrast chi: two FP64 iterations of every
    operator under both schemes agree with the oracle element by element (fields 1e-9 max-abs,
    eta histories 1e-9 relative)."""
    ph, _ = MS.boolean_spheres((128, 128, 128), 6.0, 0.3, seed=1)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (contrast, 0.3)])
    eb = np.diag([1.0, 0.0, 0.0])
    for case in C2_CASES:
        n, _, _, _, chi, green, scheme, iters = case
        if n != 128 or chi != contrast:
            continue
        comp, eta = c2_oracle[case]
        got = solver.solve(ph, lam, mu, eb, GREENS[green], ["DS", "AS"][scheme], tol=0.0, max_iter=iters)
        assert np.abs(got.strain - comp).max() < FIELD_TOL, (GREENS[green], scheme)
        np.testing.assert_allclose(got.eta_history, eta, rtol=1e-9)


def test_config_64_ms_accelerated_parity(solver, c2_oracle):
    """Operator G under the accelerated scheme at 64^3: the x1 pass transforms tau and sigma together
    (eta in Fourier space) on the compile-time tile of length 64."""
    case = C2_CASES[-1]
    n, radius, fraction, seed, chi, green, scheme, iters = case
    ph, _ = MS.boolean_spheres((n, n, n), radius, fraction, seed=seed)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (chi, 0.3)])
    comp, eta = c2_oracle[case]
    got = solver.solve(ph, lam, mu, np.diag([1.0, 0.0, 0.0]), "MS", "AS", tol=0.0, max_iter=iters)
    assert np.abs(got.strain - comp).max() < FIELD_TOL
    np.testing.assert_allclose(got.eta_history, eta, rtol=1e-9)


@pytest.mark.parametrize("contrast", C2_CHIS)
def test_config_128_boolean_ladder(solver, contrast):
    """128^3 Boolean spheres, every operator with the accelerated scheme under the FP32 -> FP64 ladder
    to eta <= 1e-6: the oracle recomputes eta from the returned FP64 field (<= tol) and <sigma> agrees
    with the plain FP64 solve to 1e-6 relative."""
    ph, _ = MS.boolean_spheres((128, 128, 128), 6.0, 0.3, seed=1)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (contrast, 0.3)])
    eb = np.diag([1.0, 0.0, 0.0])
    tol = 1e-6
    for green in range(4):
        mix = solver.solve(ph, lam, mu, eb, GREENS[green], "AS", tol=tol, max_iter=5000, precision="fp32_refine64",
                           want_stress=False)
        f64 = solver.solve(ph, lam, mu, eb, GREENS[green], "AS", tol=tol, max_iter=5000, precision="fp64",
                           want_strain=False, want_stress=False, history=False)
        assert mix.converged and f64.converged
        assert oracle_eta(ph, lam, mu, mix.strain, green) <= tol * 1.0001
        rel = np.abs(mix.mean_stress - f64.mean_stress).max() / np.abs(f64.mean_stress).max()
        assert rel < 1e-6, (GREENS[green], rel)


def _laminate_exact(layers, lam, mu, eb):
    lam_x, mu_x = lam[layers], mu[layers]
    M = lam_x + 2 * mu_x
    others = eb[1, 1] + eb[2, 2]
    S = (eb[0, 0] + np.mean(lam_x / M) * others) / np.mean(1 / M)
    out = np.zeros((6, layers.size))
    out[0] = (S - lam_x * others) / M
    out[1], out[2], out[3] = eb[1, 1], eb[2, 2], eb[1, 2]
    out[4] = (2 * eb[0, 2] / np.mean(1 / mu_x)) / (2 * mu_x)
    out[5] = (2 * eb[0, 1] / np.mean(1 / mu_x)) / (2 * mu_x)
    return out


def test_full_size_512_properties(solver):
    """512^3 (the benchmark's size and launch configuration): exact special cases."""
    torch = pytest.importorskip("torch")
    n = 512
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)])
    eb = np.array([[1.0, 0.2, 0.1], [0.2, -0.3, 0.05], [0.1, 0.05, 0.4]])
    # homogeneous medium: eps = eps_bar exactly after one eta evaluation per precision
    # (the ladder certifies the FP32 result with one FP64 evaluation)
    hom = torch.zeros((n, n, n), dtype=torch.uint8, device="cuda")
    r = solver.solve(hom, lam[:1], mu[:1], eb, "R", "AS", tol=1e-6, precision="fp32_refine64",
                     want_stress=False)
    assert r.converged and r.iterations_fp32 == 1 and r.iterations == 2
    ebv = np.array([eb[0, 0], eb[1, 1], eb[2, 2], eb[1, 2], eb[0, 2], eb[0, 1]])
    assert float((r.strain - torch.tensor(ebv, device="cuda").view(6, 1, 1, 1)).abs().max()) < 1e-7
    del r
    # laminate with uneven layer widths along x1: exact solution for G^R
    rng = np.random.default_rng(5)
    layers = (rng.random(n) < 0.4).astype(np.uint8)
    img = np.broadcast_to(layers, (n, n, n)).copy()
    dph = torch.from_numpy(img).cuda()
    r = solver.solve(dph, lam, mu, eb, "R", "AS", tol=1e-9, max_iter=3000, precision="fp32_refine64",
                     want_stress=False)
    assert r.converged
    exact = _laminate_exact(layers, lam, mu, eb)
    got = r.strain[:, 0, 0, :].cpu().numpy()                     # any (x2, x3): fields depend on x1 only
    assert np.abs(got - exact).max() < 1e-7 * np.abs(exact).max()
    spread = float((r.strain - r.strain[:, :1, :1, :]).abs().max())
    assert spread < 1e-7 * np.abs(exact).max()


@pytest.mark.parametrize("shape_np", [(1, 1, 1), (1, 1), (1, 2, 1024), (3, 1, 1), (2, 2048), (2048, 2),
                                      (1, 2, 2048), (2048, 1, 2)])
def test_degenerate_and_maximum_lengths(solver, shape_np):
    """Single voxel, single-pixel 2D grid, the longest supported axes (2048: in 3D FP64 refused along
    x2 / x3, whose tiles of six complex doubles per mode do not fit shared memory, and for G along
    x1, whose tau and sigma lines share one tile), unit axes."""
    from paper_1412_8398_gb300 import fftls
    rng = np.random.default_rng(0)
    ph = (rng.random(shape_np) < 0.5).astype(np.uint8)
    d = ph.ndim
    lam, mu = MS.binary_moduli(7.0, d)
    eb = np.eye(d) * 0.5
    eb[0, d - 1] = eb[d - 1, 0] = 0.25
    for g in range(4):
        if d == 3 and (max(ph.shape[:2]) > 2000 or (g == O.MS and ph.shape[-1] > 1600)):
            with pytest.raises(fftls.FftlsError) as e:
                solver.solve(ph, lam, mu, eb, GREENS[g], "AS", tol=0.0, max_iter=3)
            assert e.value.status == fftls.E_UNSUPPORTED_SIZE
            continue
        ref = O.solve(ph, lam, mu, eb, g, O.ACCELERATED, tol=0.0, max_iter=3)
        got = solver.solve(ph, lam, mu, eb, GREENS[g], "AS", tol=0.0, max_iter=3)
        assert np.abs(got.strain - comps(ref["strain"])).max() < FIELD_TOL
