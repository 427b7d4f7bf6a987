"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (FP64 mode): fields within 1e-9 max-abs, effective moduli / mean
stresses within 1e-10 relative.  Inputs are seeded synthetic
microstructures; sizes span several column tiles and ragged tails.
"""
import math

import numpy as np
import pytest

from oracle import fftls_oracle as O
from paper_1412_8398_gb300 import microstructure as MS

pytestmark = pytest.mark.gpu

GREEN_NAMES = ["MS", "C", "W", "R"]
SCHEME_NAMES = ["DS", "AS"]
FIELD_TOL = 1e-9
MODULI_TOL = 1e-10


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


def to_components(t):
    """(d, d, grid) tensor field -> (n_c, grid) in the library's component order."""
    d = t.shape[0]
    if d == 3:
        return np.stack([t[0, 0], t[1, 1], t[2, 2], t[1, 2], t[0, 2], t[0, 1]])
    return np.stack([t[0, 0], t[1, 1], t[0, 1]])


def vec_components(m):
    d = m.shape[0]
    if d == 3:
        return np.array([m[0, 0], m[1, 1], m[2, 2], m[1, 2], m[0, 2], m[0, 1]])
    return np.array([m[0, 0], m[1, 1], m[0, 1]])


def load(d):
    e = np.zeros((d, d))
    e[0, 0] = 1.0
    e[0, 1] = e[1, 0] = 0.3
    e[d - 1, d - 1] -= 0.2
    if d == 3:
        e[1, 2] = e[2, 1] = -0.15
        e[0, 2] = e[2, 0] = 0.05
    return e


def random_phase(shape_np, seed, p=0.35, n_phases=2):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_phases, size=shape_np).astype(np.uint8) if n_phases > 2 else \
        (rng.random(shape_np) < p).astype(np.uint8)


SHAPES = [(16, 12), (5, 5), (12, 10, 8), (3, 3, 3), (9, 5, 15), (6, 20, 18)]


@pytest.mark.parametrize("shape_np", SHAPES)
@pytest.mark.parametrize("green", range(4))
@pytest.mark.parametrize("scheme", range(2))
def test_fixed_iterations_match_oracle(solver, shape_np, green, scheme):
    """eps^k after k = 1 and 3 updates, the eta and <sigma> histories (FP64)."""
    ph = random_phase(shape_np, seed=len(shape_np) * 100 + green * 10 + scheme)
    d = ph.ndim
    lam, mu = MS.binary_moduli(20.0, d)
    eb = load(d)
    for k in (1, 3):
        ref = O.solve(ph, lam, mu, eb, green, scheme, tol=0.0, max_iter=k)
        got = solver.solve(ph, lam, mu, eb, GREEN_NAMES[green], SCHEME_NAMES[scheme], tol=0.0, max_iter=k)
        assert got.iterations == k
        err = np.abs(got.strain - to_components(ref["strain"])).max()
        assert err < FIELD_TOL, f"k={k} strain max-abs {err:.3e}"
        err_s = np.abs(got.stress - to_components(ref["stress"])).max()
        assert err_s < FIELD_TOL * max(1.0, np.abs(lam).max() * 10)
        np.testing.assert_allclose(got.eta_history, ref["eta_history"], rtol=1e-9, atol=1e-14)
        for i in range(k):
            np.testing.assert_allclose(got.mean_stress_history[i], vec_components(ref["mean_stress_history"][i]),
                                       rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("shape_np", [(48, 96, 20), (96, 48, 16)])
@pytest.mark.parametrize("green", range(4))
@pytest.mark.parametrize("scheme", range(2))
def test_radix3_strided_lengths_match_oracle(solver, shape_np, green, scheme):
    """x2 / x3 lengths 48 and 96, whose strided transforms run compile-time stages with a radix-3
    stage (48 = 4 4 3, 96 = 4 8 3): eps^2, the eta and <sigma> histories against the oracle (FP64)."""
    ph = random_phase(shape_np, seed=7 + green * 10 + scheme)
    lam, mu = MS.binary_moduli(20.0, 3)
    eb = load(3)
    ref = O.solve(ph, lam, mu, eb, green, scheme, tol=0.0, max_iter=2)
    got = solver.solve(ph, lam, mu, eb, GREEN_NAMES[green], SCHEME_NAMES[scheme], tol=0.0, max_iter=2)
    assert got.iterations == 2
    assert np.abs(got.strain - to_components(ref["strain"])).max() < FIELD_TOL
    np.testing.assert_allclose(got.eta_history, ref["eta_history"], rtol=1e-9, atol=1e-14)
    for i in range(2):
        np.testing.assert_allclose(got.mean_stress_history[i], vec_components(ref["mean_stress_history"][i]),
                                   rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("green", range(4))
@pytest.mark.parametrize("scheme", range(2))
def test_converged_moduli_match_oracle(solver, green, scheme):
    """Boolean spheres 24^3 (radius 3, f = 0.3, contrast 10): converged fields and <sigma>."""
    ph, _ = MS.boolean_spheres((24, 24, 24), 3.0, 0.3, seed=7)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (10.0, 0.3)])
    eb = np.diag([1.0, 0.0, 0.0])
    ref = O.solve(ph, lam, mu, eb, green, scheme, tol=1e-11, max_iter=3000)
    got = solver.solve(ph, lam, mu, eb, GREEN_NAMES[green], SCHEME_NAMES[scheme], tol=1e-11, max_iter=3000)
    assert ref["converged"] and got.converged
    assert got.iterations == ref["iterations"]
    assert np.abs(got.strain - to_components(ref["strain"])).max() < FIELD_TOL
    ms_ref = vec_components(ref["mean_stress"])
    assert np.abs(got.mean_stress - ms_ref).max() < MODULI_TOL * np.abs(ms_ref).max()


def test_effective_stiffness_matches_oracle(solver):
    ph, _ = MS.boolean_spheres((12, 12, 12), 2.0, 0.25, seed=3)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (30.0, 0.2)])
    Cref = O.effective_stiffness(ph, lam, mu, O.ROTATED, O.ACCELERATED, tol=1e-11, max_iter=3000)
    C, its, st = solver.effective_stiffness(ph, lam, mu, "R", "AS", tol=1e-11, max_iter=3000)
    assert st == 0
    assert np.abs(C - Cref).max() < MODULI_TOL * np.abs(Cref).max()
    assert np.abs(C - C.T).max() < 1e-9 * np.abs(C).max()


@pytest.mark.parametrize("green", range(4))
def test_homogeneous_one_iteration(solver, green):
    ph = np.zeros((8, 6, 10), dtype=np.uint8)
    lam, mu = np.array([1.3]), np.array([0.7])
    eb = load(3)
    for scheme in SCHEME_NAMES:
        got = solver.solve(ph, lam, mu, eb, GREEN_NAMES[green], scheme, lam0=0.4, mu0=2.0, tol=1e-12)
        assert got.converged and got.iterations == 1
        assert np.abs(got.strain - vec_components(eb)[:, None, None, None]).max() == 0.0


@pytest.mark.parametrize("green", range(4))
def test_maxdelta_stop_matches_oracle(solver, green):
    ph = random_phase((10, 12), seed=5)
    lam, mu = MS.binary_moduli(50.0, 2)
    eb = load(2)
    ref = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=1e-9, max_iter=3000, stop=O.STOP_MAXDELTA)
    got = solver.solve(ph, lam, mu, eb, GREEN_NAMES[green], "AS", tol=1e-9, max_iter=3000, stop="maxdelta")
    assert ref["converged"] and got.converged
    assert got.iterations == ref["iterations"]
    assert np.abs(got.strain - to_components(ref["strain"])).max() < FIELD_TOL


@pytest.mark.parametrize("scheme", range(2))
def test_warm_start_matches_oracle(solver, scheme):
    ph = random_phase((8, 10, 6), seed=9)
    lam, mu = MS.binary_moduli(5.0, 3)
    eb = load(3)
    rng = np.random.default_rng(1)
    init = eb[:, :, None, None, None] + 0.1 * rng.standard_normal((3, 3) + ph.shape)
    init = 0.5 * (init + init.transpose(1, 0, 2, 3, 4))
    for k in (1, 4):
        ref = O.solve(ph, lam, mu, eb, O.ROTATED, scheme, tol=0.0, max_iter=k, eps_init=init)
        got = solver.solve(ph, lam, mu, eb, "R", SCHEME_NAMES[scheme], tol=0.0, max_iter=k,
                           eps_init=to_components(init))
        assert np.abs(got.strain - to_components(ref["strain"])).max() < FIELD_TOL


def test_multiphase_and_degenerate_axes(solver):
    """Five phases; grids with unit-length axes (n1 = 1, n3 = 1 in 3D)."""
    lam = np.array([0.5, 1.0, 2.0, 4.0, 8.0])
    mu = np.array([0.4, 0.9, 1.5, 3.0, 6.0])
    for shape_np in [(4, 6, 1), (1, 6, 10), (15, 1, 4)]:
        ph = random_phase(shape_np, seed=2, n_phases=5)
        ref = O.solve(ph, lam, mu, load(3), O.WILLOT, O.ACCELERATED, tol=0.0, max_iter=3)
        got = solver.solve(ph, lam, mu, load(3), "W", "AS", tol=0.0, max_iter=3)
        assert np.abs(got.strain - to_components(ref["strain"])).max() < FIELD_TOL


def test_device_pointers(solver):
    torch = pytest.importorskip("torch")
    ph = random_phase((10, 12, 16), seed=4)
    lam, mu = MS.binary_moduli(10.0, 3)
    host = solver.solve(ph, lam, mu, load(3), "R", "AS", tol=0.0, max_iter=4)
    dph = torch.from_numpy(ph).cuda()
    dev = solver.solve(dph, lam, mu, load(3), "R", "AS", tol=0.0, max_iter=4)
    assert dev.strain.is_cuda
    assert np.abs(dev.strain.cpu().numpy() - host.strain).max() == 0.0


def test_invalid_arguments(solver):
    from paper_1412_8398_gb300 import fftls
    ph = np.zeros((8, 8), dtype=np.uint8)
    with pytest.raises(fftls.FftlsError) as e:
        solver.solve(np.zeros((7, 8), dtype=np.uint8), [1.0], [1.0], load(2), "R", "AS")
    assert e.value.status == fftls.E_UNSUPPORTED_SIZE
    with pytest.raises(fftls.FftlsError) as e:
        solver.solve(ph, [1.0], [-1.0], load(2), "R", "AS")
    assert e.value.status == fftls.E_INVALID_ARG
    with pytest.raises(fftls.FftlsError) as e:
        solver.solve(ph + 3, [1.0, 2.0], [1.0, 2.0], load(2), "R", "AS")
    assert e.value.status == fftls.E_INVALID_ARG
    with pytest.raises(fftls.FftlsError) as e:   # porous phase, default C0 degenerates
        solver.solve(ph, [1.0, 0.0], [1.0, 0.0], load(2), "R", "AS")
    assert e.value.status == fftls.E_INVALID_ARG


def test_not_converged_and_diverged(solver):
    from paper_1412_8398_gb300 import fftls
    ph = random_phase((8, 8, 8), seed=1)
    lam, mu = MS.binary_moduli(100.0, 3)
    r = solver.solve(ph, lam, mu, load(3), "R", "AS", tol=1e-14, max_iter=3)
    assert r.status == fftls.E_NOT_CONVERGED and r.iterations == 3
    # direct scheme with a reference medium far too soft: the iteration diverges
    r = solver.solve(ph, lam, mu, load(3), "R", "DS", lam0=0.05, mu0=0.05, tol=1e-10, max_iter=500,
                     raise_on_error=False)
    assert r.status == fftls.E_DIVERGED
    ref = O.solve(ph, lam, mu, load(3), O.ROTATED, O.DIRECT, lam0=0.05, mu0=0.05, tol=1e-10, max_iter=500)
    assert not ref["converged"] and r.iterations == ref["iterations"]


def test_eta_only_criterion_vs_mean_guard(solver):
    """The accelerated scheme's iterates need not have mean eps_bar (reading 12): the default stop
    also requires |<eps> - eps_bar| <= tol |eps_bar|; eta_only (the paper's criterion) stops on eta
    alone, never later."""
    layers = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1, 0], dtype=np.uint8)     # odd layer widths
    ph = MS.laminate((layers.size, 4), layers)
    lam, mu = MS.binary_moduli(25.0, 2)
    eb = np.array([[0.7, 0.2], [0.2, -0.3]])
    tol = 1e-12
    for green in ("W", "R"):
        g = solver.solve(ph, lam, mu, eb, green, "AS", tol=tol, max_iter=2000)
        e = solver.solve(ph, lam, mu, eb, green, "AS", tol=tol, max_iter=2000, eta_only=True)
        assert g.converged and e.converged
        assert e.iterations <= g.iterations
        ebv = np.array([0.7, -0.3, 0.2])
        w = np.array([1.0, 1.0, 2.0])
        err = np.sqrt(np.sum(w * (g.mean_strain - ebv) ** 2) / np.sum(w * ebv ** 2))
        assert err <= tol * 1.0001
