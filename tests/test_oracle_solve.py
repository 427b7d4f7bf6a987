"""Pins of the oracle's full iteration against what the paper and the
mathematics fix: exact discrete fixed points (dense brute force), the
homogeneous medium, laminates, bounds, symmetry, DS = AS, eta by Parseval,
the Nyquist realness rule and the paper's printed numbers.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import fftls_oracle as O
from paper_1412_8398_gb300 import microstructure as MS

GREENS = [O.MS, O.CENTERED, O.WILLOT, O.ROTATED]
SCHEMES = [O.DIRECT, O.ACCELERATED]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def _random_phase(shape_np, seed, p=0.4):
    rng = np.random.default_rng(seed)
    return (rng.random(shape_np) < p).astype(np.uint8)


def _moduli(d, chi=10.0):
    return MS.binary_moduli(chi, d)


def _load(d):
    e = np.zeros((d, d))
    e[0, 0] = 1.0
    e[0, 1] = e[1, 0] = 0.3
    e[d - 1, d - 1] += -0.2
    return e


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape_np", [(8, 8), (5, 5), (4, 4, 4), (3, 3, 3), (8, 6, 4)])
@pytest.mark.parametrize("green", GREENS)
def test_fixed_point_equals_dense_solve(shape_np, green):
    """Converged fields equal the energy minimum of the discrete problem (Sec. 4)."""
    ph = _random_phase(shape_np, seed=sum(shape_np) + green)
    d = ph.ndim
    lam, mu = _moduli(d)
    eb = _load(d)
    if green == O.MS:
        ref = BF.solve_galerkin_ms(ph, lam, mu, eb)
    else:
        ref = BF.solve_stencil(ph, lam, mu, eb, green)
    for scheme in SCHEMES:
        r = O.solve(ph, lam, mu, eb, green, scheme, tol=1e-14, max_iter=5000)
        assert r["converged"]
        assert np.abs(r["strain"] - ref).max() < 1e-11


@pytest.mark.parametrize("green", GREENS)
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape_np", [(6, 4), (4, 5, 6)])
def test_homogeneous_one_iteration(green, scheme, shape_np):
    """A homogeneous medium returns eps = eps_bar after one eta evaluation, for any C0."""
    ph = np.zeros(shape_np, dtype=np.uint8)
    d = ph.ndim
    lam, mu = np.array([1.3]), np.array([0.7])
    eb = _load(d)
    r = O.solve(ph, lam, mu, eb, green, scheme, lam0=0.4, mu0=2.0, tol=1e-14, max_iter=10)
    assert r["iterations"] == 1 and r["converged"]
    assert np.abs(r["strain"] - eb.reshape((d, d) + (1,) * d)).max() == 0.0
    sig = lam[0] * np.trace(eb) * np.eye(d) + 2 * mu[0] * eb
    assert np.abs(r["mean_stress"] - sig).max() < 1e-15


def _laminate_exact(layers, lam, mu, eb, d):
    """Exact laminate fields (phases vary along x1): sigma_1j uniform, eps_jk (j,k>1) = eps_bar."""
    lam_x = lam[layers]
    mu_x = mu[layers]
    M = lam_x + 2 * mu_x
    others = sum(eb[a, a] for a in range(1, d))
    S = (eb[0, 0] + np.mean(lam_x / M) * others) / np.mean(1 / M)
    n1 = layers.size
    eps = np.zeros((d, d, n1))
    for a in range(d):
        for b in range(d):
            eps[a, b] = eb[a, b]
    eps[0, 0] = (S - lam_x * others) / M
    for j in range(1, d):
        s1j = 2 * eb[0, j] / np.mean(1 / mu_x)
        eps[0, j] = eps[j, 0] = s1j / (2 * mu_x)
    return eps


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("green", GREENS)
def test_laminate(dim, green):
    """Laminates normal to e1: W and R are exact for any layer widths; C and MS for even widths."""
    odd_layers = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1, 0], dtype=np.uint8)      # widths 3,2,1,3,1
    even_layers = np.array([0, 0, 1, 1, 1, 1, 0, 0, 1, 1], dtype=np.uint8)     # widths 2,4,2,2
    lam, mu = _moduli(dim, chi=25.0)
    eb = _load(dim)
    if dim == 3:
        eb[1, 2] = eb[2, 1] = 0.15
    for layers, must_match in [(even_layers, True),
                               (odd_layers, green in (O.WILLOT, O.ROTATED))]:
        shape = (layers.size, 4) if dim == 2 else (layers.size, 4, 2)
        ph = MS.laminate(shape, layers)
        r = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=1e-14, max_iter=2000)
        exact = _laminate_exact(layers, lam, mu, eb, dim)
        err = np.abs(r["strain"] - exact.reshape((dim, dim) + (1,) * (dim - 1) + (layers.size,))).max()
        if must_match:
            assert err < 1e-12
        else:
            assert err > 1e-3  # C and MS do not reproduce odd layer widths (checkerboard decoupling)


@pytest.mark.parametrize("green", GREENS)
def test_direct_and_accelerated_share_fixed_point(green):
    """DS and AS give the same fields up to round-off (Sec. 4.2, end)."""
    ph = _random_phase((6, 6, 6), seed=11)
    lam, mu = _moduli(3, chi=0.1)
    eb = _load(3)
    a = O.solve(ph, lam, mu, eb, green, O.DIRECT, tol=1e-14, max_iter=5000)
    b = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=1e-14, max_iter=5000)
    assert np.abs(a["strain"] - b["strain"]).max() < 1e-11


@pytest.mark.parametrize("green", GREENS)
def test_voigt_reuss_bounds(green):
    """Uniform strain is admissible and uniform stress equilibrated: C~ lies between Reuss and Voigt."""
    ph = _random_phase((6, 6, 6), seed=4, p=0.3)
    lam, mu = _moduli(3, chi=50.0)
    C = O.effective_stiffness(ph, lam, mu, green, O.ACCELERATED, tol=1e-12, max_iter=3000)
    f = ph.mean()
    frac = [1 - f, f]
    Cm = [BF._mandel_stiffness(lam[a], mu[a], 3) for a in range(2)]
    voigt = sum(w * c for w, c in zip(frac, Cm))
    reuss = np.linalg.inv(sum(w * np.linalg.inv(c) for w, c in zip(frac, Cm)))
    assert np.linalg.eigvalsh(voigt - 0.5 * (C + C.T)).min() > -1e-9
    assert np.linalg.eigvalsh(0.5 * (C + C.T) - reuss).min() > -1e-9
    assert np.abs(C - C.T).max() < 1e-8 * np.abs(C).max()


@pytest.mark.parametrize("green", [O.CENTERED, O.WILLOT, O.ROTATED])
def test_eta_equals_real_space_divergence(green):
    """eta (eq. criterion, reading A3) equals the RMS of the real-space stencil divergence / ||<sigma>||."""
    ph = _random_phase((5, 6, 4), seed=2)
    lam, mu = _moduli(3)
    eb = _load(3)
    r = O.solve(ph, lam, mu, eb, green, O.DIRECT, tol=0.0, max_iter=2)
    sig = r["stress"]
    k = O.wave_vector(O.grid_shape_xyz(ph), green)
    eta, mean = O.equilibrium_eta(sig, k)
    div = BF.divergence_field(sig, green)
    ref = math.sqrt(np.mean(np.sum(div**2, axis=0))) / math.sqrt(np.sum(mean**2))
    assert abs(eta - ref) < 1e-12 * max(ref, 1e-300)
    assert eta > 1e-6


def test_nyquist_rule_makes_field_real(monkeypatch):
    """Without eq. (hfreq) the inverse transform of G:tau is not real at even L (planted mistake)."""
    ph = _random_phase((6, 6), seed=9)
    lam, mu = _moduli(2)
    eb = _load(2)
    O.solve(ph, lam, mu, eb, O.MS, O.DIRECT, tol=0.0, max_iter=3)   # passes with the rule
    monkeypatch.setattr(O, "nyquist_mask", lambda shape: np.zeros(tuple(reversed(shape)), bool))
    with pytest.raises(AssertionError):
        O.solve(ph, lam, mu, eb, O.MS, O.DIRECT, tol=0.0, max_iter=3)


def test_centered_disc_symmetry():
    """A centred disc keeps its symmetries for G, G^C, G^R and not for G^W (Sec. 4.1, 5.1)."""
    n = 16
    ph = MS.centered_disc(n, 0.25)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (100.0, 0.3)])
    eb = np.array([[0.0, 1.0], [1.0, 0.0]])
    for green in GREENS:
        r = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=1e-12, max_iter=3000)
        s12 = r["stress"][0, 1]
        asym = max(np.abs(s12 - s12[::-1, ::-1]).max(), np.abs(s12 - s12.T).max())
        if green == O.WILLOT:
            assert asym > 1e-3
        else:
            assert asym < 1e-10


def test_eight_cube_symmetry():
    """The centred cube (the 3D four-cell of Sec. 5.2) under eps_bar_12: sigma_12 is invariant
    under the mirrors x_i -> -x_i and the swap x1 <-> x2 for G, G^C, G^R and not for G^W."""
    n = 8
    ph = MS.square_inclusion(n, 3)
    lam, mu = MS.young_poisson_phases([(1.0, 0.25), (1000.0, 0.25)])
    eb = np.zeros((3, 3))
    eb[0, 1] = eb[1, 0] = 0.5
    for green in GREENS:
        r = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=1e-12, max_iter=5000)
        assert r["converged"]
        s12 = r["stress"][0, 1]
        maps = [s12[:, :, ::-1], s12[:, ::-1, :], s12[::-1, :, :], np.swapaxes(s12, 1, 2)]
        asym = max(np.abs(s12 - t).max() for t in maps) / np.abs(s12).max()
        if green == O.WILLOT:
            assert asym > 1e-3
        else:
            assert asym < 1e-10


def test_porous_periodic_sphere_ordering():
    """Sec. 5.3: every operator under-estimates C~_1111 at finite L; G^R is closest, G farthest."""
    g = _golden("periodic_sphere.txt")
    n = 16
    ph = MS.periodic_sphere(n, g["fraction"])
    lam, mu = MS.binary_moduli(g["chi"], 3)
    eb = np.diag([1.0, 0.0, 0.0])
    vals = {}
    for green in GREENS:
        if green == O.MS:
            kw = {}
        else:
            l0, m0 = MS.lame_from_young(0.2, 0.25)
            kw = {"lam0": l0, "mu0": m0}
        r = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=1e-8, max_iter=2000, **kw)
        assert r["converged"]
        vals[green] = r["mean_stress"][0, 0]
    lim = g["c1111_limit"] + g["c1111_limit_pm"]
    assert all(v < lim for v in vals.values())
    err = {k: g["c1111_limit"] - v for k, v in vals.items()}
    assert err[O.ROTATED] < min(err[O.CENTERED], err[O.WILLOT]) <= max(err[O.CENTERED], err[O.WILLOT]) < err[O.MS]


def test_reference_medium_defaults():
    lam, mu = MS.binary_moduli(9.0, 3)
    l0, m0 = O.reference_medium(lam, mu, 3, O.ACCELERATED)
    assert abs(m0 - 0.6 * 3.0) < 1e-15 and abs(l0 + 2 * m0 / 3 - 3.0) < 1e-14   # sqrt(1 * 9) = 3
    l0, m0 = O.reference_medium(lam, mu, 3, O.DIRECT)
    assert abs(m0 - 0.5 * 0.6 * 10) < 1e-14 and abs(l0 + 2 * m0 / 3 - 5.0) < 1e-14


def test_maxdelta_stop_returns_next_iterate():
    ph = _random_phase((6, 6), seed=5)
    lam, mu = _moduli(2)
    eb = _load(2)
    r = O.solve(ph, lam, mu, eb, O.ROTATED, O.ACCELERATED, tol=1e-10, max_iter=3000, stop=O.STOP_MAXDELTA)
    assert r["converged"]
    assert len(r["eta_history"]) == r["iterations"]
    full = O.solve(ph, lam, mu, eb, O.ROTATED, O.ACCELERATED, tol=0.0, max_iter=r["iterations"])
    assert np.abs(full["strain"] - r["strain"]).max() == 0.0
