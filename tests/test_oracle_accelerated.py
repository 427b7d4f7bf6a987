"""Pins of the accelerated scheme's step (Sec. 3, eq. as) beyond its fixed point.

The other oracle pins check where the iteration ends (dense solves, laminates,
the homogeneous medium), which every relaxation of the form
eps + omega M:(e - eps) shares.  These check the step itself:

* a closed form of one step on a homogeneous medium C = c C0 started from
  eps_bar + a + b, with a a constant tensor and b a compatible fluctuation built
  from the paper's finite-difference stencils (eq. mul1, wil071, disc3deps) or,
  for operator G, by differentiating a trigonometric polynomial: the direct
  scheme returns eps_bar - (c - 1) b, the accelerated one
  eps_bar + (c - 1)/(c + 1) (a - b);
* the Eyre-Milton contraction rate: with C0 from eq. refAcc and equal Poisson
  ratios, the error of the accelerated scheme contracts asymptotically by
  (sqrt(chi) - 1) / (sqrt(chi) + 1) per iteration (G' is a C0-orthogonal
  projector, so 2 G'C0 - I is a reflection and each phase contributes the
  Cayley factor (c - c0)/(c + c0); the extreme phases attain it).

Each test also plants a wrong relaxation factor in the oracle and checks that
the pin catches it.  CPU only.
"""
import math

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import fftls_oracle as O
from paper_1412_8398_gb300 import microstructure as MS

GREENS = [O.MS, O.CENTERED, O.WILLOT, O.ROTATED]


def _tensor_grid(v, d, grid):
    return np.broadcast_to(np.asarray(v, dtype=np.float64).reshape((d, d) + (1,) * d), (d, d) + grid).copy()


def _compatible_stencil(shape_np, green, seed):
    """b = sym(grad_h u) for a random nodal displacement u, with the discrete gradient of
    operator `green` written out as its real-space stencil (bruteforce.strain_operator)."""
    d = len(shape_np)
    shape_xyz = tuple(reversed(shape_np))
    N = int(np.prod(shape_np))
    u = np.random.default_rng(seed).standard_normal(d * N)
    B = BF.strain_operator(shape_xyz, green)
    return BF._mandel_to_tensor_field(B @ u, d, tuple(shape_np))


def _compatible_trig(shape_np, seed, modes=3):
    """b = sym(grad u) of a trigonometric polynomial u without Nyquist frequencies,
    differentiated by hand: u_j = A_j cos(q.x + phi_j) gives d_i u_j = -A_j q_i sin(q.x + phi_j)."""
    d = len(shape_np)
    shape_xyz = tuple(reversed(shape_np))
    rng = np.random.default_rng(seed)
    coords = np.meshgrid(*[np.arange(n) for n in shape_np], indexing="ij")   # numpy axes
    x = [coords[d - 1 - i] for i in range(d)]                                 # x_1 .. x_d
    grad = np.zeros((d, d) + tuple(shape_np))                                # grad[i, j] = d_i u_j
    for _ in range(modes):
        m = [int(rng.integers(-((L - 1) // 2), (L - 1) // 2 + 1)) for L in shape_xyz]
        q = [2.0 * math.pi * m[i] / shape_xyz[i] for i in range(d)]
        phase = sum(q[i] * x[i] for i in range(d))
        for j in range(d):
            A, phi = rng.standard_normal(), rng.uniform(0, 2 * math.pi)
            for i in range(d):
                grad[i, j] += -A * q[i] * np.sin(phase + phi)
    return 0.5 * (grad + grad.transpose(1, 0, *range(2, 2 + d)))


def _one_step(shape_np, green, scheme, c, omega=2.0):
    d = len(shape_np)
    lam0, mu0 = 0.4, 0.7
    lam, mu = np.array([c * lam0]), np.array([c * mu0])
    ph = np.zeros(shape_np, dtype=np.uint8)
    eb = np.zeros((d, d))
    eb[0, 0], eb[0, 1], eb[1, 0] = 1.0, 0.25, 0.25
    a = np.zeros((d, d))
    a[0, 0], a[1, 1], a[0, 1], a[1, 0] = 0.1, -0.2, 0.05, 0.05
    if green == O.MS:
        b = _compatible_trig(shape_np, seed=7 + d)
    else:
        b = _compatible_stencil(shape_np, green, seed=7 + d)
    grid = tuple(shape_np)
    eps0 = _tensor_grid(eb, d, grid) + _tensor_grid(a, d, grid) + b
    r = O.solve(ph, lam, mu, eb, green, scheme, lam0=lam0, mu0=mu0, tol=0.0, max_iter=1, eps_init=eps0,
                omega=omega)
    return r["strain"], _tensor_grid(eb, d, grid), _tensor_grid(a, d, grid), b


@pytest.mark.parametrize("green", GREENS)
@pytest.mark.parametrize("shape_np", [(6, 8), (4, 6, 8)])
def test_one_step_closed_form(green, shape_np):
    """One step on C = c C0 from eps_bar + a + b: DS gives eps_bar - (c-1) b (eq. ds),
    AS gives eps_bar + (c-1)/(c+1) (a - b) (eq. as)."""
    c = 3.0
    got, eb, a, b = _one_step(shape_np, green, O.DIRECT, c)
    assert np.abs(b).max() > 0.1
    assert np.abs(got - (eb - (c - 1.0) * b)).max() < 1e-12
    got, eb, a, b = _one_step(shape_np, green, O.ACCELERATED, c)
    assert np.abs(got - (eb + (c - 1.0) / (c + 1.0) * (a - b))).max() < 1e-12


@pytest.mark.parametrize("green", [O.MS, O.ROTATED])
def test_one_step_catches_wrong_relaxation(green):
    """The closed form fails with the relaxation factor 1 (or 1.9) in place of 2."""
    c = 3.0
    for omega in (1.0, 1.9):
        got, eb, a, b = _one_step((4, 6, 8), green, O.ACCELERATED, c, omega=omega)
        assert np.abs(got - (eb + (c - 1.0) / (c + 1.0) * (a - b))).max() > 1e-3


def _rate(ph, lam, mu, eb, green, omega, k0=40, k1=90):
    """Asymptotic contraction of ||eps^k - eps*||_2 between iterations k0 and k1 (the iteration
    is memoryless, so the run from k0 continues from the returned field)."""
    ref = BF.solve_galerkin_ms(ph, lam, mu, eb) if green == O.MS else BF.solve_stencil(ph, lam, mu, eb, green)
    r0 = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=0.0, max_iter=k0, omega=omega)
    r1 = O.solve(ph, lam, mu, eb, green, O.ACCELERATED, tol=0.0, max_iter=k1 - k0, eps_init=r0["strain"],
                 omega=omega)
    e0 = np.linalg.norm(r0["strain"] - ref)
    e1 = np.linalg.norm(r1["strain"] - ref)
    assert e1 > 1e-12 * np.linalg.norm(ref)     # still above round-off: the ratio measures the rate
    return (e1 / e0) ** (1.0 / (k1 - k0))


@pytest.mark.parametrize("green", GREENS)
def test_eyre_milton_contraction_rate(green):
    """Two-phase 6^3 medium, chi = 100, nu = 0.25 in both phases, C0 from eq. refAcc (the default):
    the accelerated scheme contracts at (sqrt(chi) - 1)/(sqrt(chi) + 1) = 9/11 per iteration; with the
    relaxation factor 1 it contracts at about 1/(1 + 1/sqrt(chi)) = 10/11 instead."""
    chi = 100.0
    ph = (np.random.default_rng(3).random((6, 6, 6)) < 0.4).astype(np.uint8)
    lam, mu = MS.binary_moduli(chi, 3)
    eb = np.diag([1.0, 0.0, 0.0])
    eb[0, 1] = eb[1, 0] = 0.3
    bound = (math.sqrt(chi) - 1.0) / (math.sqrt(chi) + 1.0)
    rate = _rate(ph, lam, mu, eb, green, 2.0)
    assert bound - 0.01 < rate < bound + 2e-3
    if green == O.ROTATED:
        planted = _rate(ph, lam, mu, eb, green, 1.0)
        assert planted > bound + 0.05
