"""Pins of the oracle's wave vectors and Green operators against closed forms
and invariants stated in the paper (Sec. 3-4).  CPU only."""
import itertools
import math

import numpy as np
import pytest

from oracle import fftls_oracle as O

GREENS = [O.MS, O.CENTERED, O.WILLOT, O.ROTATED]
LAM0, MU0 = 0.7, 0.45


def _modes(shape_xyz):
    return list(itertools.product(*[range(L) for L in shape_xyz]))


def _kvec(k, mode):
    """k at mode (m1, .., md) from the (d, nd, .., n1) array."""
    return k[(slice(None),) + tuple(reversed(mode))]


def _sym(X):
    X = 0.5 * (X + X.transpose(1, 0, 2, 3))
    return 0.5 * (X + X.transpose(0, 1, 3, 2))


def _closed_form(k_vec, lam0, mu0, s_mode="corrected"):
    """eq. (green1) in 2D and eq. (green3) in 3D, typed from the paper.

    s_mode='printed' uses s_jk exactly as printed in the paper,
    'corrected' uses s_jk = -4 Im(r_i r_j*) Im(r_i r_k*) with i the third index.
    """
    r = np.asarray(k_vec, dtype=complex)
    r = r / math.sqrt(float(np.sum(np.abs(r) ** 2)))
    d = r.size
    I = np.eye(d)
    t1 = _sym(np.einsum("i,l,jk->ijkl", r, np.conj(r), I))
    Re = np.real(np.outer(r, np.conj(r)))
    t2 = np.einsum("ij,kl->ijkl", Re, Re)
    t3 = np.einsum("i,j,k,l->ijkl", r, r, np.conj(r), np.conj(r))
    num = (lam0 + 2 * mu0) * t1 - lam0 * t2 - mu0 * t3
    if d == 3:
        s = np.zeros((3, 3))
        for j in range(3):
            i, k = [a for a in range(3) if a != j]
            s[j, j] = 4 * np.imag(r[i] * np.conj(r[k])) ** 2
        for j, k in [(0, 1), (0, 2), (1, 2)]:
            i = 3 - j - k
            if s_mode == "corrected":
                v = -4 * np.imag(r[i] * np.conj(r[j])) * np.imag(r[i] * np.conj(r[k]))
            else:  # as printed: -4 Im(r_k r_j*) Im(r_k r_i*)
                v = -4 * np.imag(r[k] * np.conj(r[j])) * np.imag(r[k] * np.conj(r[i]))
            s[j, k] = s[k, j] = v
        num = num + lam0 * _sym(np.einsum("i,l,jk->ijkl", r, np.conj(r), s))
    den = mu0 * (2 * (lam0 + mu0) - lam0 * abs(np.sum(r * r)) ** 2)
    return num / den


def _continuum_G(q, lam0, mu0):
    """eq. (green0b): the Moulinec-Suquet operator at a real wave vector q."""
    q = np.asarray(q, dtype=float)
    d = q.size
    n2 = float(q @ q)
    I = np.eye(d)
    a = _sym(np.einsum("i,l,jk->ijkl", q, q, I)) / n2
    b = np.einsum("i,j,k,l->ijkl", q, q, q, q) / n2**2
    return (a - (lam0 + mu0) / (lam0 + 2 * mu0) * b) / mu0


def _C0(d):
    return O.stiffness_tensor(LAM0, MU0, d)


@pytest.mark.parametrize("shape", [(8, 8), (5, 6), (4, 4, 4), (3, 5, 4)])
@pytest.mark.parametrize("green", [O.CENTERED, O.WILLOT, O.ROTATED])
def test_displacement_form_equals_closed_form(shape, green):
    """u-form G' = eq. (green1) (2D) / corrected eq. (green3) (3D) at every mode with k != 0."""
    k = O.wave_vector(shape, green)
    n = 0
    for mode in _modes(shape):
        kv = _kvec(k, mode)
        if np.all(kv == 0):
            continue
        G = O.green_tensor(kv, LAM0, MU0)
        Gc = _closed_form(kv, LAM0, MU0)
        assert np.abs(G - Gc).max() < 1e-13
        n += 1
    assert n > 0


def test_printed_green3_is_misprinted_for_W():
    """The s_jk printed in eq. (green3) does not reproduce G^W; the corrected one does."""
    k = O.wave_vector((4, 4, 4), O.WILLOT)
    kv = _kvec(k, (1, 2, 3))
    G = O.green_tensor(kv, LAM0, MU0)
    assert np.abs(G - _closed_form(kv, LAM0, MU0, "corrected")).max() < 1e-13
    assert np.abs(G - _closed_form(kv, LAM0, MU0, "printed")).max() > 1e-3


@pytest.mark.parametrize("shape", [(6, 6), (4, 5, 6)])
@pytest.mark.parametrize("green", GREENS)
def test_idempotence_and_projection(shape, green):
    """G':C0:G' = G'; G' maps onto compatible fields and preserves k*.tau (Sec. 4)."""
    d = len(shape)
    C0 = _C0(d)
    k = O.wave_vector(shape, green)
    rng = np.random.default_rng(3)
    for mode in _modes(shape):
        kv = _kvec(k, mode)
        if np.all(kv == 0):
            continue
        G = O.green_tensor(kv, LAM0, MU0)
        GCG = np.einsum("ijmn,mnpq,pqkl->ijkl", G, C0, G)
        assert np.abs(GCG - G).max() < 1e-13
        u = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        e = 0.5 * (np.outer(kv, u) + np.outer(u, kv))
        assert np.abs(np.einsum("ijmn,mnkl,kl->ij", G, C0, e) - e).max() < 1e-13
        t = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        t = t + t.T
        ctg = np.einsum("ijkl,klmn,mn->ij", C0, G, t)
        assert np.abs(np.conj(kv) @ ctg - np.conj(kv) @ t).max() < 1e-12


@pytest.mark.parametrize("green", GREENS)
def test_symmetries(green):
    """Minor and major (Hermitian) symmetry eq. (greenSym); G'(-q) = G'(q)* eq. (greenSym2)."""
    shape = (5, 7, 3)  # odd: -q is a mode for every q, no Nyquist
    k = O.wave_vector(shape, green)
    for mode in _modes(shape):
        kv = _kvec(k, mode)
        if np.all(kv == 0):
            continue
        G = O.green_tensor(kv, LAM0, MU0)
        assert np.abs(G - G.transpose(1, 0, 2, 3)).max() < 1e-14
        assert np.abs(G - np.conj(G.transpose(2, 3, 0, 1))).max() < 1e-13
        neg = tuple((-m) % L for m, L in zip(mode, shape))
        Gn = O.green_tensor(_kvec(k, neg), LAM0, MU0)
        assert np.abs(Gn - np.conj(G)).max() < 1e-13


def test_rotated_operator_real_and_even():
    """G^R is real and G^R(q) = G^R(-q) (eq. grsym), also at even L."""
    shape = (6, 4, 8)
    k = O.wave_vector(shape, O.ROTATED)
    for mode in _modes(shape):
        kv = _kvec(k, mode)
        if np.all(kv == 0):
            continue
        G = O.green_tensor(kv, LAM0, MU0)
        assert np.abs(G.imag).max() < 1e-14
        neg = tuple((-m) % L for m, L in zip(mode, shape))
        assert np.abs(O.green_tensor(_kvec(k, neg), LAM0, MU0) - G).max() < 1e-13


@pytest.mark.parametrize("shape", [(8, 6), (6, 4, 8)])
def test_rotated_wave_vector_tan_form(shape):
    """Product form of k^R equals eq. (wil14)/(wil14b) wherever tan(q_i/2) is finite."""
    d = len(shape)
    k = O.wave_vector(shape, O.ROTATED)
    for mode in _modes(shape):
        q = [2 * math.pi * O.signed_modes(L)[m] / L for m, L in zip(mode, shape)]
        if any(abs(abs(qi) - math.pi) < 1e-12 for qi in q):
            continue
        prod = np.prod([1 + np.exp(1j * qi) for qi in q])
        ref = np.array([(1j / 2 ** (d - 1)) * math.tan(qi / 2) * prod for qi in q])
        assert np.abs(_kvec(k, mode) - ref).max() < 1e-14


def test_zero_modes():
    """k = 0 exactly at the special modes of eq. (mulfix), (mysymgr) and the 3D R rule."""
    shape = (4, 6, 8)
    kc = O.wave_vector(shape, O.CENTERED)
    kr = O.wave_vector(shape, O.ROTATED)
    kw = O.wave_vector(shape, O.WILLOT)
    for mode in _modes(shape):
        at_pi = [m == L // 2 for m, L in zip(mode, shape)]
        at_0 = [m == 0 for m in mode]
        c_zero = all(p or z for p, z in zip(at_pi, at_0))
        r_zero = sum(at_pi) >= 2 or all(at_0)
        assert np.all(_kvec(kc, mode) == 0) == c_zero
        assert np.all(_kvec(kr, mode) == 0) == r_zero
        assert np.all(_kvec(kw, mode) == 0) == all(at_0)
    k2 = O.wave_vector((6, 6), O.ROTATED)
    assert np.all(_kvec(k2, (3, 3)) == 0)
    assert not np.all(_kvec(k2, (3, 0)) == 0)


@pytest.mark.parametrize("green", GREENS)
def test_small_q_limit(green):
    """G' -> G (eq. green0b) as q -> 0 for any k ~ i q (Sec. 4.1)."""
    L = 4096
    for mode in [(1, 0, 0), (1, 2, 0), (2, 1, 3)]:
        # k typed per discretisation at one low mode of a 4096^3 grid
        q = np.array([2 * math.pi * m / L for m in mode])
        E = np.exp(1j * q)
        if green == O.MS:
            kv = 1j * q
        elif green == O.CENTERED:
            kv = 1j * np.sin(q)
        elif green == O.WILLOT:
            kv = E - 1
        else:
            kv = np.array([(E[i] - 1) * np.prod([1 + E[m] for m in range(3) if m != i]) / 4 for i in range(3)])
        G = O.green_tensor(kv, LAM0, MU0)
        Gc = _continuum_G(q, LAM0, MU0)
        assert np.abs(G - Gc).max() < 50 * float(q @ q) + 1e-12


def test_ms_equals_continuum_formula():
    """With k = i q the u-form reproduces eq. (green0b) (Sec. 4.1, last remark)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        q = rng.standard_normal(3)
        G = O.green_tensor(1j * q, LAM0, MU0)
        assert np.abs(G - _continuum_G(q, LAM0, MU0)).max() < 1e-13
        q2 = rng.standard_normal(2)
        G2 = O.green_tensor(1j * q2, LAM0, MU0)
        assert np.abs(G2 - _continuum_G(q2, LAM0, MU0)).max() < 1e-13


@pytest.mark.parametrize("green", GREENS)
def test_apply_green_matches_tensor(green):
    """apply_green (per-mode solve) agrees with the explicit tensor G':tau, incl. special modes."""
    shape = (4, 6, 4)
    d = 3
    k = O.wave_vector(shape, green)
    rng = np.random.default_rng(7)
    grid = tuple(reversed(shape))
    t = rng.standard_normal((d, d) + grid) + 1j * rng.standard_normal((d, d) + grid)
    t = t + t.transpose(1, 0, 2, 3, 4)
    out = O.apply_green(t, k, LAM0, MU0, green, shape)
    nyq = O.nyquist_mask(shape)
    S0 = O.compliance(LAM0, MU0, d)
    for mode in _modes(shape):
        idx = tuple(reversed(mode))
        kv = _kvec(k, mode)
        tv = t[(slice(None), slice(None)) + idx]
        if green == O.MS and nyq[idx]:
            ref = np.einsum("ijkl,kl->ij", S0, tv)
        elif np.all(kv == 0):
            ref = np.zeros((d, d))
        else:
            ref = np.einsum("ijkl,kl->ij", O.green_tensor(kv, LAM0, MU0), tv)
        assert np.abs(out[(slice(None), slice(None)) + idx] - ref).max() < 1e-12


def test_compliance_inverts_C0():
    for d in (2, 3):
        S = O.compliance(LAM0, MU0, d)
        C = O.stiffness_tensor(LAM0, MU0, d)
        I = np.eye(d)
        Isym = 0.5 * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))
        assert np.abs(np.einsum("ijmn,mnkl->ijkl", C, S) - Isym).max() < 1e-13
