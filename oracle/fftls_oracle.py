"""CPU FP64 oracle of the FFT Lippmann-Schwinger iteration (Willot 2015).

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this module: only
the tests, the package entry point's smoke check and the benchmark's CPU
baseline leg call it.  It shares no code with the CUDA path.

It is written to be checked against the paper by eye: plain numpy, float64,
full (not half) complex spectra from ``numpy.fft``, full d x d tensors and
one explicit small linear solve per Fourier mode.

Paper passages followed (section / equation of the paper):
  * Sec. 2, eq. (a1): isotropic C = lambda dd + mu (dd + dd), kappa = lambda + (2/d) mu.
  * Sec. 3, eq. (ls), (ds): tau = sigma - C0:eps, eps^{k+1} = eps_bar - G * tau^k, eps^0 = eps_bar.
  * Sec. 3, eq. (ft), (ft2): forward DFT unnormalised, inverse with 1/N.
  * Sec. 3, eq. (contmodes): q_i = 2 pi m_i / L_i.
  * Sec. 3, eq. (hfreq): even L, some q_i = pi  =>  G = C0^{-1} (operator G only).
  * Sec. 3, eq. (as): accelerated scheme, (refAcc) and (ref) reference media.
  * Sec. 4, eq. (discFour), (discFour2): G' from the discrete gradient k and divergence k*.
  * Sec. 4, eq. (mul2), (wil072), (wil14), (wil14b): k^C, k^W, k^R.
  * Sec. 4, eq. (mulfix), (mysymgr) and the 3D rule: G' = 0 where k(q) = 0, q != 0.
  * Sec. 6.1, eq. (criterion): equilibrium norm eta.

Readings where the paper is silent or garbled (each repeated where used):
  * G' is applied in its displacement form: solve (k*.C0.k) u = k*.tau per
    mode and return -sym(k (x) u).  Writing out eq. (discFour) with the
    divergence k* gives A_jl = lambda0 k_j* k_l + mu0 k_j k_l* + mu0 |k|^2 d_jl.
  * k^R is evaluated in its tan-free product form
    (e^{iq_i} - 1) prod_{m != i} (1 + e^{iq_m}) / 2^{d-1}, which equals
    eq. (wil14)/(wil14b) wherever tan(q_i/2) is finite and is its
    continuous limit at q_i = pi.
  * eta uses the divergence k* (the one each scheme enforces), includes
    Parseval's 1/N, measures derivatives in voxel units and normalises by the
    Frobenius norm of <sigma> with off-diagonal entries counted twice.
  * `iterations` counts evaluations of eta (stresses sigma^k computed).
"""
from __future__ import annotations

import math

import numpy as np

MS, CENTERED, WILLOT, ROTATED = 0, 1, 2, 3
DIRECT, ACCELERATED = 0, 1
STOP_ETA, STOP_MAXDELTA = 0, 1

GREEN_NAMES = {MS: "MS", CENTERED: "C", WILLOT: "W", ROTATED: "R"}


# ---------------------------------------------------------------------------
# grid and modes
# ---------------------------------------------------------------------------
def grid_shape_xyz(phase: np.ndarray):
    """(n1, .., nd) from a phase image stored in numpy order (nd, .., n1)."""
    return tuple(reversed(phase.shape))


def signed_modes(L: int) -> np.ndarray:
    """m_i in DFT order, mapped to -(L-1)/2 .. L/2 (eq. contmodes); L/2 -> +L/2."""
    m = np.arange(L)
    return np.where(m <= L // 2, m, m - L)


def _exp_iq(L: int) -> np.ndarray:
    """e^{i q} for q = 2 pi m / L with exactly representable special values.

    cos is set to exactly 0 at q = +-pi/2, sin to exactly 0 at q = 0, pi,
    so that products like 1 + e^{i pi} vanish exactly (they define the
    zero modes of eq. mulfix / mysymgr).
    """
    s = signed_modes(L)
    q = 2.0 * np.pi * s / L
    c = np.cos(q)
    sn = np.sin(q)
    sn[(2 * s) % L == 0] = 0.0
    c[(4 * s) % (4 * L) == L] = 0.0  # q = pi/2
    c[(4 * s) % (4 * L) == 3 * L] = 0.0  # q = -pi/2
    c[(2 * s) == L] = -1.0
    c[s == 0] = 1.0
    return c + 1j * sn


def _axis_array(v1d: np.ndarray, i: int, d: int) -> np.ndarray:
    """Reshape a 1D per-axis array of coordinate x_{i+1} to broadcast on the grid."""
    shape = [1] * d
    shape[d - 1 - i] = v1d.size
    return v1d.reshape(shape)


def wave_vector(shape_xyz, green: int) -> np.ndarray:
    """Discrete wave vector k(q), complex array of shape (d, nd, .., n1).

    MS: k = i q (continuum, Sec. 3, used in eq. criterion for G).
    C:  k_i = i sin q_i                      (eq. mul2)
    W:  k_i = e^{i q_i} - 1                  (eq. wil072)
    R:  k_i = (e^{iq_i}-1) prod_{m!=i} (1+e^{iq_m}) / 2^{d-1}
        (= eq. wil14 in 2D, eq. wil14b in 3D; product form, see header).
    """
    d = len(shape_xyz)
    grid = tuple(reversed(shape_xyz))
    k = np.zeros((d,) + grid, dtype=np.complex128)
    E = [_axis_array(_exp_iq(L), i, d) for i, L in enumerate(shape_xyz)]
    for i, L in enumerate(shape_xyz):
        s = signed_modes(L)
        q = _axis_array(2.0 * np.pi * s / L, i, d)
        if green == MS:
            k[i] = 1j * q
        elif green == CENTERED:
            k[i] = 1j * E[i].imag
        elif green == WILLOT:
            k[i] = E[i] - 1.0
        elif green == ROTATED:
            v = E[i] - 1.0
            for m in range(d):
                if m != i:
                    v = v * (1.0 + E[m])
            k[i] = v / 2.0 ** (d - 1)
        else:
            raise ValueError("unknown Green operator")
    return k


def nyquist_mask(shape_xyz) -> np.ndarray:
    """True at modes where some q_i = pi with L_i even (eq. hfreq)."""
    d = len(shape_xyz)
    grid = tuple(reversed(shape_xyz))
    mask = np.zeros(grid, dtype=bool)
    for i, L in enumerate(shape_xyz):
        if L % 2 == 0:
            s = signed_modes(L)
            mask = mask | _axis_array(s == L // 2, i, d)
    return mask


# ---------------------------------------------------------------------------
# materials
# ---------------------------------------------------------------------------
def stiffness_tensor(lam: float, mu: float, d: int) -> np.ndarray:
    """C_ijkl = lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (Sec. 2)."""
    I = np.eye(d)
    return (lam * np.einsum("ij,kl->ijkl", I, I)
            + mu * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I)))


def bulk_modulus(lam, mu, d):
    """kappa = lambda + (2/d) mu (Sec. 2)."""
    return lam + (2.0 / d) * mu


def reference_medium(lam, mu, d, scheme, beta=0.5):
    """Default reference (lambda0, mu0).

    Accelerated scheme, eq. (refAcc): kappa0 = sqrt(k_min k_max), mu0 = sqrt(mu_min mu_max).
    Direct scheme, eq. (ref):       kappa0 = beta (k_min + k_max), mu0 = beta (mu_min + mu_max).
    The paper states both for binary media; with several phases the extreme
    phases are used.  lambda0 = kappa0 - (2/d) mu0.
    """
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    kap = bulk_modulus(lam, mu, d)
    if scheme == ACCELERATED:
        k0 = math.sqrt(kap.min() * kap.max())
        m0 = math.sqrt(mu.min() * mu.max())
    else:
        k0 = beta * (kap.min() + kap.max())
        m0 = beta * (mu.min() + mu.max())
    return k0 - (2.0 / d) * m0, m0


def _contract(Cfield_by_phase, phase, eps):
    """sigma_ij(x) = C_ijkl(x) eps_kl(x) with C looked up by phase."""
    out = np.zeros_like(eps)
    for a, Ca in enumerate(Cfield_by_phase):
        m = phase == a
        if not m.any():
            continue
        out[:, :, m] = np.einsum("ijkl,kln->ijn", Ca, eps[:, :, m])
    return out


# ---------------------------------------------------------------------------
# Green operator
# ---------------------------------------------------------------------------
def compliance(lam0, mu0, d):
    """(C0)^{-1} on symmetric tensors, as a d^4 tensor."""
    return compliance_general(stiffness_tensor(lam0, mu0, d), d)


def apply_green(tau_hat: np.ndarray, k: np.ndarray, lam0: float, mu0: float,
                green: int, shape_xyz) -> np.ndarray:
    """Return G'(q):tau_hat(q) at every mode (q = 0 gives 0).

    Displacement form of eq. (discFour2): with b_j = k_i* tau_ij and
    A_jl = lambda0 k_j* k_l + mu0 k_j k_l* + mu0 |k|^2 d_jl, solve A u = b
    and return sym(k (x) u).  (The strain correction is -G':tau.)
    Special modes:
      * k(q) = 0 (q = 0, and for C / R the modes of eq. mulfix, mysymgr and
        the 3D rule of Sec. 4.2): G' = 0.
      * operator G (MS) at even-L modes with some q_i = pi: G = C0^{-1} (eq. hfreq).
    Modes are processed in slabs of the outermost axis to bound memory.
    """
    d = k.shape[0]
    out = np.zeros_like(tau_hat)
    nyq = nyquist_mask(shape_xyz) if green == MS else None
    S0 = compliance(lam0, mu0, d) if green == MS else None
    for z in range(k.shape[1]):
        kz = k[:, z]                      # (d, ...)
        tz = tau_hat[:, :, z]             # (d, d, ...)
        flat = kz.reshape(d, -1)          # (d, M)
        tflat = tz.reshape(d, d, -1)      # (d, d, M)
        M = flat.shape[1]
        b = np.einsum("im,ijm->jm", np.conj(flat), tflat)         # b_j = k_i* tau_ij
        A = (lam0 * np.einsum("jm,lm->mjl", np.conj(flat), flat)
             + mu0 * np.einsum("jm,lm->mjl", flat, np.conj(flat)))
        knorm2 = np.sum(np.abs(flat) ** 2, axis=0)
        A = A + mu0 * knorm2[:, None, None] * np.eye(d)[None, :, :]
        zero = np.all(flat == 0, axis=0)
        A[zero] = np.eye(d)
        u = np.linalg.solve(A, b.T[:, :, None])[:, :, 0].T        # (d, M)
        g = 0.5 * (np.einsum("im,jm->ijm", flat, u) + np.einsum("jm,im->ijm", flat, u))
        g[:, :, zero] = 0.0
        if green == MS:
            nz = nyq[z].reshape(-1)
            if nz.any():
                g[:, :, nz] = np.einsum("ijkl,klm->ijm", S0, tflat[:, :, nz])
        out[:, :, z] = g.reshape(tz.shape)
    return out


def green_tensor(k_vec: np.ndarray, lam0: float, mu0: float) -> np.ndarray:
    """Full G'_ijkl at one mode with wave vector k_vec != 0 (displacement form).

    G'_ijkl = sym_(ij),(kl) k_i (A^{-1})_jk k_l*, A as in apply_green.
    """
    k_vec = np.asarray(k_vec, dtype=np.complex128)
    d = k_vec.size
    A = (lam0 * np.outer(np.conj(k_vec), k_vec) + mu0 * np.outer(k_vec, np.conj(k_vec))
         + mu0 * np.vdot(k_vec, k_vec).real * np.eye(d))
    Ainv = np.linalg.inv(A)
    G = np.einsum("i,jk,l->ijkl", k_vec, Ainv, np.conj(k_vec))
    G = 0.5 * (G + G.transpose(1, 0, 2, 3))
    G = 0.5 * (G + G.transpose(0, 1, 3, 2))
    return G


# ---------------------------------------------------------------------------
# equilibrium norm
# ---------------------------------------------------------------------------
def equilibrium_eta(sig: np.ndarray, k: np.ndarray):
    """eta of eq. (criterion) and <sigma>.

    eta = sqrt(sum_q |k*(q) . sigma_hat(q)|^2) / (N ||<sigma>||_F),
    (k* . s)_j = sum_i k_i* s_ij; <sigma> = mean over voxels.
    0/0 is taken as 0 and x/0 (x > 0) as +inf.
    """
    d = sig.shape[0]
    axes = tuple(range(2, 2 + d))
    N = sig[0, 0].size
    sh = np.fft.fftn(sig, axes=axes)
    div = np.einsum("i...,ij...->j...", np.conj(k), sh)
    num = math.sqrt(float(np.sum(np.abs(div) ** 2)))
    mean = sig.reshape(d, d, -1).mean(axis=2)
    den = N * math.sqrt(float(np.sum(mean ** 2)))
    if num == 0.0:
        eta = 0.0
    elif den == 0.0:
        eta = math.inf
    else:
        eta = num / den
    return eta, mean


# ---------------------------------------------------------------------------
# the iteration
# ---------------------------------------------------------------------------
def _tensor_from_vector(v, d):
    """Tensor components from (11,22,33,23,13,12) (3D) or (11,22,12) (2D)."""
    t = np.zeros((d, d))
    if d == 3:
        t[0, 0], t[1, 1], t[2, 2] = v[0], v[1], v[2]
        t[1, 2] = t[2, 1] = v[3]
        t[0, 2] = t[2, 0] = v[4]
        t[0, 1] = t[1, 0] = v[5]
    else:
        t[0, 0], t[1, 1] = v[0], v[1]
        t[0, 1] = t[1, 0] = v[2]
    return t


def mean_strain_error(eps, eps_bar):
    """|<eps> - eps_bar|_F / |eps_bar|_F (absolute when eps_bar = 0).

    Reading of the stop rule for the accelerated scheme: its iterates need
    not have mean eps_bar (eq. as), and an iterate can be exactly
    equilibrated with the wrong mean (a laminate does this every other
    iteration), so eta <= tol is accepted only together with this error
    <= tol.  Direct-scheme iterates have mean eps_bar exactly.
    """
    d = eps.shape[0]
    mean = eps.reshape(d, d, -1).mean(axis=2)
    den = math.sqrt(float(np.sum(eps_bar ** 2)))
    num = math.sqrt(float(np.sum((mean - eps_bar) ** 2)))
    return num / den if den > 0 else num


def solve(phase, lam, mu, eps_bar, green, scheme, lam0=None, mu0=None,
          tol=1e-8, max_iter=1000, stop=STOP_ETA, eps_init=None, beta=0.5,
          check_real=True, omega=2.0):
    """Run the direct (eq. ds) or accelerated (eq. as) scheme with operator `green`.

    phase: uint8 image, numpy order (n3, n2, n1) or (n2, n1).
    lam, mu: per-phase Lame coefficients.  eps_bar: (d, d) tensor or the
    component vector (11,22,33,23,13,12) / (11,22,12).
    Returns a dict with the strain and stress fields (d, d, grid), <sigma>,
    the eta and <sigma> histories, `iterations` and `converged`.

    Iteration k (k = 0, 1, ...):
      sigma^k = C:eps^k; eta_k; stop if eta_k <= tol and the mean strain
      error (see mean_strain_error) <= tol (stop=STOP_ETA);
      tau^k = sigma^k - C0:eps^k; e_hat = -G':tau_hat (q != 0), e_hat(0) = N eps_bar;
      e = IDFT(e_hat) (imaginary part checked to be round-off);
      DS: eps^{k+1} = e;  AS: eps^{k+1} = eps^k + 2 (C + C0)^{-1} C0 : (e - eps^k).
    With stop=STOP_MAXDELTA the test is max over voxels and components of
    |eps^{k+1} - eps^k| and |sigma^{k+1} - sigma^k| below tol (Sec. 5.1, 5.3);
    the field returned is then eps^{k+1} and `iterations` = k + 1.
    The iteration is declared diverged (and stops, no update) when eta_k is
    not finite or exceeds 1e4 eta_0.
    omega is the factor 2 of eq. (as); the tests pass other values only to
    plant a wrong relaxation and check that the pins of the accelerated step
    catch it.
    """
    phase = np.asarray(phase)
    d = phase.ndim
    shape_xyz = grid_shape_xyz(phase)
    N = phase.size
    lam = np.asarray(lam, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    eb = np.asarray(eps_bar, dtype=np.float64)
    if eb.ndim == 1:
        eb = _tensor_from_vector(eb, d)
    if lam0 is None or mu0 is None:
        lam0, mu0 = reference_medium(lam, mu, d, scheme, beta)
    Cs = [stiffness_tensor(lam[a], mu[a], d) for a in range(lam.size)]
    C0 = stiffness_tensor(lam0, mu0, d)
    # (C + C0)^{-1} C0 per phase, as a d^2 x d^2 solve restricted to symmetric tensors
    Ms = []
    for Ca in Cs:
        S = compliance_general(Ca + C0, d)
        Ms.append(np.einsum("ijmn,mnkl->ijkl", S, C0))
    k = wave_vector(shape_xyz, green)
    axes = tuple(range(2, 2 + d))

    if eps_init is None:
        eps = np.broadcast_to(eb[:, :, None], (d, d, N)).reshape((d, d) + phase.shape).copy()
    else:
        eps = np.array(eps_init, dtype=np.float64, copy=True)
    eta_hist, mean_hist = [], []
    converged = False
    diverged = False
    iterations = 0
    final_eta = math.nan
    sig = _contract(Cs, phase, eps)
    for it in range(max_iter):
        eta, mean = equilibrium_eta(sig, k)
        eta_hist.append(eta)
        mean_hist.append(mean)
        iterations = it + 1
        final_eta = eta
        if not np.isfinite(eta) or (eta_hist[0] > 0 and eta > 1e4 * eta_hist[0]):
            diverged = True
            break
        if stop == STOP_ETA and eta <= tol and mean_strain_error(eps, eb) <= tol:
            converged = True
            break
        tau = sig - np.einsum("ijkl,kl...->ij...", C0, eps)
        tau_hat = np.fft.fftn(tau, axes=axes)
        e_hat = -apply_green(tau_hat, k, lam0, mu0, green, shape_xyz)
        e_hat[(slice(None), slice(None)) + (0,) * d] = N * eb
        e = np.fft.ifftn(e_hat, axes=axes)
        if check_real:
            scale = max(1.0, float(np.abs(e.real).max()))
            im = float(np.abs(e.imag).max())
            if im > 1e-10 * scale:
                raise AssertionError(f"inverse DFT not real: max|Im e| = {im:.3e}")
        e = e.real
        if scheme == DIRECT:
            new = e
        else:
            new = eps + omega * _contract(Ms, phase, e - eps)
        new_sig = _contract(Cs, phase, new)
        if stop == STOP_MAXDELTA:
            delta = max(float(np.abs(new - eps).max()), float(np.abs(new_sig - sig).max()))
            eps, sig = new, new_sig
            if delta < tol:
                converged = True
                break
        else:
            eps, sig = new, new_sig
    return {
        "strain": eps,
        "stress": sig,
        "mean_stress": sig.reshape(d, d, -1).mean(axis=2),
        "eta_history": np.array(eta_hist),
        "mean_stress_history": np.array(mean_hist),
        "iterations": iterations,
        "converged": converged,
        "diverged": diverged,
        "final_eta": final_eta,
        "lambda0": lam0,
        "mu0": mu0,
    }


def compliance_general(Cten, d):
    """Inverse of a (minor- and major-symmetric) stiffness on symmetric tensors."""
    M = Cten.reshape(d * d, d * d)
    I = np.eye(d)
    Psym = 0.5 * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I)).reshape(d * d, d * d)
    S = Psym @ np.linalg.pinv(M) @ Psym
    return S.reshape(d, d, d, d)


# ---------------------------------------------------------------------------
# effective stiffness
# ---------------------------------------------------------------------------
MANDEL_3D = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
MANDEL_2D = [(0, 0), (1, 1), (0, 1)]


def mandel_pairs(d):
    return MANDEL_3D if d == 3 else MANDEL_2D


def to_mandel(t: np.ndarray) -> np.ndarray:
    """Mandel vector of a symmetric tensor: shear entries scaled by sqrt(2)."""
    d = t.shape[0]
    out = []
    for (i, j) in mandel_pairs(d):
        out.append(t[i, j] if i == j else math.sqrt(2.0) * t[i, j])
    return np.array(out)


def from_mandel(v: np.ndarray, d: int) -> np.ndarray:
    t = np.zeros((d, d))
    for a, (i, j) in enumerate(mandel_pairs(d)):
        if i == j:
            t[i, i] = v[a]
        else:
            t[i, j] = t[j, i] = v[a] / math.sqrt(2.0)
    return t


def effective_stiffness(phase, lam, mu, green, scheme, **kw):
    """Effective C~ (Mandel matrix) from <sigma> = C~ eps_bar (Sec. 2), unit Mandel loads."""
    d = np.asarray(phase).ndim
    nc = 6 if d == 3 else 3
    Ceff = np.zeros((nc, nc))
    for J in range(nc):
        e = np.zeros(nc)
        e[J] = 1.0
        res = solve(phase, lam, mu, from_mandel(e, d), green, scheme, **kw)
        Ceff[:, J] = to_mandel(res["mean_stress"])
    return Ceff
