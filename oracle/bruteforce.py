"""Dense brute-force solves of the discretised cell problems (test infrastructure only).

These do not iterate and do not use the Green operator: they minimise the
elastic energy  sum_x (eps_bar + B u)(x) : C(x) : (eps_bar + B u)(x)  over
the periodic nodal displacement u, with B the real-space strain stencil of
each discretisation, and so give the exact fixed point that the FFT schemes
must reach.  Sizes are tiny (a few hundred unknowns); numpy's least-squares
solver handles the null (rigid and checkerboard) displacement modes.

Stencils (Sec. 4):
  * C, eq. (mul1):  d_j u(x) = (u(x + e_j) - u(x - e_j)) / 2, u at voxel centres.
  * W, eq. (wil071): d_j u(x) = u(x + e_j) - u(x), u at voxel centres.
  * R, eq. (discFull) in 2D, eq. (disc3deps) in 3D: u lives at voxel corners;
    d_j u at the centre x is the difference across the voxel along e_j,
    averaged over the 2^{d-1} edges parallel to e_j.  Corner c (integer
    index) sits at c - (1/2, .., 1/2).
  eps_ij = (d_j u_i + d_i u_j) / 2.

For the operator G (MS) the reachable set is a Galerkin space (Sec. 3):
the fluctuation has zero mean, lies in the compatible fields sym(i q (x) u)
at every mode with no |q_i| = pi, and is unconstrained at the even-L modes
with some q_i = pi (where eq. hfreq sets G = C0^{-1}, i.e. sigma_hat = 0).
It is built from the explicit DFT matrix.

Strains are handled as Mandel vectors so that eps : C : eps is a dot product.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import fftls_oracle as O


def _mandel_pairs(d):
    return O.mandel_pairs(d)


def _mandel_stiffness(lam, mu, d):
    """6x6 (3x3 in 2D) Mandel matrix of the isotropic stiffness."""
    C = O.stiffness_tensor(lam, mu, d)
    pairs = _mandel_pairs(d)
    nc = len(pairs)
    M = np.zeros((nc, nc))
    for a, (i, j) in enumerate(pairs):
        for b, (k, l) in enumerate(pairs):
            fa = 1.0 if i == j else math.sqrt(2.0)
            fb = 1.0 if k == l else math.sqrt(2.0)
            M[a, b] = fa * fb * C[i, j, k, l]
    return M


def _voxel_index(shape_xyz):
    """Flat index of voxel (x1, .., xd) in numpy C order (nd, .., n1)."""
    strides = []
    s = 1
    for L in shape_xyz:
        strides.append(s)
        s *= L
    return strides


def _derivative_matrix(shape_xyz, j, green):
    """N x N matrix of the discrete derivative along axis j at voxel centres."""
    d = len(shape_xyz)
    N = int(np.prod(shape_xyz))
    strides = _voxel_index(shape_xyz)
    D = np.zeros((N, N))

    def flat(coord):
        return sum(((coord[a] % shape_xyz[a]) * strides[a]) for a in range(d))

    for x in itertools.product(*[range(L) for L in shape_xyz]):
        row = flat(x)
        if green == O.CENTERED:
            xp = list(x); xp[j] += 1
            xm = list(x); xm[j] -= 1
            D[row, flat(xp)] += 0.5
            D[row, flat(xm)] -= 0.5
        elif green == O.WILLOT:
            xp = list(x); xp[j] += 1
            D[row, flat(xp)] += 1.0
            D[row, flat(x)] -= 1.0
        elif green == O.ROTATED:
            others = [a for a in range(d) if a != j]
            w = 1.0 / 2 ** (d - 1)
            for offs in itertools.product((0, 1), repeat=d - 1):
                hi = list(x)
                lo = list(x)
                for a, o in zip(others, offs):
                    hi[a] += o
                    lo[a] += o
                hi[j] += 1
                D[row, flat(hi)] += w
                D[row, flat(lo)] -= w
        else:
            raise ValueError("stencil solve needs C, W or R")
    return D


def strain_operator(shape_xyz, green):
    """B: (d N) nodal displacements -> (nc N) Mandel strains, component-major."""
    d = len(shape_xyz)
    N = int(np.prod(shape_xyz))
    Ds = [_derivative_matrix(shape_xyz, j, green) for j in range(d)]
    pairs = _mandel_pairs(d)
    B = np.zeros((len(pairs) * N, d * N))
    for a, (i, j) in enumerate(pairs):
        f = 1.0 if i == j else math.sqrt(2.0)
        # eps_ij = (d_j u_i + d_i u_j) / 2
        B[a * N:(a + 1) * N, i * N:(i + 1) * N] += 0.5 * f * Ds[j]
        B[a * N:(a + 1) * N, j * N:(j + 1) * N] += 0.5 * f * Ds[i]
    return B


def _stiffness_blocks(phase_flat, lam, mu, d):
    """Block-diagonal (nc N)^2 stiffness, component-major ordering."""
    N = phase_flat.size
    nc = 3 if d == 2 else 6
    Cm = [_mandel_stiffness(lam[a], mu[a], d) for a in range(len(lam))]
    K = np.zeros((nc * N, nc * N))
    for x in range(N):
        Ca = Cm[phase_flat[x]]
        idx = np.arange(nc) * N + x
        K[np.ix_(idx, idx)] = Ca
    return K


def _eps_bar_mandel(eps_bar, d, N):
    t = np.asarray(eps_bar, dtype=np.float64)
    if t.ndim == 1:
        t = O._tensor_from_vector(t, d)
    v = O.to_mandel(t)
    return np.repeat(v, N)


def _mandel_to_tensor_field(v, d, grid):
    N = int(np.prod(grid))
    out = np.zeros((d, d) + grid)
    for a, (i, j) in enumerate(_mandel_pairs(d)):
        comp = v[a * N:(a + 1) * N].reshape(grid)
        if i == j:
            out[i, i] = comp
        else:
            out[i, j] = out[j, i] = comp / math.sqrt(2.0)
    return out


def solve_stencil(phase, lam, mu, eps_bar, green):
    """Exact strain field of the C / W / R discrete problem by energy minimisation."""
    phase = np.asarray(phase)
    d = phase.ndim
    shape_xyz = O.grid_shape_xyz(phase)
    N = phase.size
    B = strain_operator(shape_xyz, green)
    K = _stiffness_blocks(phase.reshape(-1), np.asarray(lam), np.asarray(mu), d)
    e0 = _eps_bar_mandel(eps_bar, d, N)
    lhs = B.T @ K @ B
    rhs = -B.T @ K @ e0
    u, *_ = np.linalg.lstsq(lhs, rhs, rcond=None)
    eps = e0 + B @ u
    return _mandel_to_tensor_field(eps, d, phase.shape)


def _ms_projector(shape_xyz):
    """Real (nc N)^2 projector onto the Galerkin fluctuation space of operator G."""
    d = len(shape_xyz)
    grid = tuple(reversed(shape_xyz))
    N = int(np.prod(shape_xyz))
    pairs = _mandel_pairs(d)
    nc = len(pairs)
    # 1D DFT matrices per axis, combined with Kronecker products in numpy order
    F = np.ones((1, 1), dtype=np.complex128)
    for L in reversed(shape_xyz):  # numpy order: outermost axis first
        m = np.arange(L)
        F1 = np.exp(-2j * np.pi * np.outer(m, m) / L)
        F = np.kron(F, F1)
    Finv = np.conj(F).T / N
    nyq = O.nyquist_mask(shape_xyz).reshape(-1)
    qs = []
    for i, L in enumerate(shape_xyz):
        s = O.signed_modes(L)
        qs.append(O._axis_array(2.0 * np.pi * s / L, i, d) * np.ones(grid))
    qv = np.stack([q.reshape(-1) for q in qs])   # (d, N)
    P = np.zeros((N, nc, nc))
    for m in range(N):
        if m == 0:
            continue
        if nyq[m]:
            P[m] = np.eye(nc)
            continue
        q = qv[:, m]
        cols = []
        for a in range(d):
            u = np.zeros(d)
            u[a] = 1.0
            t = 0.5 * (np.outer(q, u) + np.outer(u, q))
            cols.append(O.to_mandel(t))
        Q, _ = np.linalg.qr(np.array(cols).T)
        P[m] = Q @ Q.T
    big = np.zeros((nc * N, nc * N), dtype=np.complex128)
    for a in range(nc):
        for b in range(nc):
            big[a * N:(a + 1) * N, b * N:(b + 1) * N] = Finv @ (P[:, a, b][:, None] * F)
    assert np.abs(big.imag).max() < 1e-10
    return big.real


def solve_galerkin_ms(phase, lam, mu, eps_bar):
    """Exact strain field of the operator-G (MS) scheme: energy minimum over eps_bar + W0."""
    phase = np.asarray(phase)
    d = phase.ndim
    shape_xyz = O.grid_shape_xyz(phase)
    N = phase.size
    P = _ms_projector(shape_xyz)
    w, V = np.linalg.eigh(0.5 * (P + P.T))
    V = V[:, w > 0.5]
    K = _stiffness_blocks(phase.reshape(-1), np.asarray(lam), np.asarray(mu), d)
    e0 = _eps_bar_mandel(eps_bar, d, N)
    a = np.linalg.solve(V.T @ K @ V, -V.T @ K @ e0)
    eps = e0 + V @ a
    return _mandel_to_tensor_field(eps, d, phase.shape)


def divergence_field(sig, green):
    """Real-space discrete divergence of sigma whose symbol is k*(q) (Sec. 4).

    It is the adjoint of the strain stencil: (div s)_j = -sum_i D_i^T s_ij,
    so its Fourier symbol is (k*) . s up to sign; used to pin eta by Parseval.
    """
    d = sig.shape[0]
    shape_xyz = tuple(reversed(sig.shape[2:]))
    N = int(np.prod(shape_xyz))
    Ds = [_derivative_matrix(shape_xyz, i, green) for i in range(d)]
    out = np.zeros((d, N))
    for j in range(d):
        for i in range(d):
            out[j] -= Ds[i].T @ sig[i, j].reshape(-1)
    return out
