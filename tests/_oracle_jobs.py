"""Oracle runs executed in spawned worker processes by the GPU parity tests (CPU only).

A worker imports nothing from the CUDA path: it builds the seeded input and runs
the FP64 oracle, returning the strain components and the eta history."""
import numpy as np


def boolean_case(args):
    """Two (or `iters`) iterations of the oracle on the 128^3-style Boolean recipe."""
    n, radius, fraction, seed, chi, green, scheme, iters = args
    from oracle import fftls_oracle as O
    from paper_1412_8398_gb300 import microstructure as MS
    ph, _ = MS.boolean_spheres((n, n, n), radius, fraction, seed=seed)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (chi, 0.3)])
    r = O.solve(ph, lam, mu, np.diag([1.0, 0.0, 0.0]), green, scheme, tol=0.0, max_iter=iters)
    t = r["strain"]
    comp = np.stack([t[0, 0], t[1, 1], t[2, 2], t[1, 2], t[0, 2], t[0, 1]])
    return args, comp, np.asarray(r["eta_history"])
