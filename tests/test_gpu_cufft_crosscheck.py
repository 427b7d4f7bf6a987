"""GPU: the library's fused FP32 path against an unfused cuFFT pipeline.

The pipeline in bench.py (torch elementwise kernels + cuFFT real transforms of
sigma and tau, G' of G^R applied per mode) computes the same AS iteration from
the paper's formulas independently of the library's kernels; after three
iterations both give the same eta history and strain field to FP32 rounding.
"""
import numpy as np
import pytest

from paper_1412_8398_gb300 import microstructure as MS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [(32, 32, 32), (48, 40, 64)])
def test_fused_path_matches_cufft_pipeline(n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_1412_8398_gb300 import build, fftls
    build.build()
    ph, _ = MS.boolean_spheres(n, 3.0, 0.25, seed=3)
    lam, mu = MS.young_poisson_phases([(1.0, 0.3), (1000.0, 0.2)])
    dph = torch.from_numpy(ph).cuda()
    l0, m0 = fftls.reference_medium(lam, mu, 3, "AS")
    base = bench.CufftBaseline(dph, lam, mu, l0, m0, [1.0, 0, 0, 0, 0, 0])
    etas = [base.step() for _ in range(3)]
    s = fftls.Solver(0)
    try:
        r = s.solve(dph, lam, mu, np.diag([1.0, 0, 0]), "R", "AS", tol=0.0, max_iter=3, precision="fp32",
                    device_outputs=True, want_stress=False)
    finally:
        s.close()
    np.testing.assert_allclose(r.eta_history[:3], etas, rtol=2e-4)
    got = r.strain.float()
    assert float((got - base.eps).abs().max()) < 2e-4 * float(base.eps.abs().max())
