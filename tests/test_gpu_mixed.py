"""Mixed-precision path (DCLNO_MIXED): the cubic contractions run on BF16 tensor cores
with FP64 emulated by 8-bit slices; everything else is FP64.

Against the oracle on the small systems: eigenvalues within the first-order
perturbation bound of each state (1e-10 Ha floor), weights and density-matrix
elements to 1e-9.  The full-size workloads compare the mixed form with the
oracle on sampled clusters and with the FP64 form's band energy
(test_gpu_workload_cfg2.py, test_gpu_workload_cfg5.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from gpu_helpers import gpu_context, spectral_moments, state_tol, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_MIXED  # noqa: E402


@pytest.mark.parametrize("which", ["cfg1", "mixed_system"])
def test_mixed_matches_oracle_small(which, request):
    s = request.getfixturevalue(which)
    rho0 = O.plain_dc_density(s, s.r_core)[2]
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.compute_lnos(to_dev(rho0))
    ctx.solve_clusters(DCLNO_MIXED)
    spec = ctx.spectrum()
    mus = np.linspace(-1.2, 0.0, 13)
    for i, r in res.items():
        e_gpu, q_gpu = spec[i]
        assert np.all(np.abs(np.sort(e_gpu) - r.eps) <= state_tol(r)), f"cluster {i}"
        np.testing.assert_allclose(spectral_moments(e_gpu, q_gpu, mus, s.kT),
                                   spectral_moments(r.eps, r.q, mus, s.kT), rtol=0, atol=1e-9)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(e - e_band) <= 1e-9 * abs(e_band)
    ctx.close()
