"""Threshold selection of LNOs (Sec. II.B step (iii): the eigenvectors of Lambda with
eigenvalue >= lambda_th, 0.1 in the paper) on the GPU against the oracle: the same
per-atom counts, cluster dimensions, spectra and density-matrix rows; switching the
threshold off restores the fixed-count layout.  The input density scales the rows
of every third atom by 1.5, so that at lambda_th = 0.3 the atoms keep one or two
LNOs (42 and 22 of them)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import gpu_context, spectral_moments, state_tol, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DclnoError  # noqa: E402

LAMBDA_TH = 0.3
K_MAX = 4


def test_threshold_step_matches_oracle(cfg1):
    s = cfg1
    rho0 = T.synthetic_density(s, seed=3)
    for i in range(0, s.natoms, 3):
        rho0[s.blk_off[s.row_ptr[i]]:s.blk_off[s.row_ptr[i + 1] - 1] + 16] *= 1.5
    ctx = gpu_context(s, s.r_core, s.r_lno, K_MAX)
    dims_fixed = ctx.cluster_info()[0].copy()
    ctx.set_lno_threshold(LAMBDA_TH)
    ctx.compute_lnos(to_dev(rho0))
    counts = ctx.lno_counts()
    lno = O.compute_lnos(s, rho0, K_MAX, lambda_th=LAMBDA_TH)
    ko = np.array([lno[j][0].shape[1] for j in range(s.natoms)])
    for j in np.nonzero(counts != ko)[0]:  # only an eigenvalue within rounding of lambda_th may differ
        assert np.min(np.abs(lno[j][1].real - LAMBDA_TH)) < 1e-9, f"atom {j}"
    assert set(counts.tolist()) == {1, 2}
    V = {j: v[0] for j, v in lno.items()}
    kat = {j: int(counts[j]) for j in range(s.natoms)}
    Vg = ctx.lnos()
    for j in range(s.natoms):
        kj = kat[j]
        np.testing.assert_allclose(Vg[j][0][:, :kj] @ Vg[j][0][:, :kj].T, V[j][:, :kj] @ V[j][:, :kj].T,
                                   rtol=0, atol=1e-9)
        assert not np.any(Vg[j][0][:, kj:])
    ctx.solve_clusters()
    mu, n = ctx.find_mu(s.n_electrons, s.kT)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e_gpu = ctx.density_matrix(mu, s.kT, out)
    spec = ctx.spectrum()
    dims = ctx.cluster_info()[0]
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, K_MAX, k_atoms=kat)
    mu_o, n_o, rho_o, e_o = O.finish_step(s, res, V, s.n_electrons, s.kT)
    assert [len(r.eps) for _, r in sorted(res.items())] == list(dims)
    assert np.all(dims <= dims_fixed) and np.any(dims < dims_fixed)
    for i, r in res.items():
        assert np.all(np.abs(np.sort(spec[i][0]) - r.eps) <= state_tol(r)), f"cluster {i}"
        np.testing.assert_allclose(spectral_moments(spec[i][0], spec[i][1], [mu_o], s.kT),
                                   spectral_moments(r.eps, r.q, [mu_o], s.kT), rtol=0, atol=1e-9)
    assert abs(mu - mu_o) <= 1e-9
    np.testing.assert_allclose(out.cpu().numpy(), rho_o, rtol=0, atol=1e-9)
    assert abs(e_gpu - e_o) <= 1e-9 * abs(e_o)
    # the graph-captured SCF loop cannot re-lay out the clusters between steps
    with pytest.raises(DclnoError, match="threshold"):
        ctx.scf_run(to_dev(rho0.copy()), 1, 0.3, s.n_electrons, s.kT, use_graph=False)
    # threshold off: every atom back to K_MAX and the fixed-count dimensions
    ctx.set_lno_threshold(None)
    ctx.compute_lnos(to_dev(rho0))
    assert np.all(ctx.lno_counts() == K_MAX)
    np.testing.assert_array_equal(ctx.cluster_info()[0], dims_fixed)
    ctx.close()
