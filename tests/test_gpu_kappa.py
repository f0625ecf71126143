"""The paper's region rule (Sec. III: short-range region sized to N_F + kappa N_S,
kappa = 3/10) on the GPU against the oracle: the same clusters (dimensions and
short-range membership) and the same LNO step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import spectral_moments, state_tol, to_dev  # noqa: E402
from paper_1809_05637_gb300 import Context  # noqa: E402

KAPPA, S_FNA = 0.3, 0.05


def _ctx(s):
    ctx = Context()
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                       to_dev(s.S), 0.0, s.r_lno, s.k_lno, kappa=KAPPA, s_fna=S_FNA)
    return ctx


def test_kappa_clusters_and_step_match_oracle(cfg1):
    s = cfg1
    ctx = _ctx(s)
    dims, nmem, _ = ctx.cluster_info()
    cls = [O.cluster_members(s, i, 0.0, s.r_lno, s.k_lno, kappa=KAPPA, s_fna=S_FNA) for i in range(s.natoms)]
    assert [c.dim for c in cls] == list(dims)
    assert [len(c.atoms) for c in cls] == list(nmem)
    ncore = np.array([int(np.count_nonzero(c.core)) for c in cls])
    assert ncore.min() < nmem.min()  # the rule leaves a long-range region
    rho_in = T.synthetic_density(s, seed=21)
    ctx.compute_lnos(to_dev(rho_in))
    ctx.solve_clusters()
    mu, n = ctx.find_mu(s.n_electrons, s.kT)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e_gpu = ctx.density_matrix(mu, s.kT, out)
    spec = ctx.spectrum()
    ctx.close()
    lno = O.compute_lnos(s, rho_in, s.k_lno)
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, 0.0, s.r_lno, s.k_lno, kappa=KAPPA, s_fna=S_FNA)
    mu_o, n_o, rho_o, e_o = O.finish_step(s, res, V, s.n_electrons, s.kT)
    for i, r in res.items():
        assert np.all(np.abs(np.sort(spec[i][0]) - r.eps) <= state_tol(r)), f"cluster {i}"
        np.testing.assert_allclose(spectral_moments(spec[i][0], spec[i][1], [mu_o], s.kT),
                                   spectral_moments(r.eps, r.q, [mu_o], s.kT), rtol=0, atol=1e-9)
    assert abs(mu - mu_o) <= 1e-9
    np.testing.assert_allclose(out.cpu().numpy(), rho_o, rtol=0, atol=1e-9)
    assert abs(e_gpu - e_o) <= 1e-9 * abs(e_o)


def test_kappa_argument_checks(cfg1):
    s = cfg1
    ctx = Context()
    with pytest.raises(Exception, match="kappa"):
        ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                           to_dev(s.S), 0.0, s.r_lno, s.k_lno, kappa=1.5, s_fna=S_FNA)
    ctx.close()
