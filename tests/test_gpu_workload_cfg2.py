"""The 1,728-atom gapped rock-salt workload at full size, in the benchmark's launch
configuration (all clusters in one batch, FP64).

Sampled clusters are recomputed by the oracle one by one from the same seeded
input density; every other check is a property that holds at any size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import fermi, gpu_context, spectral_moments, state_tol, to_dev  # noqa: E402

SAMPLE = [0, 777, 1727]
MU_TEST = -0.25  # a fixed chemical potential for element-wise rho comparison


@pytest.fixture(scope="module")
def run():
    s = T.make_system(2)
    rho_in = T.synthetic_density(s, seed=11)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.compute_lnos(to_dev(rho_in))
    ctx.solve_clusters()
    mu, n = ctx.find_mu(s.n_electrons, s.kT)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e_band = ctx.density_matrix(mu, s.kT, out)
    rho_mu = out.cpu().numpy()
    spec = ctx.spectrum()
    lnos = ctx.lnos()
    dims = ctx.cluster_info()[0]
    e_test = ctx.density_matrix(MU_TEST, s.kT, out)
    rho_test = out.cpu().numpy()
    ctx.close()
    return dict(s=s, rho_in=rho_in, mu=mu, n=n, e_band=e_band, rho_mu=rho_mu, spec=spec, lnos=lnos, dims=dims,
                rho_test=rho_test, e_test=e_test)


def test_cluster_sizes(run):
    dims = run["dims"]
    assert dims.min() >= 500 and dims.max() <= 800


def test_sampled_clusters_match_oracle(run):
    s = run["s"]
    need = set()
    cls = {i: O.cluster_members(s, i, s.r_core, s.r_lno, s.k_lno) for i in SAMPLE}
    for cl in cls.values():
        need |= {int(a) for a, c in zip(cl.atoms, cl.core) if not c}
    lno = O.compute_lnos(s, run["rho_in"], s.k_lno, atoms=sorted(need))
    for j, (Vo, evo, flo) in lno.items():
        Vg, evg, flg = run["lnos"][j]
        np.testing.assert_allclose(evg, evo, rtol=0, atol=1e-10)
        np.testing.assert_allclose(Vg @ Vg.T, Vo @ Vo.T, rtol=0, atol=1e-9)
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno, atoms=SAMPLE, threads=len(SAMPLE))
    mus = np.linspace(-0.9, 0.1, 11)
    for i, r in res.items():
        e_gpu, q_gpu = run["spec"][i]
        tol = state_tol(r)
        assert np.all(np.abs(np.sort(e_gpu) - r.eps) <= tol), f"cluster {i}: eigenvalues"
        # weights through smooth spectral sums; the eigenvalue bound propagated through f'
        for x in mus:
            g = spectral_moments(e_gpu, q_gpu, [x], s.kT)[0]
            o = spectral_moments(r.eps, r.q, [x], s.kT)[0]
            f = fermi((r.eps - x) / s.kT)
            fp = f * (1.0 - f) / s.kT
            assert abs(g - o) <= 1e-9 + float(np.sum(fp * tol * np.abs(r.q))), f"cluster {i}: weights at {x}"
        rows = np.zeros_like(s.S)
        O.density_rows(s, r.cluster, r.eps, r.C, V, MU_TEST, s.kT, rows)
        b0, b1 = s.row_ptr[i], s.row_ptr[i + 1]
        o0 = s.blk_off[b0]
        o1 = s.blk_off[b1 - 1] + s.norb[i] * s.norb[s.col[b1 - 1]]
        # elements relative to the row's largest element: rows reach 1e4 where the
        # nearly dependent basis gives large coefficients (cond S^(i) ~ 3e7)
        big = float(np.max(np.abs(rows[o0:o1])))
        np.testing.assert_allclose(run["rho_test"][o0:o1], rows[o0:o1], rtol=0, atol=1e-9 + 4e-9 * big)


def test_invariants_at_full_size(run):
    s = run["s"]
    for i, (e, q) in enumerate(run["spec"]):
        assert abs(q.sum() - s.norb[i]) < 1e-8
    assert abs(run["n"] - s.n_electrons) <= 1e-10 * s.n_electrons
    rho = run["rho_mu"]
    assert abs(2 * float(np.dot(rho, s.S)) - run["n"]) < 1e-8 * s.n_electrons
    assert abs(2 * float(np.dot(rho, s.H)) - run["e_band"]) < 1e-8 * abs(run["e_band"])
