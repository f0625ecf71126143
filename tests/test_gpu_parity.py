"""GPU path (C ABI) against the oracle, element by element, on small seeded systems.

Tolerances: eigenvalues 1e-10 Ha (+1e-12 |eps| for the large spurious states of
the nearly dependent Gaussian basis), density-matrix elements 1e-9, chemical
potential through N(mu) = N_e.  Degenerate eigenvalues make individual weights
q_mu basis-dependent, so weights are compared through smooth spectral sums
sum_mu f((eps_mu - x)/kT) q_mu, which are invariant.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import eps_tol, gpu_context, spectral_moments, to_dev  # noqa: E402
from paper_1809_05637_gb300 import Context, DclnoError  # noqa: E402


def _compare_spectra(ctx, res, kT, mus):
    spec = ctx.spectrum()
    for i, r in res.items():
        e_gpu, q_gpu = spec[i]
        assert len(e_gpu) == len(r.eps)
        es = np.sort(e_gpu)
        assert np.all(np.abs(es - r.eps) <= eps_tol(r.eps)), f"cluster {i}: eigenvalues"
        assert abs(q_gpu.sum() - r.q.sum()) < 1e-9
        m_g = spectral_moments(e_gpu, q_gpu, mus, kT)
        m_o = spectral_moments(r.eps, r.q, mus, kT)
        np.testing.assert_allclose(m_g, m_o, rtol=0, atol=1e-9, err_msg=f"cluster {i}: weights")
    return spec


def _n_of_mu(res, mu, kT):
    return O.n_of_mu(np.concatenate([r.eps for r in res.values()]), np.concatenate([r.q for r in res.values()]),
                     mu, kT)


def test_plain_dc_cfg1(cfg1, cfg1_dc0):
    s = cfg1
    mu0, n0, rho0, e0, res = cfg1_dc0
    ctx = gpu_context(s, s.r_core, s.r_core, 0)
    dims, nmem, tot = ctx.cluster_info()
    assert [int(d) for d in dims] == [res[i].cluster.dim for i in range(s.natoms)]
    ctx.compute_lnos(None)
    ctx.solve_clusters()
    _compare_spectra(ctx, res, s.kT, np.linspace(-1.2, -0.4, 9))
    mu, n = ctx.find_mu(s.n_electrons, s.kT)
    assert abs(n - s.n_electrons) <= 1e-10 * s.n_electrons
    assert abs(_n_of_mu(res, mu, s.kT) - s.n_electrons) <= 1e-9 * s.n_electrons
    rho = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e = ctx.density_matrix(mu0, s.kT, rho)
    np.testing.assert_allclose(rho.cpu().numpy(), rho0, rtol=0, atol=1e-9)
    assert abs(e - e0) <= 1e-9 * abs(e0)
    ctx.close()


def test_lno_step_cfg1(cfg1, cfg1_dc0):
    s = cfg1
    rho0 = cfg1_dc0[2]
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)

    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.compute_lnos(to_dev(rho0))
    g = ctx.lnos()
    for i, (Vo, evo, flo) in lno.items():
        Vg, evg, flg = g[i]
        assert flg == flo
        np.testing.assert_allclose(evg, evo, rtol=0, atol=1e-10)
        np.testing.assert_allclose(Vg @ Vg.T, Vo @ Vo.T, rtol=0, atol=1e-9)
        np.testing.assert_allclose(Vg, Vo, rtol=0, atol=1e-9)
    ctx.solve_clusters()
    _compare_spectra(ctx, res, s.kT, np.linspace(-1.2, -0.4, 9))
    mu_g, n_g = ctx.find_mu(s.n_electrons, s.kT)
    assert abs(_n_of_mu(res, mu_g, s.kT) - s.n_electrons) <= 1e-9 * s.n_electrons
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(e - e_band) <= 1e-9 * abs(e_band)
    # rho and the energy density matrix together (Eq. (edm))
    edm = torch.zeros_like(out)
    e2 = ctx.density_matrices(mu, s.kT, out, edm)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    np.testing.assert_allclose(edm.cpu().numpy(), O.energy_density(s, res, V, mu, s.kT), rtol=0, atol=1e-9)
    assert e2 == e
    ctx.close()


def test_mixed_basis(mixed_system):
    s = mixed_system
    mu0, n0, rho0, e0, _ = O.plain_dc_density(s, s.r_core)
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    mu_g, n_g, e_g = ctx.step(to_dev(rho0), out, s.n_electrons, s.kT)
    _compare_spectra(ctx, res, s.kT, np.linspace(-1.0, 0.0, 11))
    assert abs(n_g - s.n_electrons) <= 1e-10 * s.n_electrons
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(e - e_band) <= 1e-9 * abs(e_band)
    ctx.close()


def test_full_cover_matches_exact(cfg1, cfg1_exact):
    s = cfg1
    eps, C, mu, n_mu, rho_ex, e_ex = cfg1_exact
    ctx = gpu_context(s, 13.5, 13.5, 0)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    mu_g, n_g, e_g = ctx.step(None, out, s.n_electrons, s.kT)
    for e_gpu, q_gpu in ctx.spectrum():
        assert np.all(np.abs(np.sort(e_gpu) - eps) <= eps_tol(eps))
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho_ex, rtol=0, atol=1e-9)
    assert abs(e - e_ex) <= 1e-9 * abs(e_ex)
    ctx.close()


def test_host_buffer_step_equals_device_step(mixed_system):
    s = mixed_system
    rho0 = O.plain_dc_density(s, s.r_core)[2]
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    d_out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    a = ctx.step(to_dev(rho0), d_out, s.n_electrons, s.kT)
    h_out = np.zeros(len(s.S))
    b = ctx.step(np.ascontiguousarray(rho0), h_out, s.n_electrons, s.kT, host_buffers=True)
    assert a == b
    np.testing.assert_array_equal(d_out.cpu().numpy(), h_out)
    ctx.close()


def test_single_atom():
    s = T.small_lattice(1, 1, 1, r_core=3.0, r_lno=3.0, k_lno=0)
    eps, C, mu, n_mu, rho_ex, e_ex = O.full_diag(s)
    ctx = gpu_context(s, 3.0, 3.0, 0)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    ctx.step(None, out, s.n_electrons, s.kT)
    assert np.all(np.abs(np.sort(ctx.spectrum()[0][0]) - eps) <= eps_tol(eps))
    ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho_ex, rtol=0, atol=1e-9)
    ctx.close()


def test_errors_are_reported(cfg1):
    s = cfg1
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    with pytest.raises(DclnoError) as e:
        ctx.solve_clusters()
    assert e.value.status == 8  # LNOs not computed
    ctx.close()
    ctx = gpu_context(s, s.r_core, s.r_core, 0)
    ctx.solve_clusters()
    with pytest.raises(DclnoError) as e:
        ctx.find_mu(10 * s.n_electrons, s.kT)
    assert e.value.status == 5  # no bracket
    ctx.close()
    # a corrupted overlap (negative on-site diagonal of atom 0) must give NOT_SPD
    S_bad = s.S.copy()
    b = next(b for b in range(s.row_ptr[0], s.row_ptr[1]) if s.col[b] == 0 and not np.any(s.shift[b]))
    S_bad[s.blk_off[b]] = -1.0
    ctx = gpu_context(s, s.r_core, s.r_core, 0, S=to_dev(S_bad))
    with pytest.raises(DclnoError) as e:
        ctx.solve_clusters()
    assert e.value.status == 4
    ctx.close()


def test_empty_system_and_call_order_are_refused():
    """No atoms: refused with an argument error (no kernel runs); calls out of order
    on an unbuilt context are refused the same way."""
    ctx = Context()
    empty = torch.zeros(0, dtype=torch.float64, device="cuda:0")
    with pytest.raises(DclnoError) as e:
        ctx.build_clusters(np.zeros((0, 3)), np.eye(3) * 10.0, np.zeros(3, bool), np.zeros(0, np.int32),
                           np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros((0, 3), np.int8),
                           np.zeros(0, np.int64), empty, empty, 3.0, 6.0, 2)
    assert e.value.status == 1 and "empty" in str(e.value)
    for call in (lambda: ctx.compute_lnos(empty), lambda: ctx.solve_clusters(),
                 lambda: ctx.find_mu(2.0, 0.01)):
        with pytest.raises(DclnoError) as e:
            call()
        assert e.value.status == 1
    ctx.close()

