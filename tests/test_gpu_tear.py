"""Cuppen's tear applied twice (four QL segments, the halves merged first, then the
halves merged: dclno_set_tear), in both precisions and both tridiagonalisation forms,
against the oracle (which diagonalises each cluster whole); the pole form of the
density undoes all three tears.  The full-size workloads take the automatic mode,
which tears clusters of dimension >= 512 twice (tests/test_gpu_workload_cfg2.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import eps_tol, gpu_context, spectral_moments, state_tol, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, DclnoError  # noqa: E402


@pytest.mark.parametrize("prec,tridiag", [(DCLNO_FP64, 1), (DCLNO_FP64, 2), (DCLNO_MIXED, 1), (DCLNO_MIXED, 2)])
def test_tear_twice_lno_step_cfg1(cfg1, cfg1_dc0, prec, tridiag):
    s = cfg1
    rho0 = cfg1_dc0[2]
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    dims = np.array([r.cluster.dim for r in res.values()])
    assert dims.min() >= 64  # every cluster torn twice

    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=tridiag, tear=2)
    ctx.compute_lnos(to_dev(rho0))
    ctx.solve_clusters(prec)
    spec = ctx.spectrum()
    mus = np.linspace(-1.2, 0.0, 13)
    for i, r in res.items():
        e_gpu, q_gpu = spec[i]
        tol = eps_tol(r.eps) if prec == DCLNO_FP64 else state_tol(r)
        assert np.all(np.abs(np.sort(e_gpu) - r.eps) <= tol), f"cluster {i} (n = {len(r.eps)})"
        assert abs(q_gpu.sum() - s.norb[i]) < 1e-9
        np.testing.assert_allclose(spectral_moments(e_gpu, q_gpu, mus, s.kT),
                                   spectral_moments(r.eps, r.q, mus, s.kT), rtol=0, atol=1e-9)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(e - e_band) <= 1e-9 * abs(e_band)
    edm = torch.zeros_like(out)
    e2 = ctx.density_matrices(mu, s.kT, out, edm)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(2.0 * float(torch.dot(edm, to_dev(s.S))) - e2) <= 1e-9 * abs(e2)
    ctx.close()


def test_tear_once_and_twice_agree(cfg1, cfg1_dc0):
    """The same step torn once and torn twice: eigenvalues and density rows agree to
    rounding (well-conditioned clusters)."""
    s = cfg1
    R = to_dev(cfg1_dc0[2])
    got = {}
    for tear in (1, 2):
        ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tear=tear)
        out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
        mu, n, eb = ctx.step(R, out, s.n_electrons, s.kT)
        got[tear] = (mu, eb, np.concatenate([np.sort(e) for e, _ in ctx.spectrum()]), out.cpu().numpy())
        ctx.close()
    assert abs(got[1][0] - got[2][0]) < 1e-11
    np.testing.assert_allclose(got[1][2], got[2][2], rtol=0, atol=1e-11)
    np.testing.assert_allclose(got[1][3], got[2][3], rtol=0, atol=1e-11)


def test_tear_twice_batches_and_poles():
    """Torn twice on a periodic lattice: memory-admitted batches give the single-workspace
    bits, and the pole form (three tears undone) matches the spectral rows."""
    import math

    s = T.small_lattice(5, 5, 5, a=2.5, exps=(0.5, 1.5), onsite=(-0.4, 0.2), e_per_atom=2.0, r_core=5.0,
                        r_lno=8.0, k_lno=1, periodic=True)
    R = to_dev(T.synthetic_density(s, seed=3))
    outs = []
    for limit in (0, 3):
        from paper_1809_05637_gb300 import Context

        ctx = Context()
        ctx.set_tear(2)
        if limit:
            probe = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tear=2)
            ws1 = probe.batch_info()[1]
            probe.close()
            ctx.set_workspace_limit(ws1 // limit + (1 << 20))
        ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                           to_dev(s.S), s.r_core, s.r_lno, s.k_lno)
        assert ctx.cluster_info()[0].min() >= 64
        if limit:
            assert ctx.batch_info()[0] >= 2
        out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
        mu, n, eb = ctx.step(R, out, s.n_electrons, s.kT)
        outs.append((mu, eb, out.cpu().numpy()))
        if not limit:
            rad = max(float(np.max(np.abs(e - mu))) for e, _ in ctx.spectrum())
            npoles = int(40.0 * rad / (2.0 * math.pi * s.kT)) + 1
            pole = torch.zeros_like(out)
            ctx.density_matrix(mu, s.kT, out)
            spec = out.cpu().numpy()
            ctx.density_matrix_poles(mu, s.kT, npoles, pole)
            np.testing.assert_allclose(pole.cpu().numpy(), spec, rtol=0, atol=1e-9)
        ctx.close()
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1]
    np.testing.assert_array_equal(outs[0][2], outs[1][2])


def test_tear_mode_is_fixed_at_the_build(cfg1):
    s = cfg1
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    with pytest.raises(DclnoError, match="before building"):
        ctx.set_tear(2)
    ctx.set_tear(0)  # the mode it was built with
    with pytest.raises(DclnoError):
        ctx.set_tear(3)
    ctx.close()
