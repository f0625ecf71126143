"""Two-stage tridiagonalisation (dense -> band -> tridiagonal, k_band + k_chase)
against the oracle, in FP64 and in the mixed path, and against the one-stage form.

The tridiagonal matrix differs between the forms (T is unique only up to signs
and the choice of reflectors), the eigenpairs of the cluster pencil do not: the
same eigenvalue, weight and density-row tolerances as the one-stage parity tests
apply.  Clusters of dimension >= 128 take the two-stage form; the lattices below
have clusters on both sides of that bound and dimensions that are not multiples
of the band width (a ragged last panel and a short last chase window).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import (check_sampled_clusters, eps_tol, gpu_context, oracle_sample, rho_row_tol,  # noqa: E402
                         spectral_moments, state_tol, to_dev)
from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, DclnoError  # noqa: E402

TWO_STAGE_MIN = 128


def _ran(ctx, name):
    return ctx.kernel_time(name)[1]


@pytest.mark.parametrize("prec", [DCLNO_FP64, DCLNO_MIXED])
def test_two_stage_lno_step_cfg1(cfg1, cfg1_dc0, prec):
    s = cfg1
    rho0 = cfg1_dc0[2]
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    dims = np.array([r.cluster.dim for r in res.values()])
    assert dims.max() >= TWO_STAGE_MIN and np.any(dims % 32 != 0)

    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=2)
    ctx.set_profiling(True)
    ctx.compute_lnos(to_dev(rho0))
    ctx.solve_clusters(prec)
    assert _ran(ctx, "k_band") == 1 and _ran(ctx, "k_chase") == 1
    spec = ctx.spectrum()
    mus = np.linspace(-1.2, 0.0, 13)
    for i, r in res.items():
        e_gpu, q_gpu = spec[i]
        tol = eps_tol(r.eps) if prec == DCLNO_FP64 else state_tol(r)
        assert np.all(np.abs(np.sort(e_gpu) - r.eps) <= tol), f"cluster {i} (n = {len(r.eps)})"
        np.testing.assert_allclose(spectral_moments(e_gpu, q_gpu, mus, s.kT),
                                   spectral_moments(r.eps, r.q, mus, s.kT), rtol=0, atol=1e-9)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(e - e_band) <= 1e-9 * abs(e_band)
    # energy density matrix through the same back-transform (Eq. (edm)): 2 Tr(e S) = E_band
    edm = torch.zeros_like(out)
    e2 = ctx.density_matrices(mu, s.kT, out, edm)
    np.testing.assert_allclose(out.cpu().numpy(), rho, rtol=0, atol=1e-9)
    assert abs(2.0 * float(torch.dot(edm, to_dev(s.S))) - e2) <= 1e-9 * abs(e2)
    ctx.close()


@pytest.fixture(scope="module")
def periodic512():
    """The rock-salt recipe on 8^3 sites: cluster dimensions 648-705 as in the
    1,728-atom workload (many full panels, a ragged last one)."""
    return T.make_system(2, n_cells=8)


@pytest.mark.parametrize("prec", [DCLNO_FP64, DCLNO_MIXED])
def test_two_stage_full_size_clusters(periodic512, prec):
    s = periodic512
    rho_in = T.synthetic_density(s, seed=11)
    sample = [0, 255, 511]
    _, V, res = oracle_sample(s, rho_in, sample)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=2)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    R = to_dev(rho_in)
    per = {}
    for mode in (1, 2):
        ctx.set_tridiag(mode)
        ctx.compute_lnos(R)
        ctx.solve_clusters(prec)
        spec = ctx.spectrum()
        ctx.density_matrix(-0.25, s.kT, out)
        per[mode] = (spec, out.cpu().numpy())
    ctx.close()
    row_tol = (lambda r, big: 1e-9 + 4e-9 * big) if prec == DCLNO_FP64 else rho_row_tol
    for mode, (spec, rows) in per.items():
        we, wr = check_sampled_clusters(s, V, res, spec, rows, -0.25, row_tol, np.linspace(-0.9, 0.1, 11))
        print(f"prec {prec} tridiag {mode}: eigenvalues {we:.3g} of the bound, rows {wr:.3g} of the row max")


def test_two_stage_batches_match_single_workspace(periodic512):
    """Memory-admitted batches re-solve earlier batches for the density pass: with the
    two-stage form the result is bit for bit the single-workspace one."""
    s = periodic512
    R = to_dev(T.synthetic_density(s, seed=11))
    outs = []
    for limit in (0, None):
        ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=2) if limit == 0 else None
        if ctx is None:
            from paper_1809_05637_gb300 import Context
            probe = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=2)
            ws1 = probe.batch_info()[1]
            probe.close()
            ctx = Context()
            ctx.set_tridiag(2)
            ctx.set_workspace_limit(ws1 // 3 + (1 << 20))
            ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                               to_dev(s.S), s.r_core, s.r_lno, s.k_lno)
            assert ctx.batch_info()[0] >= 3
        out = torch.zeros_like(R)
        mu, n, e = ctx.step(R, out, s.n_electrons, s.kT, precision=DCLNO_MIXED)
        outs.append((mu, e, out.cpu().numpy()))
        ctx.close()
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][2], outs[1][2])


def test_two_stage_needs_its_layout(cfg1):
    """Mode 2 selected after a build without the chase-reflector log is refused, the
    context keeps solving in the one-stage form; modes 0 and 1 switch freely."""
    s = cfg1
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    with pytest.raises(DclnoError, match="before building"):
        ctx.set_tridiag(2)
    ctx.set_tridiag(1)
    ctx.set_tridiag(0)
    ctx.set_profiling(True)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    ctx.step(to_dev(T.synthetic_density(s, seed=3)), out, s.n_electrons, s.kT)
    assert _ran(ctx, "k_band") == 0 and _ran(ctx, "k_tridiag") >= 1
    ctx.close()
