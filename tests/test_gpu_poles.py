"""Density-matrix rows from the Matsubara pole sum on the GPU (the paper's Appendix,
Eq. (rho0j) in a non-orthogonal basis; dclno_density_matrix_poles), against the
oracle's pole sum and against the spectral route (Eq. (dm) with Eq. (Gi)): the
paper states the two give the same density matrix.

Narrow-spectrum systems (two s-Gaussians per atom, exponents 0.5 and 1.5, spectra a
few hartree wide) keep the pole count in the thousands; the count follows the
oracle's pin, the first omitted pole at 40 times the cluster's spectral radius
about mu.  The 7^3 periodic lattice has clusters of dimension 180: the torn
tridiagonal matrix (Cuppen's tear undone for the pole sum) and the two-stage
reduction both take part.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import gpu_context, row_range, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, DclnoError  # noqa: E402


def _poles(rad, kT):
    return int(40.0 * rad / (2.0 * math.pi * kT)) + 1


def test_poles_match_oracle_pole_sum():
    """The oracle's pin system (3^3 open lattice): every cluster's rows from the GPU pole
    sum against the oracle's pole sum with the same pole count and tail, and against
    the spectral rows."""
    s = T.small_lattice(3, 3, 3, a=2.5, exps=(0.5, 1.5), onsite=(-0.4, 0.2), e_per_atom=2.0, r_core=3.0,
                        r_lno=6.0, k_lno=1)
    rho0 = O.plain_dc_density(s, s.r_core)[2]
    lno = O.compute_lnos(s, rho0, 1)
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, 1)
    mu = O.finish_step(s, res, V, s.n_electrons, s.kT)[0]
    rad = max(float(np.max(np.abs(r.eps - mu))) for r in res.values())
    npoles = _poles(rad, s.kT)
    spec = np.zeros_like(s.S)
    pole = np.zeros_like(s.S)
    for i, r in res.items():
        Hc, Sc = O.assemble(s, r.cluster, V)
        O.density_rows(s, r.cluster, r.eps, r.C, V, mu, s.kT, spec)
        O.density_rows_poles(s, r.cluster, Hc, Sc, V, mu, s.kT, pole, npoles)
    ctx = gpu_context(s, s.r_core, s.r_lno, 1)
    ctx.compute_lnos(to_dev(rho0))
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    ctx.density_matrix_poles(mu, s.kT, npoles, out)
    g = out.cpu().numpy()
    ctx.close()
    np.testing.assert_allclose(g, pole, rtol=0, atol=1e-11)
    np.testing.assert_allclose(g, spec, rtol=0, atol=1e-10)


@pytest.fixture(scope="module")
def lattice7():
    return T.small_lattice(7, 7, 7, a=2.5, exps=(0.5, 1.5), onsite=(-0.4, 0.2), e_per_atom=2.0, r_core=5.0,
                           r_lno=8.0, k_lno=1, periodic=True)


@pytest.mark.parametrize("prec,mode", [(DCLNO_FP64, 1), (DCLNO_FP64, 2), (DCLNO_MIXED, 0)])
def test_poles_match_spectral_rows(lattice7, prec, mode):
    """All 343 clusters (dimension 180): pole rows against the spectral rows of the
    same GPU reduction form, and sampled clusters against the oracle's spectral rows."""
    s = lattice7
    rho_in = T.synthetic_density(s, seed=3)
    R = to_dev(rho_in)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=mode)
    dims = ctx.cluster_info()[0]
    assert dims.min() >= 128
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    ctx.compute_lnos(R)
    ctx.solve_clusters(prec)
    mu, _ = ctx.find_mu(s.n_electrons, s.kT)
    rad = max(float(np.max(np.abs(e - mu))) for e, _ in ctx.spectrum())
    npoles = _poles(rad, s.kT)
    ctx.density_matrix(mu, s.kT, out)
    spec = out.cpu().numpy()
    ctx.set_profiling(True)
    ctx.density_matrix_poles(mu, s.kT, npoles, out, precision=prec)
    assert ctx.kernel_time("k_poles")[1] == 1
    pole = out.cpu().numpy()
    ctx.close()
    np.testing.assert_allclose(pole, spec, rtol=0, atol=1e-9)
    # sampled clusters against the oracle
    sample = [0, 171]
    need = set()
    for i in sample:
        cl = O.cluster_members(s, i, s.r_core, s.r_lno, s.k_lno)
        need |= {int(a) for a, c in zip(cl.atoms, cl.core) if not c}
    lno = O.compute_lnos(s, rho_in, s.k_lno, atoms=sorted(need))
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno, atoms=sample, threads=2)
    rows = np.zeros_like(s.S)
    for i, r in res.items():
        O.density_rows(s, r.cluster, r.eps, r.C, V, mu, s.kT, rows)
        o0, o1 = row_range(s, i)
        np.testing.assert_allclose(pole[o0:o1], rows[o0:o1], rtol=0, atol=1e-9)


def test_poles_refuse_too_few(lattice7):
    """A pole count whose first omitted pole lies inside the cluster spectrum is refused
    (the tail expansion would diverge), and the context stays usable."""
    s = lattice7
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    R = to_dev(T.synthetic_density(s, seed=3))
    ctx.compute_lnos(R)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    with pytest.raises(DclnoError, match="too few poles"):
        ctx.density_matrix_poles(0.0, s.kT, 4, out)
    ctx.solve_clusters()
    mu, n = ctx.find_mu(s.n_electrons, s.kT)
    assert abs(n - s.n_electrons) <= 1e-10 * s.n_electrons
    ctx.close()
