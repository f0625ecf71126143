"""Pins of the DC-LNO oracle against what the method and the mathematics fix.

* full-cover exactness: a cluster that holds the whole open system reproduces
  conventional diagonalisation (the DC method is exact in that limit);
* all-LNO identity: keeping every eigenvector of Lambda makes Eq. (apop_Lambda)
  exact, so DC-LNO equals plain-PAO DC on the same radius;
* invariants: sum_mu q_mu = M_i, 2 Tr(rho S) = N(mu), E_band = 2 sum tr(rho H),
  sum_i tr Lambda_i = N_ele / 2 (Eq. (tr_i));
* Lambda against the dense product (rho S)_ii; eigenvalue range of Table I;
* the worked dimension / cost-model numbers of Sec. IV.C and Fig. 7.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
import tbsystems as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def eps_tol(e):
    """Eigenvalue tolerance: 1e-10 Ha, relative 1e-12 for the large spurious states."""
    return 1e-10 + 1e-12 * np.abs(e)


def test_full_diag_brute_force(cfg1, cfg1_exact):
    eps = cfg1_exact[0]
    H, S, _ = O.dense_matrices(cfg1)
    ref = sl.eigh(H, S, eigvals_only=True)
    assert np.all(np.abs(eps - ref) <= eps_tol(ref))
    assert abs(cfg1_exact[3] - cfg1.n_electrons) < 1e-9


def test_full_cover_exactness(cfg1, cfg1_exact):
    eps, C, mu, nmu, rho, e_band = cfg1_exact
    res = O.dclno_solve(cfg1, {}, 13.5, 13.5, 0)
    for r in res.values():
        assert r.cluster.dim == len(eps)
        assert np.all(np.abs(r.eps - eps) <= eps_tol(eps))
    mu2, n2, rho2, e2 = O.finish_step(cfg1, res, {}, cfg1.n_electrons, cfg1.kT)
    assert abs(mu2 - mu) < 1e-9
    assert np.max(np.abs(rho2 - rho)) < 1e-9
    assert abs(e2 - e_band) < 1e-9 * abs(e_band)


def test_all_lno_identity(cfg1, cfg1_dc0):
    rho0 = cfg1_dc0[2]
    lno = O.compute_lnos(cfg1, rho0, 4)
    V = {i: v[0] for i, v in lno.items()}
    a = O.dclno_solve(cfg1, V, 5.0, 8.0, 4)
    b = O.dclno_solve(cfg1, {}, 8.0, 8.0, 0)
    for i in a:
        assert a[i].cluster.dim == b[i].cluster.dim
        assert np.all(np.abs(a[i].eps - b[i].eps) <= eps_tol(b[i].eps))
        np.testing.assert_allclose(a[i].q, b[i].q, atol=1e-9)
    mua, na, rhoa, ea = O.finish_step(cfg1, a, V, cfg1.n_electrons, cfg1.kT)
    mub, nb, rhob, eb = O.finish_step(cfg1, b, {}, cfg1.n_electrons, cfg1.kT)
    assert abs(mua - mub) < 1e-9
    assert np.max(np.abs(rhoa - rhob)) < 1e-9
    assert abs(ea - eb) < 1e-9 * abs(eb)


@pytest.fixture(scope="module")
def lno_step(cfg1, cfg1_dc0):
    rho0 = cfg1_dc0[2]
    lno = O.compute_lnos(cfg1, rho0, cfg1.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(cfg1, V, cfg1.r_core, cfg1.r_lno, cfg1.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(cfg1, res, V, cfg1.n_electrons, cfg1.kT)
    return lno, V, res, mu, n_mu, rho, e_band


def _pair_trace(s, rho, X):
    brow = s.block_rows()
    tot = 0.0
    for b in range(s.nnzb):
        i = int(brow[b])
        mi, mj = int(s.norb[i]), int(s.norb[s.col[b]])
        o = int(s.blk_off[b])
        tot += float(np.sum(rho[o:o + mi * mj] * X[o:o + mi * mj]))
    return tot


def test_invariants(cfg1, lno_step):
    lno, V, res, mu, n_mu, rho, e_band = lno_step
    for i, r in res.items():
        assert abs(r.q.sum() - cfg1.norb[i]) < 1e-10
    assert abs(n_mu - cfg1.n_electrons) <= 1e-10 * cfg1.n_electrons
    assert abs(2 * _pair_trace(cfg1, rho, cfg1.S) - n_mu) < 1e-9
    assert abs(2 * _pair_trace(cfg1, rho, cfg1.H) - e_band) < 1e-9 * abs(e_band)
    lam = O.lambda_blocks(cfg1, rho)
    assert abs(sum(np.trace(x) for x in lam.values()) - n_mu / 2) < 1e-9


def test_lno_quality(cfg1, cfg1_exact, cfg1_dc0, lno_step):
    """Error per atom against exact diagonalisation: DC-LNO beats plain core-only DC."""
    e_exact = cfg1_exact[5]
    e_dc0 = cfg1_dc0[3]
    e_lno = lno_step[6]
    n = cfg1.natoms
    assert abs(e_lno - e_exact) / n < abs(e_dc0 - e_exact) / n < 5e-2


def test_lambda_matches_dense_product(mixed_system):
    import tbsystems
    s = mixed_system
    rho = tbsystems.synthetic_density(s, seed=2)
    H, S, off = O.dense_matrices(s)
    R = np.zeros_like(S)
    brow = s.block_rows()
    for b in range(s.nnzb):
        i, j = int(brow[b]), int(s.col[b])
        R[off[i]:off[i + 1], off[j]:off[j + 1]] = s.block(rho, b)
    P = R @ S
    lam = O.lambda_blocks(s, rho)
    for i in range(s.natoms):
        np.testing.assert_allclose(lam[i], P[off[i]:off[i + 1], off[i]:off[i + 1]], atol=1e-14)


def test_lno_eigen_properties(cfg1, lno_step):
    lno = lno_step[0]
    s_ii = {}
    for i in range(cfg1.natoms):
        b = next(b for b in range(cfg1.row_ptr[i], cfg1.row_ptr[i + 1])
                 if cfg1.col[b] == i and not np.any(cfg1.shift[b]))
        s_ii[i] = cfg1.block(cfg1.S, b)
    lam_blocks = O.lambda_blocks(cfg1, O.plain_dc_density(cfg1, cfg1.r_core)[2])
    for i, (V, ev, flags) in lno.items():
        # Table I: populations are dominated by the leading few, all below ~1
        assert ev.real.max() < 1.05 and ev.real.min() > -0.1
        np.testing.assert_allclose(V.T @ s_ii[i] @ V, np.eye(V.shape[1]), atol=1e-12)
        # the span is invariant under Lambda (exact for real selected eigenvalues)
        L = lam_blocks[i]
        P = V @ np.linalg.pinv(V)
        assert np.linalg.norm(L @ V - P @ L @ V) < 1e-10
        np.testing.assert_allclose(np.sort(ev.real)[::-1], ev.real)


def test_lnos_complex_pair_rule():
    """A selected complex pair contributes its real and imaginary parts; a split pair its real part."""
    A = np.array([[0.9, 0.0, 0.0], [0.0, 0.5, 0.3], [0.0, -0.3, 0.5]])
    s_ii = np.eye(3)
    V, ev, flags = O.lnos(A, s_ii, 3)
    assert flags & O.dclno_oracle.LNO_COMPLEX_SELECTED and not flags & O.dclno_oracle.LNO_PAIR_SPLIT
    V2, ev2, flags2 = O.lnos(A, s_ii, 2)
    assert flags2 & O.dclno_oracle.LNO_PAIR_SPLIT
    assert abs(ev[0] - 0.9) < 1e-14 and abs(ev[1] - (0.5 + 0.3j)) < 1e-14


def test_fermi_and_mu():
    f = O.fermi(np.array([0.0, 1000.0, -1000.0, 3.0, -3.0]))
    assert f[0] == 0.5 and f[1] == 0.0 and f[2] == 1.0
    assert abs(f[3] + f[4] - 1.0) <= 2.3e-16
    eps = np.array([-1.0, 0.2])
    mu, n = O.find_mu(eps, np.ones(2), 2.0, 0.05)
    assert abs(mu - (-0.4)) < 1e-12
    with pytest.raises(O.NoBracket):
        O.find_mu(eps, np.ones(2), 4.5, 0.05)


def test_worked_dimensions():
    with open(os.path.join(GOLD, "time_ratio.json")) as fh:
        g = json.load(fh)
    for c in g["cases"]:
        assert O.cluster_dim(c["n_short"], c["n_long"], c["m_pao"], c["m_lno"]) == c["dim"]
        if "ratio_2dp" in c:
            r = O.time_ratio(c["m_pao"], c["m_lno"], c["n_short"], c["n_long"])
            assert round(r, 2) == c["ratio_2dp"]


def test_mixed_basis_step(mixed_system):
    """Ragged basis (M = 3 and 4): the step runs and keeps its invariants."""
    s = mixed_system
    mu0, n0, rho0, e0, _ = O.plain_dc_density(s, s.r_core)
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    assert abs(n_mu - s.n_electrons) < 1e-9
    assert abs(2 * _pair_trace(s, rho, s.S) - n_mu) < 1e-9
    assert abs(2 * _pair_trace(s, rho, s.H) - e_band) < 1e-9 * abs(e_band)


def test_energy_density_matrix(cfg1, cfg1_exact, lno_step):
    """Eq. (edm): 2 Tr(e S) = E_band; for a cluster covering the whole open system
    e = S^-1 H rho exactly (H C = S C E), i.e. S e = H rho."""
    lno, V, res, mu, n_mu, rho, e_band = lno_step
    e = O.energy_density(cfg1, res, V, mu, cfg1.kT)
    assert abs(2 * _pair_trace(cfg1, e, cfg1.S) - e_band) < 1e-9 * abs(e_band)
    full = O.dclno_solve(cfg1, {}, 13.5, 13.5, 0)
    mu_f, n_f, rho_f, e_f = O.finish_step(cfg1, full, {}, cfg1.n_electrons, cfg1.kT)
    ed = O.energy_density(cfg1, full, {}, mu_f, cfg1.kT)
    H, S, off = O.dense_matrices(cfg1)

    def dense(x):
        D = np.zeros_like(S)
        brow = cfg1.block_rows()
        for b in range(cfg1.nnzb):
            i, j = int(brow[b]), int(cfg1.col[b])
            D[off[i]:off[i + 1], off[j]:off[j + 1]] = cfg1.block(x, b)
        return D

    np.testing.assert_allclose(S @ dense(ed), H @ dense(rho_f), rtol=0, atol=1e-9)


# ---------------------------------------------------------------------------
# Region rule of Sec. III (kappa buffer): worked example on a simple-cubic lattice
# ---------------------------------------------------------------------------
def test_kappa_region_rule_worked_example():
    """Periodic 8^3 SC lattice, spacing 1, one Gaussian (exponent 1) per atom, so the
    overlap of two atoms at distance d is exp(-d^2/2).  r_L = 2.5 holds the shells
    d^2 = 0, 1, 2, 3, 4, 5, 6 with 1, 6, 12, 8, 6, 24, 24 atoms (81).  With the
    first neighbours taken as overlaps above 0.3 (d^2 <= 2: e^-1 = 0.37 > 0.3 >
    e^-1.5 = 0.22): N_F = 19, N_S = 62, N_F + 3/10 N_S = 37.6.  Spheres hold
    1, 7, 19, 27, 33, 57, 81 atoms; the closest is 33 (d^2 <= 4), so the short-range
    region has 33 atoms and the long-range region 48."""
    import tbsystems as T
    s = T.small_lattice(8, 8, 8, a=1.0, exps=(1.0,), onsite=(0.0,), e_per_atom=1.0, r_core=1.0, r_lno=2.5,
                        k_lno=1, periodic=True)
    for i in (0, 137, 511):
        cl = O.cluster_members(s, i, 0.0, 2.5, 1, kappa=0.3, s_fna=0.3)
        assert len(cl.atoms) == 81
        assert int(np.count_nonzero(cl.core)) == 33
        assert np.max(cl.dist[cl.core]) == pytest.approx(2.0)
        assert np.min(cl.dist[~cl.core]) == pytest.approx(np.sqrt(5.0))
    # kappa = 0: the short-range region is the first neighbours (19); kappa = 1: all 81
    assert int(np.count_nonzero(O.cluster_members(s, 0, 0.0, 2.5, 1, kappa=0.0, s_fna=0.3).core)) == 19
    assert int(np.count_nonzero(O.cluster_members(s, 0, 0.0, 2.5, 1, kappa=1.0, s_fna=0.3).core)) == 81
    # the literal "non-zero overlap" (any stored block): every atom within r_L overlaps
    assert int(np.count_nonzero(O.cluster_members(s, 0, 0.0, 2.5, 1, kappa=0.3, s_fna=0.0).core)) == 81


def test_kappa_radius_ties_go_to_the_larger_sphere():
    # shells of 1, 3, 3 atoms; N_F = 1, N_S = 6, kappa = 0.5 -> target 4: spheres 1, 4, 7 -> 4;
    # kappa = 1/3 -> target 3: |1-3| = 2 > |4-3| = 1 -> 4; target 5.5 (kappa 0.75): |4-5.5| = |7-5.5| -> 7
    d = np.array([0.0, 1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    fna = np.array([True, False, False, False, False, False, False])
    assert O.kappa_radius(d, fna, 0.5) == 1.0
    assert O.kappa_radius(d, fna, 1.0 / 3.0) == 1.0
    assert O.kappa_radius(d, fna, 0.75) == 2.0


# ---------------------------------------------------------------------------
# Threshold selection of LNOs (Sec. II.B step (iii), lambda_th)
# ---------------------------------------------------------------------------
def test_lno_threshold_selects_eigenvalues_above_lambda_th():
    """Lambda = X diag(lam) X^-1 with known real eigenvalues: the threshold keeps
    exactly those >= lambda_th (capped at k), spanning their eigenvectors."""
    rng = np.random.default_rng(4)
    m = 6
    lam = np.array([0.95, 0.6, 0.12, 0.1 + 1e-7, 0.1 - 1e-7, -0.02])
    X = rng.normal(size=(m, m)) + 3 * np.eye(m)
    L = X @ np.diag(lam) @ np.linalg.inv(X)
    S = np.eye(m)
    V, ev, fl = O.lnos(L, S, 5, lambda_th=0.1)
    assert V.shape == (m, 4)  # 0.95, 0.6, 0.12 and 0.1 + 1e-7, not 0.1 - 1e-7
    P = X[:, :4] @ np.linalg.pinv(X[:, :4])  # projector on the selected eigenvectors
    np.testing.assert_allclose(P @ V, V, atol=1e-10)
    assert O.lnos(L, S, 2, lambda_th=0.1)[0].shape == (m, 2)      # capped at k
    assert O.lnos(L, S, 5, lambda_th=0.99)[0].shape == (m, 0)     # none qualifies
    np.testing.assert_allclose(O.lnos(L, S, 4)[0] @ O.lnos(L, S, 4)[0].T, V @ V.T, atol=1e-10)


def test_threshold_with_all_lnos_equals_plain_dc(cfg1):
    """lambda_th below every eigenvalue and k = M: every atom keeps its whole basis,
    the all-LNO identity again (Eq. (apop_Lambda) with every term kept)."""
    s = cfg1
    r = 6.0
    rho0 = O.plain_dc_density(s, s.r_core)[2]
    lno = O.compute_lnos(s, rho0, int(s.norb[0]), lambda_th=-1e9)
    V = {j: v[0] for j, v in lno.items()}
    kat = {j: v.shape[1] for j, v in V.items()}
    assert set(kat.values()) == {int(s.norb[0])}
    atoms = [0, 21, 63]
    res = O.dclno_solve(s, V, 3.0, r, 2, atoms=atoms, k_atoms=kat)
    ref = O.dclno_solve(s, V, r, r, 2, atoms=atoms)
    for i in atoms:
        np.testing.assert_allclose(res[i].eps, ref[i].eps, atol=1e-9)


def test_density_rows_equal_matsubara_pole_sum():
    """Eq. (dm) through the spectral form Eq. (Gi) equals the Green function summed
    over the Matsubara poles (Eq. (rho0j), non-orthogonal form) for every cluster of
    a small system with a narrow spectrum (two Gaussians per atom), the poles taken
    until w_P is 40 times the cluster's spectral radius about mu."""
    s = T.small_lattice(3, 3, 3, a=2.5, exps=(0.5, 1.5), onsite=(-0.4, 0.2), e_per_atom=2.0, r_core=3.0,
                        r_lno=6.0, k_lno=1)
    rho0 = O.plain_dc_density(s, s.r_core)[2]
    lno = O.compute_lnos(s, rho0, 1)
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, 1)
    mu = O.finish_step(s, res, V, s.n_electrons, s.kT)[0]
    a = np.zeros_like(s.S)
    b = np.zeros_like(s.S)
    assert any(not np.all(r.cluster.core) for r in res.values())  # LNO members take part
    for i, r in res.items():
        Hc, Sc = O.assemble(s, r.cluster, V)
        rad = float(np.max(np.abs(r.eps - mu)))
        n_poles = int(40.0 * rad / (2 * np.pi * s.kT)) + 1
        O.density_rows(s, r.cluster, r.eps, r.C, V, mu, s.kT, a)
        O.density_rows_poles(s, r.cluster, Hc, Sc, V, mu, s.kT, b, n_poles)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-11)


def test_periodic_invariants():
    """A periodic cell (several images of every pair stored): sum_mu q_mu = M_i,
    2 Tr(rho S) = N(mu) and 2 Tr(rho H) = E_band hold for a DC-LNO step, which
    needs each row block scattered to its own image (atom, cell shift)."""
    s = T.small_lattice(4, 4, 4, a=2.5, jitter=0.05, periodic=True, r_core=4.0, r_lno=6.0, k_lno=2)
    assert len(np.unique(s.shift, axis=0)) > 27  # pairs reach beyond the nearest images
    rho0 = O.plain_dc_density(s, s.r_core)[2]
    lno = O.compute_lnos(s, rho0, s.k_lno)
    V = {i: v[0] for i, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu, n_mu, rho, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    for i, r in res.items():
        assert abs(r.q.sum() - s.norb[i]) < 1e-10
    assert abs(n_mu - s.n_electrons) <= 1e-10 * s.n_electrons
    assert abs(2 * _pair_trace(s, rho, s.S) - n_mu) < 1e-9
    assert abs(2 * _pair_trace(s, rho, s.H) - e_band) < 1e-9 * abs(e_band)

