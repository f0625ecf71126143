"""Pins of the oracle's symmetric LNO mode: G v = lambda S_ii v with G the on-site
block of the occupied-space projector, (S rho S)_ii (the symmetric counterpart of
the paper's Lambda_0i = (rho S)_ii of Eq. (Lambda)).

* G against the dense product S rho S of an open system, and of a periodic
  system whose cell is more than three neighbour radii wide (there the image sum
  of every block folds into one dense entry without aliasing);
* rho = S^-1 (every state occupied, exact on a fully connected open system):
  S rho S = S, so every eigenvalue is 1;
* the exact finite-temperature density matrix: 0 <= S rho S <= S as quadratic
  forms, so every eigenvalue lies in [0, 1];
* the eigen step against the library's generalized symmetric eigensolver;
* keeping all M_i LNOs reproduces plain-PAO DC, as in the paper's mode.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
import tbsystems as T


def _dense(s, vals):
    """Open system: BSR values -> dense matrix (each block at its (i, j) place)."""
    off = np.concatenate([[0], np.cumsum(s.norb)])
    D = np.zeros((off[-1], off[-1]))
    brow = s.block_rows()
    for b in range(s.nnzb):
        i, j = int(brow[b]), int(s.col[b])
        D[off[i]:off[i + 1], off[j]:off[j + 1]] += s.block(vals, b)
    return D, off


def _from_dense(s, D, off):
    out = np.zeros_like(s.S)
    brow = s.block_rows()
    for b in range(s.nnzb):
        i, j = int(brow[b]), int(s.col[b])
        mi, mj = int(s.norb[i]), int(s.norb[j])
        o = int(s.blk_off[b])
        out[o:o + mi * mj] = D[off[i]:off[i + 1], off[j]:off[j + 1]].reshape(-1)
    return out


def _s_ii(s, i):
    b = next(b for b in range(s.row_ptr[i], s.row_ptr[i + 1]) if s.col[b] == i and not np.any(s.shift[b]))
    return s.block(s.S, b)


@pytest.fixture(scope="module")
def periodic_small():
    """512 atoms on a jittered simple-cubic lattice (2.4 bohr), periodic cube of
    19.2 bohr; two s-Gaussians (1.5, 3.5) per atom keep the overlap pattern
    within 5.6 bohr, less than a third of the cell."""
    pos, _ = T._sc_lattice(8, 8, 8, 2.4)
    pos = pos + np.random.default_rng(3).normal(0, 0.05, pos.shape)
    n = len(pos)
    return T.assemble_system("periodic512", pos, np.eye(3) * 19.2, np.ones(3, bool), np.zeros(n, np.int32),
                             [np.array([1.5, 3.5])] * n, [np.array([-0.4, 0.3])] * n, float(n), 0.02,
                             3.0, 5.0, 1)


@pytest.mark.parametrize("which", ["cfg1", "mixed"])
def test_projector_matches_dense_product(which, cfg1, mixed_system):
    s = cfg1 if which == "cfg1" else mixed_system
    rho = T.synthetic_density(s, seed=4)
    S, off = _dense(s, s.S)
    R, _ = _dense(s, rho)
    P = S @ R @ S
    G = O.projector_blocks(s, rho)
    for i in range(s.natoms):
        np.testing.assert_allclose(G[i], P[off[i]:off[i + 1], off[i]:off[i + 1]], rtol=0, atol=1e-13)


def test_projector_periodic_fold(periodic_small):
    s = periodic_small
    brow = s.block_rows()
    d = np.linalg.norm(s.pos[s.col] + s.shift @ s.cell - s.pos[brow], axis=1)
    assert 3 * d.max() < s.cell[0, 0]
    rho = T.synthetic_density(s, seed=8)
    S, off = _dense(s, s.S)  # image sum: every (i, j) pair has one stored shift at most
    R, _ = _dense(s, rho)
    atoms = [0, 77, 300, 511]
    G = O.projector_blocks(s, rho, atoms=atoms)
    for i in atoms:
        rows = slice(off[i], off[i + 1])
        np.testing.assert_allclose(G[i], S[rows] @ R @ S[:, rows], rtol=0, atol=1e-13)


def test_full_occupation_gives_unit_eigenvalues(cfg1):
    s = cfg1
    assert np.diff(s.row_ptr).min() == s.natoms  # fully connected: S^-1 fits the pattern
    S, off = _dense(s, s.S)
    rho = _from_dense(s, np.linalg.inv(S), off)
    lno = O.compute_lnos(s, rho, 4, mode="sym")
    for i, (V, ev, flags) in lno.items():
        np.testing.assert_allclose(ev.real, 1.0, rtol=0, atol=1e-8)
        np.testing.assert_allclose(V.T @ _s_ii(s, i) @ V, np.eye(4), rtol=0, atol=1e-12)


def test_exact_density_eigenvalues_in_unit_interval(cfg1, cfg1_exact):
    s = cfg1
    rho = cfg1_exact[4]
    lno = O.compute_lnos(s, rho, s.k_lno, mode="sym")
    ev = np.concatenate([v[1].real for v in lno.values()])
    assert ev.min() > -1e-10 and ev.max() < 1 + 1e-10
    # occupied states exist near every atom: the leading eigenvalue is a real population
    assert min(v[1].real[0] for v in lno.values()) > 0.5


def test_eigen_step_matches_generalized_eigh():
    rng = np.random.default_rng(12)
    for m, k in [(4, 2), (9, 4), (13, 3)]:
        X = rng.normal(size=(m, m))
        s_ii = X @ X.T + m * np.eye(m)
        Y = rng.normal(size=(m, m))
        G = Y @ Y.T
        Gn = G + 0.3 * (Y - Y.T)  # antisymmetric part: must not matter
        V, ev, flags = O.lnos_sym(Gn, s_ii, k)
        w, C = sl.eigh(G, s_ii)
        np.testing.assert_allclose(ev.real, w[::-1], rtol=1e-12, atol=1e-12 * np.abs(w).max())
        assert not np.any(ev.imag) and flags == 0
        Ck = C[:, ::-1][:, :k]
        np.testing.assert_allclose(V @ V.T, Ck @ Ck.T, rtol=0, atol=1e-10)
        np.testing.assert_allclose(V.T @ s_ii @ V, np.eye(k), rtol=0, atol=1e-12)
        # threshold selection: eigenvalues >= lambda_th only, at most k
        th = 0.5 * (w[-2] + w[-3])
        Vt, _, _ = O.lnos_sym(G, s_ii, k, lambda_th=th)
        assert Vt.shape[1] == 2


def test_sym_all_lno_identity(cfg1, cfg1_dc0):
    """k = M_i: the LNO block spans the whole atom, whatever the mode."""
    rho0 = cfg1_dc0[2]
    lno = O.compute_lnos(cfg1, rho0, 4, mode="sym")
    V = {i: v[0] for i, v in lno.items()}
    a = O.dclno_solve(cfg1, V, 5.0, 8.0, 4)
    b = O.dclno_solve(cfg1, {}, 8.0, 8.0, 0)
    for i in a:
        assert np.all(np.abs(a[i].eps - b[i].eps) <= 1e-10 + 1e-12 * np.abs(b[i].eps))
        np.testing.assert_allclose(a[i].q, b[i].q, atol=1e-9)


def test_unknown_mode_is_refused(cfg1):
    with pytest.raises(ValueError):
        O.compute_lnos(cfg1, np.zeros_like(cfg1.S), 2, atoms=[0], mode="hermitian")
