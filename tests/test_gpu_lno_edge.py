"""The edge cases of the LNO eigenproblem on the GPU (Sec. II.B, Eq. (eigendecomp)):
Lambda_0i is nonsymmetric, so its leading eigenvalues can be a complex pair, the
cut at k can fall between the two members of a pair, and two eigenvalues can
nearly tie at the cut.

The input density is the plain-DC density of the 64-atom lattice with the on-site
blocks of a few atoms changed so that their Lambda blocks have a chosen
spectrum: Lambda_0i gains Delta S_ii when rho_ii gains Delta (Eq. (Lambda)), so
rho_ii += (Lambda_target - Lambda_0i) S_ii^-1 gives Lambda_0i = Lambda_target =
X D X^-1 with a real block-diagonal D (a 2 x 2 block [[a, b], [-b, a]] is the
pair a +- i b).  Compared with the oracle: flags, eigenvalues, the span of the
kept vectors (projector in the S_ii metric) and, for the complex cases, every
cluster's spectrum and the density rows.  For the near tie only what is unique
is compared: the eigenvalues, and that the kept span holds the leading
eigenvector and lies in the well-separated invariant subspace of the top three.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from oracle.dclno_oracle import LNO_COMPLEX_SELECTED, LNO_PAIR_SPLIT  # noqa: E402
from gpu_helpers import gpu_context, spectral_moments, state_tol, to_dev  # noqa: E402

PAIR_ATOM, SPLIT_ATOM, TIE_ATOM = 0, 21, 42
TIE_GAP = 5e-9


def _target(D, seed):
    rng = np.random.default_rng(seed)
    X = np.eye(D.shape[0]) + 0.3 * rng.standard_normal(D.shape)
    return X @ D @ np.linalg.inv(X), X


def _pair(a, b):
    return np.array([[a, b], [-b, a]])


def _block_diag(*blocks):
    m = sum(b.shape[0] for b in blocks)
    out = np.zeros((m, m))
    o = 0
    for b in blocks:
        out[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return out


def _with_lambda(s, rho, targets):
    """rho with the on-site blocks of the given atoms changed so that Lambda_0i of
    each equals its target."""
    rho = rho.copy()
    lam = O.lambda_blocks(s, rho, atoms=sorted(targets))
    for i, T in targets.items():
        m = int(s.norb[i])
        b = next(b for b in range(int(s.row_ptr[i]), int(s.row_ptr[i + 1]))
                 if int(s.col[b]) == i and not np.any(s.shift[b]))
        o = int(s.blk_off[b])
        Sii = s.S[o:o + m * m].reshape(m, m)
        rho[o:o + m * m] += ((T - lam[i]) @ np.linalg.inv(Sii)).reshape(-1)
    return rho


def _s_projector(V, Sii):
    """Projector onto span(V) orthogonal in the S_ii metric (V S_ii-orthonormal)."""
    return V @ V.T @ Sii


def _onsite(s, i):
    m = int(s.norb[i])
    b = next(b for b in range(int(s.row_ptr[i]), int(s.row_ptr[i + 1]))
             if int(s.col[b]) == i and not np.any(s.shift[b]))
    o = int(s.blk_off[b])
    return s.S[o:o + m * m].reshape(m, m)


@pytest.fixture(scope="module")
def targets():
    pair, Xp = _target(_block_diag(_pair(0.9, 0.05), np.diag([0.3, 0.1])), 1)
    split, Xs = _target(_block_diag(np.diag([0.95]), _pair(0.6, 0.04), np.diag([0.05])), 2)
    tie, Xt = _target(np.diag([0.9, 0.5 + TIE_GAP, 0.5, 0.1]), 3)
    return dict(pair=(pair, Xp), split=(split, Xs), tie=(tie, Xt))


def test_complex_pair_and_split_pair(cfg1, cfg1_dc0, targets):
    s = cfg1
    assert s.k_lno == 2 and np.all(s.norb == 4)
    rho = _with_lambda(s, cfg1_dc0[2], {PAIR_ATOM: targets["pair"][0], SPLIT_ATOM: targets["split"][0]})
    lno = O.compute_lnos(s, rho, s.k_lno)
    assert lno[PAIR_ATOM][2] == LNO_COMPLEX_SELECTED
    assert lno[SPLIT_ATOM][2] == LNO_COMPLEX_SELECTED | LNO_PAIR_SPLIT
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.compute_lnos(to_dev(rho))
    glno = ctx.lnos()
    for j in range(s.natoms):
        Vo, evo, flo = lno[j]
        Vg, evg, flg = glno[j]
        assert flg == flo, f"atom {j}: flags {flg} != {flo}"
        np.testing.assert_allclose(evg, evo, rtol=0, atol=1e-10, err_msg=f"atom {j}: eigenvalues")
        Sii = _onsite(s, j)
        np.testing.assert_allclose(_s_projector(Vg, Sii), _s_projector(Vo, Sii), rtol=0, atol=1e-9,
                                   err_msg=f"atom {j}: span")
    # the designed spectra were found: a selected pair, and a pair split by the cut
    np.testing.assert_allclose(glno[PAIR_ATOM][1][:2], [0.9 + 0.05j, 0.9 - 0.05j], atol=1e-12)
    np.testing.assert_allclose(glno[SPLIT_ATOM][1][:3], [0.95, 0.6 + 0.04j, 0.6 - 0.04j], atol=1e-12)
    # every cluster with these LNOs against the oracle
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    users = [i for i, r in res.items()
             if any((not c) and int(a) in (PAIR_ATOM, SPLIT_ATOM) for a, c in zip(r.cluster.atoms, r.cluster.core))]
    assert len(users) >= 8
    mu, n_mu, rho_out, e_band = O.finish_step(s, res, V, s.n_electrons, s.kT)
    ctx.solve_clusters()
    spec = ctx.spectrum()
    mus = np.linspace(-1.2, 0.0, 13)
    for i, r in res.items():
        e_gpu, q_gpu = spec[i]
        assert np.all(np.abs(np.sort(e_gpu) - r.eps) <= state_tol(r)), f"cluster {i}"
        np.testing.assert_allclose(spectral_moments(e_gpu, q_gpu, mus, s.kT),
                                   spectral_moments(r.eps, r.q, mus, s.kT), rtol=0, atol=1e-9)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    e = ctx.density_matrix(mu, s.kT, out)
    np.testing.assert_allclose(out.cpu().numpy(), rho_out, rtol=0, atol=1e-9)
    assert abs(e - e_band) <= 1e-9 * abs(e_band)
    ctx.close()


def test_near_tie_at_the_cut(cfg1, cfg1_dc0, targets):
    s = cfg1
    tie, X = targets["tie"]
    rho = _with_lambda(s, cfg1_dc0[2], {TIE_ATOM: tie})
    Vo, evo, flo = O.compute_lnos(s, rho, s.k_lno, atoms=[TIE_ATOM])[TIE_ATOM]
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.compute_lnos(to_dev(rho))
    Vg, evg, flg = ctx.lnos()[TIE_ATOM]
    ctx.close()
    assert flg == flo == 0
    np.testing.assert_allclose(evg, evo, rtol=0, atol=1e-10)
    assert abs(evg[1].real - evg[2].real - TIE_GAP) < 1e-10  # the tie sits at the cut k = 2
    Sii = _onsite(s, TIE_ATOM)
    # an S_ii-orthonormal basis of the top-three invariant subspace span{X_0, X_1, X_2}
    U = X[:, :3]
    U = U @ np.linalg.inv(np.linalg.cholesky(U.T @ Sii @ U).T)
    x0 = X[:, 0] / np.linalg.norm(X[:, 0])
    for V in (Vg, Vo):
        np.testing.assert_allclose(V.T @ Sii @ V, np.eye(2), rtol=0, atol=1e-12)
        np.testing.assert_allclose(_s_projector(U, Sii) @ V, V, rtol=0, atol=1e-9)  # inside the top three
        np.testing.assert_allclose(_s_projector(V, Sii) @ x0, x0, rtol=0, atol=1e-9)  # holds the leading vector
