"""dclno_refine_eigenpairs (Ogita-Aishima sweeps with FP64 residuals) against the
oracle's sweep, and against eigenpairs known in closed form.

Pencils from tbsystems.known_pencils (cond(S) = 100, eigenvalues over [-2, 2]);
starts X = C (I + eps P) with seeded Gaussian P.  Dimensions 70 and 97 leave ragged
32 x 32 tiles; a batch holds several pencils; n = 1 is the degenerate case.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from paper_1809_05637_gb300 import refine_eigenpairs  # noqa: E402


def _starts(C, eps, seed):
    rng = np.random.default_rng(seed)
    n = C.shape[1]
    return np.stack([C[p] @ (np.eye(n) + eps * rng.standard_normal((n, n))) for p in range(C.shape[0])])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_one_sweep_matches_oracle():
    count, n = 3, 70
    H, S, C, w = T.known_pencils(count, n, seed=21)
    X0 = _starts(C, 1e-5, seed=22)
    dX = _dev(X0)
    lam = refine_eigenpairs(_dev(H), _dev(S), dX, nsweeps=1).cpu().numpy()
    Xg = dX.cpu().numpy()
    for p in range(count):
        Xo, lo = O.refine_eigenpairs(H[p], S[p], X0[p])
        # the same sweep up to the rounding order of the n-term products
        assert np.max(np.abs(Xg[p] - Xo)) <= 1e-12
        assert np.max(np.abs(lam[p] - lo)) <= 1e-12
        # and it squared the start's error
        assert np.max(np.abs(Xg[p] - C[p])) <= 50.0 * np.max(np.abs(X0[p] - C[p])) ** 2


def test_sweeps_reach_known_eigenpairs():
    count, n = 2, 97
    H, S, C, w = T.known_pencils(count, n, seed=31)
    X0 = _starts(C, 1e-4, seed=32)
    dH, dS, dX = _dev(H), _dev(S), _dev(X0)
    lam = refine_eigenpairs(dH, dS, dX, nsweeps=3).cpu().numpy()
    Xg = dX.cpu().numpy()
    for p in range(count):
        assert np.max(np.abs(lam[p] - w[p])) <= 1e-12
        assert np.max(np.abs(Xg[p] - C[p])) <= 1e-12
        assert np.max(np.abs(Xg[p].T @ S[p] @ Xg[p] - np.eye(n))) <= 1e-12
    # two calls in a row from the refined X: nothing left to correct
    lam2 = refine_eigenpairs(dH, dS, dX, nsweeps=1).cpu().numpy()
    assert np.max(np.abs(lam2 - w)) <= 1e-12
    assert np.max(np.abs(dX.cpu().numpy() - C)) <= 1e-12


def test_single_element_pencil_and_argument_errors():
    H = np.array([[[0.6]]])
    S = np.array([[[2.0]]])
    X = np.array([[[0.7]]])  # exact: 1 / sqrt(2) = 0.7071...
    dX = _dev(X)
    lam = refine_eigenpairs(_dev(H), _dev(S), dX, nsweeps=4).cpu().numpy()
    assert abs(lam[0, 0] - 0.3) <= 1e-15
    assert abs(dX.cpu().numpy()[0, 0, 0] - 2.0 ** -0.5) <= 1e-15
    d = _dev(np.zeros((1, 4, 4)))
    with pytest.raises(ValueError):
        refine_eigenpairs(d, d, _dev(np.zeros((1, 4, 5))))  # not square
    with pytest.raises(ValueError):
        refine_eigenpairs(d, d.float(), d)  # float32
    from paper_1809_05637_gb300 import DclnoError

    with pytest.raises(DclnoError):
        refine_eigenpairs(d, d, d, nsweeps=0)
