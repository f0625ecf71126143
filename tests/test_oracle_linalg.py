"""Pins of the oracle's own dense solvers against library routines on random inputs."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_jacobi_vs_eigh(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    A = A + A.T
    w, V = O.jacobi(A)
    ref = np.linalg.eigvalsh(A)
    sc = max(1.0, np.abs(ref).max())
    assert np.max(np.abs(w - ref)) < 1e-13 * sc * n
    assert np.max(np.abs(A @ V - V * w)) < 1e-13 * sc * n
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13 * n


def test_jacobi_degenerate():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    d = np.array([1.0] * 4 + [2.0] * 5 + [-3.0] * 3)
    A = (Q * d) @ Q.T
    w, V = O.jacobi(A)
    np.testing.assert_allclose(w, np.sort(d), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(12), atol=1e-13)


def test_cholesky():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(30, 30))
    S = X @ X.T + 1e-3 * np.eye(30)
    L = O.cholesky(S)
    np.testing.assert_allclose(L, np.linalg.cholesky(S), rtol=1e-10, atol=1e-12)
    with pytest.raises(O.NotSPD):
        O.cholesky(np.diag([1.0, -1.0, 2.0]))


@pytest.mark.parametrize("n", [8, 33, 64])
def test_gen_eig_vs_scipy(n):
    rng = np.random.default_rng(10 + n)
    X = rng.normal(size=(n, n))
    S = X @ X.T + 0.5 * np.eye(n)
    H = rng.normal(size=(n, n))
    H = H + H.T
    eps, C = O.gen_eig(H, S)
    ref = sl.eigh(H, S, eigvals_only=True)
    sc = np.abs(ref).max()
    assert np.max(np.abs(eps - ref)) < 1e-12 * sc
    np.testing.assert_allclose(C.T @ S @ C, np.eye(n), atol=1e-11)
    np.testing.assert_allclose(H @ C, S @ C * eps, atol=1e-10 * sc)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6, 9, 13])
def test_nonsym_eig_vs_numpy(m):
    rng = np.random.default_rng(100 + m)
    for trial in range(5):
        A = rng.normal(size=(m, m))
        if trial == 1:
            A = np.triu(A)
        if trial == 2 and m > 1:  # rotation-like blocks: complex pairs
            A = A - A.T + 0.1 * np.eye(m)
        wr, wi = O.nonsym_eig(A)
        got = wr + 1j * wi
        ref = np.linalg.eigvals(A)
        # match as multisets: every reference eigenvalue has a distinct close partner
        free = list(range(m))
        for r in ref:
            k = min(free, key=lambda t: abs(got[t] - r))
            assert abs(got[k] - r) < 1e-11 * max(1.0, np.abs(ref).max())
            free.remove(k)


@pytest.mark.parametrize("gap", [5e-9, 1e-11, 0.0])
def test_nonsym_eig_close_real_pair(gap):
    """Eigenvalues closer than sqrt(u) are still resolved: A = X D X^-1 with a
    well-conditioned X (so each eigenvalue is determined to about u |A| cond(X)) and
    D = diag(0.9, 0.5 + gap, 0.5, 0.1).  A discriminant formed as tr^2 - det would
    merge the close pair into its mean."""
    rng = np.random.default_rng(3)
    X = np.eye(4) + 0.3 * rng.standard_normal((4, 4))
    d = np.array([0.9, 0.5 + gap, 0.5, 0.1])
    A = X @ np.diag(d) @ np.linalg.inv(X)
    wr, wi = O.nonsym_eig(A)
    assert np.all(np.abs(wi) <= 1e-7)  # a close pair may come out complex only at the level of sqrt(u) |A|
    got = np.sort(wr)[::-1]
    np.testing.assert_allclose(got, d, rtol=0, atol=1e-13 if gap > 0 else 1e-7)


def test_inverse_iteration():
    rng = np.random.default_rng(7)
    A = rng.normal(size=(9, 9))
    ev = np.linalg.eigvals(A)
    for lam in ev:
        x = O.inverse_iter(A, lam.real, lam.imag)
        assert abs(np.linalg.norm(x) - 1) < 1e-12
        assert np.linalg.norm(A @ x - lam * x) < 1e-10
