"""Oracle: Ogita-Aishima refinement of a generalised eigendecomposition
(``oracle.refine_eigenpairs``), the refinement the mixed-precision path would need
if it started from FP32 eigenpairs.

Pinned to a pencil whose eigenpairs are known in closed form (built from them), where
each sweep must square the error; and measured on the 64-atom lattice's pencil, whose
degenerate spectrum puts FP32 eigenpairs outside the region where the refinement
converges (the reason the mixed path emulates FP64 contractions instead).
"""
import numpy as np
import pytest

import oracle as O
import tbsystems as T

scipy_linalg = pytest.importorskip("scipy.linalg")


def _pencil(n, seed):
    """One pencil with known eigenpairs (tbsystems.known_pencils: cond(S) = 100,
    eigenvalues over [-2, 2] at least half their spacing apart)."""
    H, S, C, w = T.known_pencils(1, n, seed=seed)
    return H[0], S[0], w[0], C[0]


def test_refinement_squares_the_error():
    n = 40
    H, S, w, C = _pencil(n, seed=5)
    rng = np.random.default_rng(6)
    eps0 = 1e-5
    X = C @ (np.eye(n) + eps0 * rng.standard_normal((n, n)))
    errs = [np.max(np.abs(X - C))]
    for _ in range(3):
        X, lam = O.refine_eigenpairs(H, S, X)
        errs.append(np.max(np.abs(X - C)))
    # quadratic convergence (2.5e-5 -> 1e-8 -> rounding); a dropped or mis-signed term
    # of E leaves a first-order error behind
    assert errs[1] <= 50.0 * errs[0] ** 2
    assert errs[2] <= 1e-12
    assert errs[3] <= 1e-12
    # eigenvalues from the last sweep's input, S-orthonormality of the result
    assert np.max(np.abs(lam - w)) <= 1e-13
    assert np.max(np.abs(X.T @ S @ X - np.eye(n))) <= 1e-13
    # the same refinement reached from a start with shuffled-sign columns keeps the signs
    Xs, _ = O.refine_eigenpairs(H, S, C * np.where(np.arange(n) % 2 == 0, 1.0, -1.0))
    assert np.max(np.abs(Xs - C * np.where(np.arange(n) % 2 == 0, 1.0, -1.0))) <= 1e-12


def test_refinement_of_exact_pairs_is_exact():
    """From the exact eigenvectors R = 0 and G = diag(w): the sweep changes nothing."""
    H, S, w, C = _pencil(24, seed=9)
    X, lam = O.refine_eigenpairs(H, S, C)
    assert np.max(np.abs(lam - w)) <= 1e-13
    assert np.max(np.abs(X - C)) <= 1e-13


def test_fp32_start_outside_convergence_region_on_lattice_pencil():
    """The 64-atom lattice (the small workload, 256 x 256 pencil, cond(S) ~ 1e4):
    its spectrum has exactly degenerate levels (lattice symmetry), FP32 eigenvalues are
    off by far more than the smallest gaps, and refinement sweeps from the FP32
    eigenvectors stall well above FP64 accuracy."""
    s = T.make_system(1)
    H, S, _ = O.dense_matrices(s)
    w = scipy_linalg.eigh(H, S, eigvals_only=True)
    w32, V32 = scipy_linalg.eigh(H.astype(np.float32), S.astype(np.float32))
    gaps = np.diff(w)
    assert np.max(np.abs(w32 - w)) > 100.0 * np.min(gaps)
    X = V32.astype(np.float64)
    for _ in range(5):
        X, lam = O.refine_eigenpairs(H, S, X)
    assert np.max(np.abs(lam - w)) > 1e-8
