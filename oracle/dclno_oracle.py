"""DC-LNO oracle (FP64, CPU).  TEST INFRASTRUCTURE ONLY -- see oracle/__init__.py.

Every function states the passage of the paper it follows.  Heavy numerics
(Cholesky, Jacobi, nonsymmetric QR, inverse iteration) are the oracle's own C
code in csrc/oracle_linalg.c; numpy is used for array bookkeeping and for
plain matrix products.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

__all__ = [
    "cholesky", "jacobi", "gen_eig", "nonsym_eig", "inverse_iter",
    "Cluster", "cluster_members", "kappa_radius", "lambda_blocks", "projector_blocks", "lnos", "lnos_sym",
    "compute_lnos",
    "assemble", "solve_cluster", "fermi", "n_of_mu", "find_mu", "density_rows",
    "dclno_solve", "finish_step", "energy_density", "density_rows_poles", "plain_dc_density", "full_diag", "dense_matrices",
    "cluster_dim", "time_ratio", "refine_eigenpairs", "NoBracket", "NotSPD",
]

# --------------------------------------------------------------------------
# C numerics
# --------------------------------------------------------------------------
_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.orc_cholesky.argtypes = [ctypes.c_int, _dp]
        lib.orc_jacobi.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int]
        lib.orc_gen_eig.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.orc_nonsym_eig.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        lib.orc_inverse_iter.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
        for f in (lib.orc_cholesky, lib.orc_jacobi, lib.orc_gen_eig, lib.orc_nonsym_eig,
                  lib.orc_inverse_iter):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class NotSPD(RuntimeError):
    pass


class NoBracket(RuntimeError):
    pass


def cholesky(S: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor L, S = L L^T."""
    L = np.ascontiguousarray(S, dtype=np.float64).copy()
    rc = _lib().orc_cholesky(L.shape[0], _p(L))
    if rc:
        raise NotSPD(f"Cholesky failed at pivot {rc - 1}")
    return L


def jacobi(A: np.ndarray, max_sweeps: int = 60):
    """Eigenvalues (ascending) and eigenvectors of a symmetric matrix (cyclic Jacobi)."""
    n = A.shape[0]
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    w = np.empty(n)
    V = np.empty((n, n))
    rc = _lib().orc_jacobi(n, _p(a), _p(w), _p(V), max_sweeps)
    if rc:
        raise RuntimeError("Jacobi did not converge")
    return w, V


def gen_eig(H: np.ndarray, S: np.ndarray):
    """H C = S C diag(eps), C^T S C = I (Cholesky + congruence + Jacobi)."""
    n = H.shape[0]
    h = np.ascontiguousarray(H, dtype=np.float64)
    s = np.ascontiguousarray(S, dtype=np.float64)
    eps = np.empty(n)
    C = np.empty((n, n))
    rc = _lib().orc_gen_eig(n, _p(h), _p(s), _p(eps), _p(C))
    if rc > 0:
        raise NotSPD(f"cluster overlap not positive definite (pivot {rc - 1})")
    if rc < 0:
        raise RuntimeError("generalised eigensolver did not converge")
    return eps, C


def nonsym_eig(A: np.ndarray):
    """Eigenvalues (wr, wi) of a small nonsymmetric matrix (Hessenberg + Francis QR)."""
    m = A.shape[0]
    a = np.ascontiguousarray(A, dtype=np.float64)
    wr = np.empty(m)
    wi = np.empty(m)
    rc = _lib().orc_nonsym_eig(m, _p(a), _p(wr), _p(wi))
    if rc:
        raise RuntimeError("nonsymmetric QR did not converge")
    return wr, wi


def inverse_iter(A: np.ndarray, lr: float, li: float = 0.0) -> np.ndarray:
    """Eigenvector of A for eigenvalue lr + i li (complex, unit 2-norm)."""
    m = A.shape[0]
    a = np.ascontiguousarray(A, dtype=np.float64)
    xr = np.empty(m)
    xi = np.empty(m)
    _lib().orc_inverse_iter(m, _p(a), float(lr), float(li), _p(xr), _p(xi))
    return xr + 1j * xi


# --------------------------------------------------------------------------
# Truncated clusters (Fig. 1; Eq. (Hi); regions by fixed radii)
# --------------------------------------------------------------------------
MEMBER_TOL = 1e-9  # bohr: an atom at distance d belongs to a region of radius r iff d <= r + tol


@dataclasses.dataclass
class Cluster:
    centre: int
    atoms: np.ndarray    # (K,) member atom index j
    shifts: np.ndarray   # (K, 3) member cell shift R
    core: np.ndarray     # (K,) True = PAO (short-range) member, False = LNO member
    dist: np.ndarray     # (K,)
    offsets: np.ndarray  # (K+1,) orbital offset of each member in the cluster basis

    @property
    def dim(self) -> int:
        return int(self.offsets[-1])

    @property
    def centre_slice(self) -> slice:
        return slice(int(self.offsets[-2]), int(self.offsets[-1]))


def _shift_range(system, rmax):
    rng = []
    for d in range(3):
        if not system.pbc[d]:
            rng.append(np.array([0]))
            continue
        e, f = [x for x in range(3) if x != d]
        cr = np.cross(system.cell[e], system.cell[f])
        height = abs(np.dot(system.cell[d], cr)) / np.linalg.norm(cr)
        nmax = int(math.ceil(rmax / height)) + 1
        rng.append(np.arange(-nmax, nmax + 1))
    return np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)


def kappa_radius(dist, fna, kappa):
    """Short-range radius of the region rule of Sec. III, steps (ii)-(iii).

    dist: distances of all images within r_L (the centre included); fna: True
    for first neighbouring atoms (non-zero overlap with the centre, the centre
    itself included), False for second neighbouring atoms.  The radius is the
    shell distance whose sphere holds a number of atoms closest to
    N_F + kappa N_S (ties: the larger sphere).
    """
    n_f = int(np.count_nonzero(fna))
    n_s = len(fna) - n_f
    target = n_f + kappa * n_s
    best_r, best_gap, best_cnt = 0.0, math.inf, -1
    for r in np.unique(dist):
        cnt = int(np.count_nonzero(dist <= r + MEMBER_TOL))
        gap = abs(cnt - target)
        if gap < best_gap - 1e-12 or (abs(gap - best_gap) <= 1e-12 and cnt > best_cnt):
            best_r, best_gap, best_cnt = float(r), gap, cnt
    return best_r


def _overlaps_centre(system, i, atoms, shifts, s_fna):
    """Members whose stored S block with the centre has max |S| > s_fna."""
    bidx = _BlockIndex(system)
    out = np.zeros(len(atoms), dtype=bool)
    mi = int(system.norb[i])
    for m, (j, sh) in enumerate(zip(atoms, shifts)):
        b = bidx.get(i, j, sh)
        if b is None:
            continue
        mj = int(system.norb[j])
        o = int(system.blk_off[b])
        out[m] = float(np.max(np.abs(system.S[o:o + mi * mj]))) > s_fna
    return out


def cluster_members(system, i: int, r_core: float, r_lno: float, k_lno: int, kappa: float | None = None,
                    s_fna: float = 0.0, k_atoms=None) -> Cluster:
    """Members of the truncated cluster of atom i.

    Core (PAO) region: images (j, R) with |tau_j + R - tau_i| <= r_core;
    LNO region: r_core < d <= r_lno (membership tolerance MEMBER_TOL).
    With kappa given, r_core is replaced by the radius of the region rule of
    Sec. III (kappa_radius), first neighbouring atoms being those whose stored
    overlap block with the centre exceeds s_fna in magnitude.
    Member order: distance descending, ties by (j, R), so the central atom
    is last.  Core members contribute M_j basis functions, LNO members k_lno,
    or k_atoms[j] when the LNO count differs per atom (threshold selection).
    """
    shifts = _shift_range(system, r_lno)
    img = (system.pos[None, :, :] + (shifts @ system.cell)[:, None, :])  # (nS, N, 3)
    dvec = img - system.pos[i][None, None, :]
    d = np.sqrt(np.einsum("snd,snd->sn", dvec, dvec))
    s_idx, j_idx = np.nonzero(d <= r_lno + MEMBER_TOL)
    dist = d[s_idx, j_idx]
    sh = shifts[s_idx]
    order = np.lexsort((sh[:, 2], sh[:, 1], sh[:, 0], j_idx, -dist))
    # lexsort sorts ascending by the last key first: -dist ascending = dist descending
    atoms = j_idx[order].astype(np.int64)
    sh = sh[order].astype(np.int64)
    dist = dist[order]
    if kappa is not None:
        r_core = kappa_radius(dist, _overlaps_centre(system, i, atoms, sh, s_fna), kappa)
    core = dist <= r_core + MEMBER_TOL
    # the central atom itself (d = 0) must be the last member
    assert atoms[-1] == i and not np.any(sh[-1]), "central atom is not last"
    klno = np.full(len(atoms), k_lno) if k_atoms is None else np.array([int(k_atoms[int(j)]) for j in atoms])
    sizes = np.where(core, system.norb[atoms], klno).astype(np.int64)
    offsets = np.zeros(len(atoms) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return Cluster(i, atoms, sh, core, dist, offsets)


class _BlockIndex:
    """(row atom, col atom, shift) -> BSR block number, built per row on demand."""

    def __init__(self, system):
        self.s = system
        self.rows: dict = {}

    def row(self, i):
        r = self.rows.get(i)
        if r is None:
            s = self.s
            b0, b1 = int(s.row_ptr[i]), int(s.row_ptr[i + 1])
            r = {(int(s.col[b]),) + tuple(int(x) for x in s.shift[b]): b for b in range(b0, b1)}
            self.rows[i] = r
        return r

    def get(self, i, j, shift):
        return self.row(int(i)).get((int(j),) + tuple(int(x) for x in shift))


# --------------------------------------------------------------------------
# LNOs: Eq. (Lambda), Eq. (eigendecomp), Eq. (apop_Lambda)
# --------------------------------------------------------------------------

def lambda_blocks(system, rho: np.ndarray, atoms=None) -> dict:
    """Lambda_0i = sum_{Rj} rho_{0i,Rj} S_{Rj,0i} (Eq. (Lambda)), M_i x M_i.

    S_{Rj,0i} = (S_{0i,Rj})^T because S is symmetric, so each stored block b
    of row i contributes rho_b @ S_b^T.
    """
    if atoms is None:
        atoms = range(system.natoms)
    out = {}
    for i in atoms:
        mi = int(system.norb[i])
        lam = np.zeros((mi, mi))
        for b in range(int(system.row_ptr[i]), int(system.row_ptr[i + 1])):
            mj = int(system.norb[system.col[b]])
            o = int(system.blk_off[b])
            rb = rho[o:o + mi * mj].reshape(mi, mj)
            sb = system.S[o:o + mi * mj].reshape(mi, mj)
            lam += rb @ sb.T
        out[int(i)] = lam
    return out


def _on_site_block(system, i):
    for b in range(int(system.row_ptr[i]), int(system.row_ptr[i + 1])):
        if int(system.col[b]) == i and not np.any(system.shift[b]):
            mi = int(system.norb[i])
            o = int(system.blk_off[b])
            return system.S[o:o + mi * mi].reshape(mi, mi)
    raise KeyError(f"no on-site block for atom {i}")


LNO_COMPLEX_SELECTED = 1   # a selected eigenvalue is complex
LNO_PAIR_SPLIT = 2         # a complex pair straddles the cut; its real part was kept


def lnos(lam: np.ndarray, s_ii: np.ndarray, k: int, lambda_th: float | None = None):
    """LNOs of one atom from its Lambda block.

    With lambda_th given (Sec. II.B step (iii)), only eigenvalues whose real part
    is at least lambda_th are selected, at most k of them (a conjugate pair has one
    real part, so both members qualify together).

    Eigenvalues by Hessenberg + Francis QR, sorted by real part descending
    (ties: positive imaginary part first).  The eigenvectors of the leading k
    eigenvalues (Eq. (apop_Lambda) with a fixed count instead of a threshold)
    come from inverse iteration.  For a selected complex pair the real and
    imaginary parts span its real invariant subspace; if only one member of a
    pair is selected, the real part alone is kept (flag LNO_PAIR_SPLIT).

    The span is what the method fixes (cluster results are invariant under a
    change of basis inside each atom's LNO block), so the vectors are
    returned in a canonical basis of that span: S_ii-orthonormalised by
    Gram-Schmidt in the order of the eigenvalues, each with its
    largest-magnitude component positive.

    Returns (V (M x k), eigenvalues (complex, sorted), flags).
    """
    m = lam.shape[0]
    wr, wi = nonsym_eig(lam)
    order = sorted(range(m), key=lambda t: (-wr[t], -wi[t]))
    ev = np.array([wr[t] + 1j * wi[t] for t in order])
    vecs = []
    flags = 0
    pos = 0
    while len(vecs) < k and pos < m:
        t = order[pos]
        if lambda_th is not None and wr[t] < lambda_th:
            break
        if wi[t] == 0.0:
            vecs.append(inverse_iter(lam, wr[t], 0.0).real)
            pos += 1
            continue
        flags |= LNO_COMPLEX_SELECTED
        x = inverse_iter(lam, wr[t], wi[t])
        vecs.append(x.real)
        if len(vecs) < k:
            vecs.append(x.imag)
        else:
            flags |= LNO_PAIR_SPLIT
        pos += 2  # skip the conjugate partner
    V = np.column_stack(vecs[:k]) if vecs else np.zeros((m, 0))
    return _canonical_basis(V, s_ii), ev, flags


def _canonical_basis(V: np.ndarray, s_ii: np.ndarray) -> np.ndarray:
    """The columns of V made S_ii-orthonormal by Gram-Schmidt in their order (two
    passes), each with its largest-magnitude component positive."""
    V = V.copy()
    for _ in range(2):
        for c in range(V.shape[1]):
            v = V[:, c].copy()
            for d in range(c):
                v -= (V[:, d] @ s_ii @ v) * V[:, d]
            V[:, c] = v / math.sqrt(v @ s_ii @ v)
    for c in range(V.shape[1]):
        jm = int(np.argmax(np.abs(V[:, c])))
        if V[jm, c] < 0:
            V[:, c] = -V[:, c]
    return V


def projector_blocks(system, rho: np.ndarray, atoms=None) -> dict:
    """(S rho S)_{0i,0i} = sum_{Ra} sum_{Rb} S_{0i,Ra} rho_{Ra,Rb} S_{Rb,0i}, M_i x M_i.

    The on-site block of the occupied-space projector in the PAO metric: with
    rho = C f C^T (Eq. (dm)), <chi_0i|P|chi_0i> = S C f C^T S, the symmetric
    counterpart of Lambda_0i = (rho S)_{0i,0i} (Eq. (Lambda), Sec. II.B).

    rho_{Ra,Rb} = rho_{0a,(Rb-Ra)b} by translation invariance: block (a, t1) of
    row i and block (b, t2) of row a reach atom b in cell t1 + t2, whose overlap
    with the centre is block (b, t1 + t2) of row i, transposed (S is symmetric);
    terms whose block is absent from the pattern are zero.
    """
    if atoms is None:
        atoms = range(system.natoms)
    bidx = _BlockIndex(system)
    out = {}
    for i in atoms:
        i = int(i)
        mi = int(system.norb[i])
        G = np.zeros((mi, mi))
        for p in range(int(system.row_ptr[i]), int(system.row_ptr[i + 1])):
            a = int(system.col[p])
            ma = int(system.norb[a])
            t1 = system.shift[p]
            W = np.zeros((ma, mi))
            for q in range(int(system.row_ptr[a]), int(system.row_ptr[a + 1])):
                b = int(system.col[q])
                r = bidx.get(i, b, t1 + system.shift[q])
                if r is None:
                    continue
                W += system.block(rho, q) @ system.block(system.S, r).T
            G += system.block(system.S, p) @ W
        out[i] = G
    return out


def lnos_sym(G: np.ndarray, s_ii: np.ndarray, k: int, lambda_th: float | None = None):
    """LNOs of one atom from the symmetric-definite problem G v = lambda S_ii v,
    G = (S rho S)_ii (projector_blocks).

    Only the symmetric part of G enters: it is the block of S rho_s S with
    rho_s = (rho + rho^T)/2 (S is symmetric), the projector of the symmetrised
    density matrix; the raw rows of a DC step are not exactly symmetric.
    Eigenpairs by Cholesky + congruence + Jacobi, eigenvalues descending; the
    leading k are kept (with lambda_th, those >= lambda_th, at most k) and
    returned in the canonical basis of lnos().  Returns (V, eigenvalues (complex
    dtype, zero imaginary parts), flags = 0).
    """
    Gs = 0.5 * (G + G.T)
    w, C = gen_eig(Gs, s_ii)
    w, C = w[::-1].copy(), C[:, ::-1]
    kk = min(k, len(w))
    if lambda_th is not None:
        kk = min(kk, int(np.sum(w >= lambda_th)))
    return _canonical_basis(C[:, :kk], s_ii), w.astype(np.complex128), 0


def compute_lnos(system, rho: np.ndarray, k: int, atoms=None, lambda_th: float | None = None,
                 mode: str = "paper") -> dict:
    """atom -> (V, eigenvalues, flags) for the given atoms (default: all); with
    lambda_th, each atom keeps the eigenvectors whose eigenvalue is >= lambda_th
    (at most k), so V has that atom's own number of columns.  mode "paper" takes
    the nonsymmetric Lambda (lnos), mode "sym" the projector form (lnos_sym)."""
    if mode == "sym":
        G = projector_blocks(system, rho, atoms)
        return {i: lnos_sym(g, _on_site_block(system, i), k, lambda_th) for i, g in G.items()}
    if mode != "paper":
        raise ValueError(f"unknown LNO mode {mode!r}")
    lam = lambda_blocks(system, rho, atoms)
    return {i: lnos(L, _on_site_block(system, i), k, lambda_th) for i, L in lam.items()}


# --------------------------------------------------------------------------
# Cluster Hamiltonian and overlap: Eq. (Hi)
# --------------------------------------------------------------------------

def assemble(system, cl: Cluster, V: dict, bidx: _BlockIndex | None = None):
    """H^(i), S^(i) in the mixed basis.

    Basis of member m: identity on its M_j PAOs (core) or V_j (LNO member).
    Block (m1, m2) = B_m1^T X_{0 j1, (R2 - R1) j2} B_m2 for X = H, S, where
    the pair block is looked up in the BSR (zero if not stored).
    """
    if bidx is None:
        bidx = _BlockIndex(system)
    n = cl.dim
    Hc = np.zeros((n, n))
    Sc = np.zeros((n, n))
    K = len(cl.atoms)
    basis = []
    for m in range(K):
        j = int(cl.atoms[m])
        basis.append(None if cl.core[m] else V[j])
    for m1 in range(K):
        j1 = int(cl.atoms[m1])
        mi = int(system.norb[j1])
        o1a, o1b = int(cl.offsets[m1]), int(cl.offsets[m1 + 1])
        for m2 in range(K):
            j2 = int(cl.atoms[m2])
            b = bidx.get(j1, j2, cl.shifts[m2] - cl.shifts[m1])
            if b is None:
                continue
            mj = int(system.norb[j2])
            o = int(system.blk_off[b])
            hb = system.H[o:o + mi * mj].reshape(mi, mj)
            sb = system.S[o:o + mi * mj].reshape(mi, mj)
            if basis[m1] is not None:
                hb = basis[m1].T @ hb
                sb = basis[m1].T @ sb
            if basis[m2] is not None:
                hb = hb @ basis[m2]
                sb = sb @ basis[m2]
            o2a, o2b = int(cl.offsets[m2]), int(cl.offsets[m2 + 1])
            Hc[o1a:o1b, o2a:o2b] = hb
            Sc[o1a:o1b, o2a:o2b] = sb
    return Hc, Sc


# --------------------------------------------------------------------------
# Cluster eigenproblem and the spectral form of G^(i): Eq. (Gi)
# --------------------------------------------------------------------------

def solve_cluster(Hc: np.ndarray, Sc: np.ndarray, cl: Cluster):
    """eps (ascending), central-atom weights q and eigenvectors C.

    q_mu = sum_{alpha in centre} C_{alpha mu} (S^(i) C)_{alpha mu}: the
    central atom's Mulliken share of state mu, i.e. the weight of pole mu
    in the partial trace of G^(i) S^(i) over the central atom (Eq. (Gi),
    Eq. (tr_i)).  Sum over mu equals M_i.
    """
    eps, C = gen_eig(Hc, Sc)
    c = cl.centre_slice
    SC = Sc[c, :] @ C
    q = np.einsum("am,am->m", C[c, :], SC)
    return eps, q, C


def refine_eigenpairs(H: np.ndarray, S: np.ndarray, X: np.ndarray):
    """One sweep of Ogita-Aishima iterative refinement of a full eigendecomposition
    (Ogita & Aishima, Japan J. Indust. Appl. Math. 35 (2018)), carried over to the
    pencil H c = eps S c by taking every inner product in the S metric.

    Not a step of the paper: the mixed-precision path's refinement of approximate
    (FP32) eigenpairs with FP64 residuals.  With X the n x n approximate
    eigenvectors (columns),
      R = I - X^T S X,   G = X^T H X,   lam_i = G_ii / (1 - R_ii),
      E_ij = (G_ij + lam_j R_ij) / (lam_j - lam_i)   where |lam_i - lam_j| > delta,
      E_ij = R_ij / 2                                  otherwise (and on the diagonal),
      delta = 2 (||G - diag(lam)||_F + max|lam| ||R||_F),
    returns (X + X E, lam).  Two readings of the published threshold: the 2-norm of H
    becomes the pencil's spectral radius (max |lam|), the norm that bounds G in the S
    metric; and the 2-norms become Frobenius norms, upper bounds of them that one pass
    over the matrices computes (a larger delta only moves pairs to the close-pair rule).
    Each sweep squares the error while the starting error is below the gaps between
    eigenvalues; pairs closer than delta keep only their orthonormalisation."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[1]
    R = np.eye(n) - X.T @ S @ X
    G = X.T @ H @ X
    lam = np.diag(G) / (1.0 - np.diag(R))
    delta = 2.0 * (np.linalg.norm(G - np.diag(lam)) + np.max(np.abs(lam)) * np.linalg.norm(R))
    E = 0.5 * R  # the value of the close pairs and of the diagonal
    for i in range(n):
        for j in range(n):
            gap = lam[j] - lam[i]
            if i != j and abs(gap) > delta:
                E[i, j] = (G[i, j] + lam[j] * R[i, j]) / gap
    return X + X @ E, lam


def fermi(x):
    """Fermi-Dirac f(x) = 1 / (1 + e^x), evaluated without overflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x > 0
    e = np.exp(-x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def n_of_mu(eps_all: np.ndarray, q_all: np.ndarray, mu: float, kT: float) -> float:
    """N(mu) = 2 sum_i sum_mu f((eps - mu)/kT) q (spin factor 2, Eq. (tr_i))."""
    return 2.0 * float(np.sum(fermi((eps_all - mu) / kT) * q_all))


def find_mu(eps_all, q_all, n_e: float, kT: float, iters: int = 200):
    """Common chemical potential (Sec. II.C step (iv)) by bisection on N(mu) = N_e.

    Bracket [min eps - 40 kT, max eps + 40 kT]; at most ``iters`` halvings,
    stopping early when |N - N_e| <= 1e-12 N_e; returns (mu, N(mu)).
    """
    eps_all = np.asarray(eps_all, dtype=np.float64)
    q_all = np.asarray(q_all, dtype=np.float64)
    lo = float(eps_all.min()) - 40.0 * kT
    hi = float(eps_all.max()) + 40.0 * kT
    n_lo = n_of_mu(eps_all, q_all, lo, kT)
    n_hi = n_of_mu(eps_all, q_all, hi, kT)
    if not (n_lo <= n_e <= n_hi):
        raise NoBracket(f"N_e={n_e} outside [{n_lo}, {n_hi}]")
    mid = 0.5 * (lo + hi)
    n_mid = n_of_mu(eps_all, q_all, mid, kT)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        n_mid = n_of_mu(eps_all, q_all, mid, kT)
        if abs(n_mid - n_e) <= 1e-12 * n_e:
            break
        if n_mid < n_e:
            lo = mid
        else:
            hi = mid
    return mid, n_mid


def density_rows(system, cl: Cluster, eps, C, V: dict, mu: float, kT: float,
                 rho_out: np.ndarray, energy: bool = False):
    """Rows of the central atom i of rho (Eq. (dm)) or, with energy=True, of the
    energy density matrix e (Eq. (edm)), both with the spectral G^(i) of Eq. (Gi).

    The energy integrals reduce to sums over the cluster's poles:
    rho = sum_mu f(eps_mu) c_{mu,0i alpha} c_{mu,Rj beta} and
    e = sum_mu f(eps_mu) eps_mu c_{mu,0i alpha} c_{mu,Rj beta}.  Columns of an LNO
    member are returned to its PAOs with V_j; blocks of the S pattern outside the
    cluster are zero (only elements with S != 0 are kept).  Writes the rows into
    the BSR value array rho_out.
    """
    c = cl.centre_slice
    w = fermi((eps - mu) / kT)
    if energy:
        w = w * eps
    rcl = (C[c, :] * w[None, :]) @ C.T  # M_i x n
    _scatter_rows(system, cl, rcl, V, rho_out)


def density_rows_poles(system, cl: Cluster, Hc: np.ndarray, Sc: np.ndarray, V: dict, mu: float, kT: float,
                       rho_out: np.ndarray, n_poles: int) -> None:
    """The same rows from the Green function at the Matsubara poles (the
    generalisation of Eq. (rho0j) to a non-orthogonal basis), with no eigenvectors:
    f(x) = 1/2 + (2/beta) sum_{p>=0} Re 1/(i w_p - x), w_p = (2p+1) pi kT, so
        rho^(i) = S^-1 / 2 + (2/beta) Re sum_{p>=0} (z_p S - H)^-1,  z_p = mu + i w_p.
    The poles p >= n_poles are summed from the large-|z| expansion
    Re (z_p S - H)^-1 = -A_1/w_p^2 + A_3/w_p^4 - A_5/w_p^6 + ...,
    A_k = S^-1 ((H - mu S) S^-1)^k, with sum_{p>=P} w_p^-2m = (pi kT)^-2m zeta(2m, P + 1/2) / 4^m
    (Hurwitz zeta); this needs w_P well above the cluster's spectral radius about mu."""
    from scipy.special import zeta

    beta = 1.0 / kT
    n = Hc.shape[0]
    Sinv = np.linalg.inv(Sc)
    acc = np.zeros((n, n))
    for p in range(n_poles):
        z = mu + 1j * (2 * p + 1) * math.pi * kT
        acc += np.linalg.solve(z * Sc - Hc, np.eye(n)).real
    Bm = (Hc - mu * Sc) @ Sinv
    A1 = Sinv @ Bm
    A3 = A1 @ Bm @ Bm
    A5 = A3 @ Bm @ Bm
    def tail(m):  # sum_{p >= n_poles} w_p^-2m
        return (math.pi * kT) ** (-2 * m) * float(zeta(2 * m, n_poles + 0.5)) / 4 ** m
    acc += -A1 * tail(1) + A3 * tail(2) - A5 * tail(3)
    rho_c = 0.5 * Sinv + (2.0 / beta) * acc
    c = cl.centre_slice
    _scatter_rows(system, cl, rho_c[c, :], V, rho_out)


def _scatter_rows(system, cl: Cluster, rcl: np.ndarray, V: dict, rho_out: np.ndarray) -> None:
    """Central rows rcl (M_i x n, cluster basis) into the BSR rows of atom i: LNO
    columns back to PAOs with V_j, zero outside the cluster."""
    i = cl.centre
    where = {(int(cl.atoms[m]),) + tuple(int(x) for x in cl.shifts[m]): m for m in range(len(cl.atoms))}
    mi = int(system.norb[i])
    for b in range(int(system.row_ptr[i]), int(system.row_ptr[i + 1])):
        j = int(system.col[b])
        mj = int(system.norb[j])
        o = int(system.blk_off[b])
        m = where.get((j,) + tuple(int(x) for x in system.shift[b]))
        if m is None:
            blk = np.zeros((mi, mj))
        else:
            cols = rcl[:, int(cl.offsets[m]):int(cl.offsets[m + 1])]
            blk = cols if cl.core[m] else cols @ V[j].T
        rho_out[o:o + mi * mj] = blk.reshape(-1)


def energy_density(system, results: dict, V: dict, mu: float, kT: float) -> np.ndarray:
    """Energy density matrix e (Eq. (edm)) rows of every solved cluster, BSR values."""
    e = np.zeros_like(system.S)
    for r in results.values():
        density_rows(system, r.cluster, r.eps, r.C, V, mu, kT, e, energy=True)
    return e


@dataclasses.dataclass
class ClusterResult:
    cluster: Cluster
    eps: np.ndarray
    q: np.ndarray
    C: np.ndarray
    h_norm: float = 0.0  # Frobenius norms of H^(i) and S^(i) (for error bounds in tests)
    s_norm: float = 0.0


def _threads():
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


def dclno_solve(system, V: dict, r_core: float, r_lno: float, k_lno: int, atoms=None,
                threads: int | None = None, kappa: float | None = None, s_fna: float = 0.0,
                k_atoms=None) -> dict:
    """Clusters, assembly and eigen-solve for the given atoms (default all).

    Returns atom -> ClusterResult.  ``V`` must hold the LNOs of every atom that
    appears in an LNO region (unused when r_lno == r_core).  kappa, s_fna: the
    region rule of Sec. III instead of the fixed r_core (see cluster_members);
    k_atoms: per-atom LNO counts (threshold selection; default k_lno for all).
    """
    if atoms is None:
        atoms = list(range(system.natoms))
    bidx = _BlockIndex(system)
    clusters = [cluster_members(system, i, r_core, r_lno, k_lno, kappa, s_fna, k_atoms) for i in atoms]
    for cl in clusters:  # warm the per-row lookup tables outside the threads
        for j in set(int(a) for a in cl.atoms):
            bidx.row(j)

    def work(cl):
        Hc, Sc = assemble(system, cl, V, bidx)
        eps, q, C = solve_cluster(Hc, Sc, cl)
        return ClusterResult(cl, eps, q, C, float(np.linalg.norm(Hc)), float(np.linalg.norm(Sc)))

    nt = threads or _threads()
    if nt > 1 and len(clusters) > 1:
        with ThreadPoolExecutor(nt) as ex:
            res = list(ex.map(work, clusters))
    else:
        res = [work(cl) for cl in clusters]
    return {cl.centre: r for cl, r in zip(clusters, res)}


def finish_step(system, results: dict, V: dict, n_e: float, kT: float, mu: float | None = None):
    """Chemical potential (unless given), density-matrix rows and band energy.

    Returns (mu, N(mu), rho (BSR values, zero for rows of atoms not solved),
    E_band = 2 sum_i sum_mu f eps q).
    """
    eps_all = np.concatenate([r.eps for r in results.values()])
    q_all = np.concatenate([r.q for r in results.values()])
    if mu is None:
        mu, n_mu = find_mu(eps_all, q_all, n_e, kT)
    else:
        n_mu = n_of_mu(eps_all, q_all, mu, kT)
    rho = np.zeros_like(system.S)
    e_band = 0.0
    for r in results.values():
        density_rows(system, r.cluster, r.eps, r.C, V, mu, kT, rho)
        e_band += 2.0 * float(np.sum(fermi((r.eps - mu) / kT) * r.eps * r.q))
    return mu, n_mu, rho, e_band


def plain_dc_density(system, r: float, threads: int | None = None):
    """Plain-PAO divide-and-conquer step with clusters of radius r (no LNOs).

    This is the starting density of an LNO calculation (the paper updates
    LNOs every SCF step from the previous density; the first density is the
    plain DC one).  Returns (mu, N, rho, E_band, results).
    """
    res = dclno_solve(system, {}, r, r, 0, threads=threads)
    mu, n_mu, rho, e_band = finish_step(system, res, {}, system.n_electrons, system.kT)
    return mu, n_mu, rho, e_band, res


# --------------------------------------------------------------------------
# Conventional diagonalisation of a whole open system
# --------------------------------------------------------------------------

def dense_matrices(system):
    """Dense H, S of an open system (all stored shifts must be zero)."""
    if np.any(system.shift):
        raise ValueError("dense_matrices needs an open system")
    off = np.zeros(system.natoms + 1, dtype=np.int64)
    off[1:] = np.cumsum(system.norb)
    n = int(off[-1])
    H = np.zeros((n, n))
    S = np.zeros((n, n))
    brow = system.block_rows()
    for b in range(system.nnzb):
        i, j = int(brow[b]), int(system.col[b])
        mi, mj = int(system.norb[i]), int(system.norb[j])
        o = int(system.blk_off[b])
        H[off[i]:off[i + 1], off[j]:off[j + 1]] = system.H[o:o + mi * mj].reshape(mi, mj)
        S[off[i]:off[i + 1], off[j]:off[j + 1]] = system.S[o:o + mi * mj].reshape(mi, mj)
    return H, S, off


def full_diag(system, n_e=None, kT=None):
    """Exact solution of an open system: eps, C, mu, rho (BSR), E_band.

    N(mu) = 2 sum_mu f(eps_mu) (every state has total Mulliken weight 1);
    rho = C diag(f) C^T restricted to the stored pattern.
    """
    n_e = system.n_electrons if n_e is None else n_e
    kT = system.kT if kT is None else kT
    H, S, off = dense_matrices(system)
    eps, C = gen_eig(H, S)
    mu, n_mu = find_mu(eps, np.ones_like(eps), n_e, kT)
    f = fermi((eps - mu) / kT)
    R = (C * f[None, :]) @ C.T
    rho = np.zeros_like(system.S)
    brow = system.block_rows()
    for b in range(system.nnzb):
        i, j = int(brow[b]), int(system.col[b])
        mi, mj = int(system.norb[i]), int(system.norb[j])
        o = int(system.blk_off[b])
        rho[o:o + mi * mj] = R[off[i]:off[i + 1], off[j]:off[j + 1]].reshape(-1)
    e_band = 2.0 * float(np.sum(f * eps))
    return eps, C, mu, n_mu, rho, e_band


# --------------------------------------------------------------------------
# Dimension and cost model: Eq. (time-ratio)
# --------------------------------------------------------------------------

def cluster_dim(n_short: int, n_long: int, m_pao: int, m_lno: int) -> int:
    """Cluster dimension with PAOs on the short-range and LNOs on the long-range atoms."""
    return m_pao * n_short + m_lno * n_long


def time_ratio(m_pao: int, m_lno: int, n_short: float, n_long: float) -> float:
    """t_DC-LNO / t_DC = (M_P n_short + M_L n_long)^3 / (M_P (n_short + n_long))^3.

    Eq. (time-ratio) with n_short = N_F + kappa N_S and n_long = (1 - kappa) N_S,
    or with the region counts of an actual cluster.
    """
    return (cluster_dim(n_short, n_long, m_pao, m_lno) / (m_pao * (n_short + n_long))) ** 3
