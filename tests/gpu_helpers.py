"""Shared helpers of the GPU tests (no test functions here)."""
import numpy as np
import torch

from paper_1809_05637_gb300 import Context


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gpu_context(s, r_core, r_lno, k_lno, H=None, S=None):
    H = to_dev(s.H) if H is None else H
    S = to_dev(s.S) if S is None else S
    ctx = Context()
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, H, S,
                       r_core, r_lno, k_lno)
    return ctx


def fermi(x):
    x = np.asarray(x, float)
    out = np.empty_like(x)
    p = x > 0
    e = np.exp(-x[p])
    out[p] = e / (1 + e)
    out[~p] = 1 / (1 + np.exp(x[~p]))
    return out


def spectral_moments(eps, q, mus, kT):
    """sum_mu f((eps-mu)/kT) q for several mu: invariant within degenerate groups."""
    return np.array([np.sum(fermi((eps - m) / kT) * q) for m in mus])


def eps_tol(e):
    return 1e-10 + 1e-12 * np.abs(e)


U = 2.0 ** -53


def state_tol(r):
    """First-order bound for each eigenvalue of the pencil (H^(i), S^(i)): a backward
    error of n u in H and S moves eps_mu by at most n u (|H| + |eps_mu| |S|) c_mu^T c_mu
    (c_mu^T S c_mu = 1).  1e-10 Ha is the floor; well-conditioned states stay there."""
    n = len(r.eps)
    cc = np.einsum("am,am->m", r.C, r.C)
    return 1e-10 + 2.0 * n * U * (r.h_norm + np.abs(r.eps) * r.s_norm) * cc


def rho_row_tol(r, big):
    """Density-matrix elements of one cluster: rho = C F C^T with C S^(i)-orthonormal
    has a first-order relative error of at most n u kappa for a backward error of
    n u in S^(i), kappa = |S^(i)| max_mu c_mu^T c_mu (the condition number of the
    cluster overlap); big is the largest element of the rows compared."""
    n = len(r.eps)
    kappa = r.s_norm * float(np.max(np.einsum("am,am->m", r.C, r.C)))
    return 1e-9 + n * U * kappa * big
