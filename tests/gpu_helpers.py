"""Shared helpers of the GPU tests (no test functions here)."""
import numpy as np
import torch

from paper_1809_05637_gb300 import Context


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gpu_context(s, r_core, r_lno, k_lno, H=None, S=None, tridiag=None, tear=None):
    """A context with the system's clusters built; tridiag and tear (if given) are
    selected before the build (the layout depends on both)."""
    H = to_dev(s.H) if H is None else H
    S = to_dev(s.S) if S is None else S
    ctx = Context()
    if tridiag is not None:
        ctx.set_tridiag(tridiag)
    if tear is not None:
        ctx.set_tear(tear)
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


def oracle_sample(s, rho_in, sample):
    """The oracle's LNOs (of the sampled clusters' LNO members) and its solve of the
    sampled clusters, from the same input density: (lno, V, results)."""
    import oracle as O

    need = set()
    for i in sample:
        cl = O.cluster_members(s, i, s.r_core, s.r_lno, s.k_lno)
        need |= {int(a) for a, c in zip(cl.atoms, cl.core) if not c}
    lno = O.compute_lnos(s, rho_in, s.k_lno, atoms=sorted(need))
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno, atoms=list(sample), threads=len(sample))
    return lno, V, res


def row_range(s, i):
    """Value range [o0, o1) of the BSR row of atom i."""
    b0, b1 = s.row_ptr[i], s.row_ptr[i + 1]
    return int(s.blk_off[b0]), int(s.blk_off[b1 - 1] + s.norb[i] * s.norb[s.col[b1 - 1]])


def check_sampled_clusters(s, V, res, spec, rho_test, mu_test, row_tol, mus):
    """Sampled clusters of a GPU solve against the oracle: eigenvalues within the
    first-order bound of each state (state_tol), weights through smooth spectral
    sums with that bound propagated through f', and the density rows at the fixed
    chemical potential mu_test within row_tol(r, big) (big = the row's largest
    element).  Returns the largest eigenvalue difference over its bound and the
    largest row difference over the row's largest element (for reports)."""
    import oracle as O

    worst_eps, worst_rho = 0.0, 0.0
    for i, r in res.items():
        e_gpu, q_gpu = spec[i]
        assert len(e_gpu) == len(r.eps), f"cluster {i}: dimension"
        tol = state_tol(r)
        d = np.abs(np.sort(e_gpu) - r.eps)
        worst_eps = max(worst_eps, float(np.max(d / tol)))
        assert np.all(d <= tol), f"cluster {i}: eigenvalues (worst {np.max(d / tol):.3g} of the bound)"
        for x in mus:
            g = spectral_moments(e_gpu, q_gpu, [x], s.kT)[0]
            o = spectral_moments(r.eps, r.q, [x], s.kT)[0]
            f = fermi((r.eps - x) / s.kT)
            fp = f * (1.0 - f) / s.kT
            assert abs(g - o) <= 1e-9 + float(np.sum(fp * tol * np.abs(r.q))), f"cluster {i}: weights at {x}"
        rows = np.zeros_like(s.S)
        O.density_rows(s, r.cluster, r.eps, r.C, V, mu_test, s.kT, rows)
        o0, o1 = row_range(s, i)
        big = float(np.max(np.abs(rows[o0:o1])))
        worst_rho = max(worst_rho, float(np.max(np.abs(rho_test[o0:o1] - rows[o0:o1]))) / big)
        np.testing.assert_allclose(rho_test[o0:o1], rows[o0:o1], rtol=0, atol=row_tol(r, big))
    return worst_eps, worst_rho
