"""Memory-admitted batches (dclno_set_workspace_limit): a context whose cluster
workspace is split into several batches gives the same spectra, chemical
potential, density and energy density matrices, band energy and SCF history as
a context that holds every cluster at once, bit for bit (each cluster is solved
by the same kernels on the same input, whatever batch it sits in).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import tbsystems as T  # noqa: E402
from gpu_helpers import to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, Context, DclnoError  # noqa: E402


def _ctx(s, limit=0, stream=None):
    ctx = Context(stream=None if stream is None else stream.cuda_stream)
    if limit:
        ctx.set_workspace_limit(limit)
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                       to_dev(s.S), s.r_core, s.r_lno, s.k_lno)
    return ctx


def _step(ctx, s, rho_in, prec):
    ctx.compute_lnos(to_dev(rho_in))
    ctx.solve_clusters(prec)
    mu, n = ctx.find_mu(s.n_electrons, s.kT)
    rho = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    edm = torch.zeros_like(rho)
    eb = ctx.density_matrices(mu, s.kT, rho, edm)
    spec = ctx.spectrum()
    eps = np.concatenate([e for e, _ in spec])
    q = np.concatenate([w for _, w in spec])
    return dict(mu=mu, n=n, eb=eb, rho=rho.cpu().numpy(), edm=edm.cpu().numpy(), eps=eps, q=q)


@pytest.mark.parametrize("prec", [DCLNO_FP64, DCLNO_MIXED])
def test_batches_match_single_workspace(mixed_system, prec):
    s = mixed_system
    rho_in = T.synthetic_density(s, seed=5)
    one = _ctx(s)
    nb1, ws1 = one.batch_info()
    assert nb1 == 1
    ref = _step(one, s, rho_in, prec)
    one.close()
    many = _ctx(s, limit=ws1 // 3 + 1)
    nb, ws = many.batch_info()
    assert nb >= 3 and ws <= ws1 // 3 + 1
    got = _step(many, s, rho_in, prec)
    for k in ("eps", "q", "rho", "edm"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert got["mu"] == ref["mu"] and got["n"] == ref["n"] and got["eb"] == ref["eb"]
    # a second density call (the resident batch is now the last one re-solved)
    rho2 = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    assert many.density_matrix(ref["mu"], s.kT, rho2) == ref["eb"]
    np.testing.assert_array_equal(rho2.cpu().numpy(), ref["rho"])
    many.close()


def test_batched_scf_graph_matches(mixed_system):
    s = mixed_system
    rho0 = T.synthetic_density(s, seed=6)
    stream = torch.cuda.Stream()
    hist = []
    rhos = []
    with torch.cuda.stream(stream):
        ws1 = None
        for batched in (False, True):
            ctx = _ctx(s, limit=ws1 // 4 + 1 if batched else 0, stream=stream)
            nb, ws = ctx.batch_info()
            assert nb >= 4 if batched else nb == 1
            ws1 = ws
            rho = to_dev(rho0.copy())
            hist.append(ctx.scf_run(rho, 3, 0.3, s.n_electrons, s.kT, use_graph=True))
            stream.synchronize()
            rhos.append(rho.cpu().numpy())
            ctx.close()
    for a, b in zip(hist[0], hist[1]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(rhos[0], rhos[1])


def test_limit_below_one_cluster_is_refused(mixed_system):
    s = mixed_system
    ctx = Context()
    ctx.set_workspace_limit(1024)
    with pytest.raises(DclnoError, match="exceeds the workspace budget"):
        ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                           to_dev(s.S), s.r_core, s.r_lno, s.k_lno)
    ctx.close()


def test_cfg2_two_batches_match():
    """The 1,728-atom workload with half the workspace: two batches, same rho."""
    s = T.make_system(2)
    rho_in = T.synthetic_density(s, seed=11)
    H, S = to_dev(s.H), to_dev(s.S)

    def run(limit):
        ctx = Context()
        if limit:
            ctx.set_workspace_limit(limit)
        ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, H, S,
                           s.r_core, s.r_lno, s.k_lno)
        nb, ws = ctx.batch_info()
        rho = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
        mu, n, eb = ctx.step(to_dev(rho_in), rho, s.n_electrons, s.kT)
        ctx.close()
        return nb, ws, mu, eb, rho.cpu().numpy()

    nb1, ws1, mu1, eb1, rho1 = run(0)
    assert nb1 == 1
    nb2, ws2, mu2, eb2, rho2 = run(int(ws1 * 0.55))  # slack of many clusters' workspace over half
    assert nb2 == 2 and ws2 < ws1
    assert mu2 == mu1 and eb2 == eb1
    np.testing.assert_array_equal(rho2, rho1)
