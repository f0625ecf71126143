"""The 7,840-atom metallic bcc slab (2% vacancies, vacuum on both z surfaces):
five SCF steps of LNO regeneration, cluster solve and chemical potential with
linear density mixing 0.3, as one captured CUDA graph and as eager launches.

Checks: the graph and the eager loop agree bit for bit; the first step equals an
explicit dclno_step followed by the mixing formula; N(mu) = N_e at every step;
sampled clusters of the first step match the oracle (per-state eigenvalue bound);
the final step keeps sum_mu q_mu = M_i for every cluster.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import spectral_moments, state_tol, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_FP64, Context  # noqa: E402

ALPHA = 0.3
STEPS = 5


@pytest.fixture(scope="module")
def slab():
    s = T.make_system(4)
    rho0 = T.synthetic_density(s, seed=4)
    return s, rho0


def _ctx(s, stream):
    ctx = Context(stream=stream.cuda_stream)
    H, S = to_dev(s.H), to_dev(s.S)
    torch.cuda.synchronize()
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, H, S,
                       s.r_core, s.r_lno, s.k_lno)
    return ctx, (H, S)


def test_scf_loop_graph_equals_eager_and_mixing(slab):
    s, rho0 = slab
    stream = torch.cuda.Stream()
    ctx, keep = _ctx(s, stream)
    dims = ctx.cluster_info()[0]
    assert dims.min() >= 100 and dims.max() <= 400
    with torch.cuda.stream(stream):
        ra = to_dev(rho0)
        rb = to_dev(rho0)
        r1 = to_dev(rho0)
    torch.cuda.synchronize()
    mu_a, n_a, e_a = ctx.scf_run(ra, STEPS, ALPHA, s.n_electrons, s.kT, DCLNO_FP64, use_graph=True)
    mu_b, n_b, e_b = ctx.scf_run(rb, STEPS, ALPHA, s.n_electrons, s.kT, DCLNO_FP64, use_graph=False)
    torch.cuda.synchronize()
    assert torch.equal(ra, rb)
    np.testing.assert_array_equal(mu_a, mu_b)
    np.testing.assert_array_equal(e_a, e_b)
    assert np.all(np.abs(n_a - s.n_electrons) <= 1e-10 * s.n_electrons)
    # the first step by hand: dclno_step, then rho + 0.3 (rho_out - rho)
    with torch.cuda.stream(stream):
        out = torch.zeros_like(r1)
    torch.cuda.synchronize()
    mu1, n1, e1 = ctx.step(r1, out, s.n_electrons, s.kT)
    mix = r1 + ALPHA * (out - r1)
    mu_c, n_c, e_c = ctx.scf_run(r1, 1, ALPHA, s.n_electrons, s.kT, DCLNO_FP64, use_graph=False)
    torch.cuda.synchronize()
    assert mu_c[0] == mu1 and e_c[0] == e1 == e_a[0]
    assert float((r1 - mix).abs().max()) <= 1e-12 * float(mix.abs().max())
    ctx.close()


def test_first_step_sampled_clusters_match_oracle(slab):
    s, rho0 = slab
    stream = torch.cuda.Stream()
    ctx, keep = _ctx(s, stream)
    with torch.cuda.stream(stream):
        r = to_dev(rho0)
    torch.cuda.synchronize()
    ctx.scf_run(r, 1, ALPHA, s.n_electrons, s.kT, DCLNO_FP64, use_graph=False)
    spec = ctx.spectrum()
    ctx.close()
    z = s.pos[:, 2]
    sample = [0, int(np.argmin(np.abs(z - z.mean()))), int(np.argmax(z)), s.natoms // 3]
    need = set()
    for i in sample:
        cl = O.cluster_members(s, i, s.r_core, s.r_lno, s.k_lno)
        need |= {int(a) for a, c in zip(cl.atoms, cl.core) if not c}
    lno = O.compute_lnos(s, rho0, s.k_lno, atoms=sorted(need))
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno, atoms=sample, threads=len(sample))
    mus = np.linspace(-0.6, 0.2, 9)
    for i, rr in res.items():
        e_gpu, q_gpu = spec[i]
        assert np.all(np.abs(np.sort(e_gpu) - rr.eps) <= state_tol(rr)), f"cluster {i}"
        np.testing.assert_allclose(spectral_moments(e_gpu, q_gpu, mus, s.kT),
                                   spectral_moments(rr.eps, rr.q, mus, s.kT), rtol=0, atol=1e-8)
    for i, (e, q) in enumerate(spec):
        assert abs(q.sum() - s.norb[i]) < 1e-8
