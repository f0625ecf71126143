"""Symmetric LNO mode (dclno_set_lno_mode(DCLNO_LNO_SYM)): the LNOs from
(S rho S)_ii v = lambda S_ii v on the GPU against the oracle's projector form --
eigenvalues, spans, threshold counts, a whole step on the 64-atom open system, a
periodic cell (image shifts t1 + t2 in the projector sum) -- and the mode switch
back to the paper's Lambda."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import tbsystems as T  # noqa: E402
from gpu_helpers import gpu_context, spectral_moments, state_tol, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_LNO_PAPER, DCLNO_LNO_SYM, Context, DclnoError  # noqa: E402


def _check_lnos(got, ref, atoms, k_of=None):
    for j in atoms:
        Vg, evg, flg = got[j]
        Vo, evo, flo = ref[j]
        assert flg == 0 and not np.any(evg.imag)
        scale = max(1.0, float(np.max(np.abs(evo.real))))
        np.testing.assert_allclose(evg.real, evo.real, rtol=0, atol=1e-10 * scale, err_msg=f"atom {j}")
        kj = Vo.shape[1] if k_of is None else k_of[j]
        np.testing.assert_allclose(Vg[:, :kj] @ Vg[:, :kj].T, Vo @ Vo.T, rtol=0, atol=1e-8, err_msg=f"atom {j}")
        assert not np.any(Vg[:, kj:])


def test_sym_lnos_match_oracle(mixed_system):
    s = mixed_system
    rho = T.synthetic_density(s, seed=9)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.set_lno_mode(DCLNO_LNO_SYM)
    ctx.compute_lnos(to_dev(rho))
    ref = O.compute_lnos(s, rho, s.k_lno, mode="sym")
    _check_lnos(ctx.lnos(), ref, range(s.natoms))
    # threshold selection in the same mode
    th = float(np.median([r[1].real[1] for r in ref.values()]))
    ctx.set_lno_threshold(th)
    ctx.compute_lnos(to_dev(rho))
    ref_t = O.compute_lnos(s, rho, s.k_lno, lambda_th=th, mode="sym")
    counts = ctx.lno_counts()
    ko = np.array([ref_t[j][0].shape[1] for j in range(s.natoms)])
    assert np.array_equal(counts, ko) and set(ko.tolist()) == {1, 2}
    _check_lnos(ctx.lnos(), ref_t, range(s.natoms), k_of=counts)
    ctx.close()


def test_sym_exact_density_unit_interval(cfg1, cfg1_exact):
    s = cfg1
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.set_lno_mode(DCLNO_LNO_SYM)
    ctx.compute_lnos(to_dev(cfg1_exact[4]))
    ev = np.concatenate([v[1].real for v in ctx.lnos().values()])
    assert ev.min() > -1e-10 and ev.max() < 1 + 1e-10
    ctx.close()


def test_sym_step_matches_oracle(cfg1, cfg1_dc0):
    s = cfg1
    rho0 = cfg1_dc0[2]
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.set_lno_mode(DCLNO_LNO_SYM)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    mu, n, e_gpu = ctx.step(to_dev(rho0), out, s.n_electrons, s.kT)
    spec = ctx.spectrum()
    lno = O.compute_lnos(s, rho0, s.k_lno, mode="sym")
    _check_lnos(ctx.lnos(), lno, range(s.natoms))
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno)
    mu_o, n_o, rho_o, e_o = O.finish_step(s, res, V, s.n_electrons, s.kT)
    for i, r in res.items():
        assert np.all(np.abs(np.sort(spec[i][0]) - r.eps) <= state_tol(r)), f"cluster {i}"
        np.testing.assert_allclose(spectral_moments(spec[i][0], spec[i][1], [mu_o], s.kT),
                                   spectral_moments(r.eps, r.q, [mu_o], s.kT), rtol=0, atol=1e-9)
    assert abs(mu - mu_o) <= 1e-9
    np.testing.assert_allclose(out.cpu().numpy(), rho_o, rtol=0, atol=1e-9)
    assert abs(e_gpu - e_o) <= 1e-9 * abs(e_o)
    ctx.close()


def test_sym_scf_graph_matches_loop(mixed_system):
    """The graph-captured SCF loop runs the same kernels in this mode."""
    s = mixed_system
    rho0 = T.synthetic_density(s, seed=12)
    stream = torch.cuda.Stream()
    hist, rhos = [], []
    with torch.cuda.stream(stream):
        for g in (False, True):
            ctx = Context(stream=stream.cuda_stream)
            ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, to_dev(s.H),
                               to_dev(s.S), s.r_core, s.r_lno, s.k_lno)
            ctx.set_lno_mode(DCLNO_LNO_SYM)
            r = to_dev(rho0.copy())
            hist.append(ctx.scf_run(r, 3, 0.3, s.n_electrons, s.kT, use_graph=g))
            stream.synchronize()
            rhos.append(r.cpu().numpy())
            ctx.close()
    for a, b in zip(*hist):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(rhos[0], rhos[1])


def test_sym_periodic_cell():
    """512 atoms in a periodic 19.2-bohr cube: every block of the projector sum that
    crosses the cell boundary goes through the shift t1 + t2."""
    pos, _ = T._sc_lattice(8, 8, 8, 2.4)
    pos = pos + np.random.default_rng(3).normal(0, 0.05, pos.shape)
    n = len(pos)
    s = T.assemble_system("periodic512", pos, np.eye(3) * 19.2, np.ones(3, bool), np.zeros(n, np.int32),
                          [np.array([1.5, 3.5])] * n, [np.array([-0.4, 0.3])] * n, float(n), 0.02, 3.0, 5.0, 1)
    rho = T.synthetic_density(s, seed=8)
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.set_lno_mode(DCLNO_LNO_SYM)
    ctx.compute_lnos(to_dev(rho))
    atoms = [0, 7, 63, 64, 300, 511]  # corner, edge and inner sites of the cube
    ref = O.compute_lnos(s, rho, s.k_lno, atoms=atoms, mode="sym")
    _check_lnos(ctx.lnos(), ref, atoms)
    ctx.close()


def test_mode_switch_and_refusal(mixed_system):
    s = mixed_system
    rho = to_dev(T.synthetic_density(s, seed=10))
    fresh = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    fresh.compute_lnos(rho)
    paper = fresh.lnos()
    fresh.close()
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.set_lno_mode(DCLNO_LNO_SYM)
    ctx.compute_lnos(rho)
    ctx.set_lno_mode(DCLNO_LNO_PAPER)
    ctx.compute_lnos(rho)
    back = ctx.lnos()
    for j in range(s.natoms):
        np.testing.assert_array_equal(back[j][0], paper[j][0])
        np.testing.assert_array_equal(back[j][1], paper[j][1])
    with pytest.raises(DclnoError, match="unknown mode"):
        ctx.set_lno_mode(2)
    ctx.close()
