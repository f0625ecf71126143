"""Synthetic tight-binding inputs: symmetry, the drop rule and the analytic overlap."""
import numpy as np
import pytest

import tbsystems as T


def _mirror_index(s):
    key = {}
    brow = s.block_rows()
    for b in range(s.nnzb):
        key[(int(brow[b]), int(s.col[b])) + tuple(int(x) for x in s.shift[b])] = b
    return key, brow


@pytest.mark.parametrize("which", ["cfg1", "mixed_system"])
def test_blocks_symmetric(which, request):
    s = request.getfixturevalue(which)
    key, brow = _mirror_index(s)
    for b in range(s.nnzb):
        i, j = int(brow[b]), int(s.col[b])
        mb = key[(j, i) + tuple(-int(x) for x in s.shift[b])]
        np.testing.assert_array_equal(s.block(s.S, b), s.block(s.S, mb).T)
        np.testing.assert_array_equal(s.block(s.H, b), s.block(s.H, mb).T)


def test_on_site_blocks(mixed_system):
    s = mixed_system
    brow = s.block_rows()
    for b in range(s.nnzb):
        i = int(brow[b])
        if int(s.col[b]) == i and not np.any(s.shift[b]):
            np.testing.assert_allclose(np.diag(s.block(s.S, b)), 1.0, rtol=0, atol=1e-15)
            np.testing.assert_array_equal(np.diag(s.block(s.H, b)), s.onsite[i])


def test_rows_sorted(mixed_system):
    s = mixed_system
    for i in range(s.natoms):
        b0, b1 = s.row_ptr[i], s.row_ptr[i + 1]
        keys = [(int(s.col[b]),) + tuple(int(x) for x in s.shift[b]) for b in range(b0, b1)]
        assert keys == sorted(keys)


def test_overlap_by_quadrature():
    """The closed-form Gaussian overlap against a separable numerical integral."""
    a, b = 0.37, 1.9
    R = np.array([0.8, -0.3, 1.1])
    x = np.linspace(-12, 12, 20001)
    dx = x[1] - x[0]
    val = 1.0
    for d in range(3):
        ga = (2 * a / np.pi) ** 0.25 * np.exp(-a * x ** 2)
        gb = (2 * b / np.pi) ** 0.25 * np.exp(-b * (x - R[d]) ** 2)
        val *= np.sum(ga * gb) * dx
    got = T.gaussian_overlap(np.array(a), np.array(b), np.array(R @ R))
    assert abs(got - val) < 1e-12


def test_drop_rule_and_cutoff(cfg1):
    s = cfg1
    nz = s.S[s.S != 0.0]
    assert np.all(np.abs(nz) >= T.DROP_TOL)
    assert np.all(s.H[s.S == 0.0] == 0.0)
    rc = T.overlap_cutoff(0.2)
    assert abs(T.gaussian_overlap(np.array(0.2), np.array(0.2), np.array(rc ** 2)) - T.DROP_TOL) < 1e-22


def test_wolfsberg_helmholz(mixed_system):
    """Two-centre elements: K = 1.75; one-centre elements: K = 1 (diagonal = on-site energy)."""
    s = mixed_system
    brow = s.block_rows()
    b = next(b for b in range(s.nnzb) if int(s.col[b]) != int(brow[b]))
    i, j = int(brow[b]), int(s.col[b])
    want = 1.75 * s.block(s.S, b) * 0.5 * (s.onsite[i][:, None] + s.onsite[j][None, :])
    np.testing.assert_allclose(s.block(s.H, b), want, rtol=1e-15, atol=0)
    b = next(b for b in range(s.nnzb) if int(s.col[b]) == int(brow[b]) and not np.any(s.shift[b]))
    i = int(brow[b])
    want = s.block(s.S, b) * 0.5 * (s.onsite[i][:, None] + s.onsite[i][None, :])
    np.testing.assert_allclose(s.block(s.H, b), want, rtol=1e-15, atol=0)


def test_no_spurious_low_states(cfg1):
    """With the one-centre K = 1 rule no cluster eigenvalue falls far below the on-site energies."""
    import oracle
    H, S, _ = oracle.dense_matrices(cfg1)
    eps = oracle.gen_eig(H, S)[0]
    assert eps.min() > -5.0


def test_cfg1_overlap_spd(cfg1):
    import oracle
    H, S, _ = oracle.dense_matrices(cfg1)
    assert np.all(np.linalg.eigvalsh(S) > 0)


def test_synthetic_density_symmetric(mixed_system):
    s = mixed_system
    rho = T.synthetic_density(s, seed=3)
    key, brow = _mirror_index(s)
    for b in range(s.nnzb):
        i, j = int(brow[b]), int(s.col[b])
        mb = key[(j, i) + tuple(-int(x) for x in s.shift[b])]
        np.testing.assert_allclose(s.block(rho, b), s.block(rho, mb).T, rtol=1e-15, atol=0)


def test_streamed_rows_equal_full_build():
    """Row-range generation (for systems whose matrices exceed host memory) gives the
    same structure, S, H and synthetic density as the one-shot build."""
    a = T.make_system(5, n_atoms=300)
    b = T.make_system_streamed(5, n_atoms=300)
    for k in ("row_ptr", "col", "shift", "blk_off"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert len(a.S) == len(b.S) and not np.any(b.S)
    for i0, i1 in ((0, 1), (17, 120), (290, 300)):
        o0, sv, hv = T.row_values(b, i0, i1)
        assert np.array_equal(sv, a.S[o0:o0 + len(sv)]) and np.array_equal(hv, a.H[o0:o0 + len(hv)])
    rho = T.synthetic_density(a, seed=11)
    o0, o1 = int(b.blk_off[b.row_ptr[40]]), int(b.blk_off[b.row_ptr[90]])
    part = np.zeros(o1 - o0)
    T.synthetic_density_rows(b, 40, 90, part, seed=11, base=o0)
    assert np.array_equal(part, rho[o0:o1])
    T.fill_rows(b, [3, 250])
    for i in (3, 250):
        o, e = int(b.blk_off[b.row_ptr[i]]), int(b.blk_off[b.row_ptr[i + 1]])
        assert np.array_equal(b.S[o:e], a.S[o:e]) and np.array_equal(b.H[o:e], a.H[o:e])


def _rsa_brute(n, L, dmin, rng, batch=65536):
    """Random sequential addition one candidate at a time (the definition): a candidate
    is kept when no kept point lies within dmin (minimum image) and its grid cell
    (width >= dmin / sqrt(3)) holds no kept point."""
    g = max(1, int(L / (dmin / np.sqrt(3.0))))
    cw = L / g
    pts, cells = [], set()
    while len(pts) < n:
        cand = rng.uniform(0.0, L, size=(batch, 3))
        for x in cand:
            c = tuple(np.minimum((x // cw).astype(np.int64), g - 1))
            if c in cells:
                continue
            if pts:
                d = np.asarray(pts) - x
                d -= L * np.round(d / L)
                if np.min(np.einsum("kd,kd->k", d, d)) < dmin * dmin:
                    continue
            pts.append(x)
            cells.add(c)
            if len(pts) == n:
                break
    return np.asarray(pts)


@pytest.mark.parametrize("n,L", [(150, 40.0), (120, 22.0)])
def test_rsa_matches_sequential_definition(n, L):
    """The batched packing (KD-tree screen, conflict graph within a batch) places the
    same points, in the same order, as the one-candidate-at-a-time definition; the
    second case is dense enough to need several batches and in-batch conflicts."""
    fast = T._rsa(n, L, 3.8, np.random.default_rng(5), batch=4096)
    ref = _rsa_brute(n, L, 3.8, np.random.default_rng(5), batch=4096)
    np.testing.assert_array_equal(fast, ref)


def test_streamed_rows_match_full_build():
    """The tabled, threaded row generator of streamed systems gives the structure and
    the values of the per-block construction (a ragged-path BsrRows), and the
    synthetic density rows agree with synthetic_density."""
    s = T.make_system(5, n_atoms=300)
    st = T.make_system_streamed(5, n_atoms=300)
    for a in ("row_ptr", "col", "shift", "blk_off"):
        np.testing.assert_array_equal(getattr(st, a), getattr(s, a))
    Sv, Hv, Rv = np.empty(len(s.S)), np.empty(len(s.S)), np.empty(len(s.S))
    for i0, i1, o0, sv, hv, rv in T.row_chunks(st, 37, workers=3, density_seed=11):
        Sv[o0:o0 + len(sv)], Hv[o0:o0 + len(hv)], Rv[o0:o0 + len(rv)] = sv, hv, rv
    np.testing.assert_array_equal(Sv, s.S)
    np.testing.assert_array_equal(Hv, s.H)
    np.testing.assert_array_equal(Rv, T.synthetic_density(s, seed=11))
    ragged = T.BsrRows(st.pos, st.cell, st.pbc, st.exps, st.onsite)
    ragged.tabled = False
    for i0, i1 in ((0, 3), (150, 152), (297, 300)):
        for (c1, sh1, s1, h1), (c2, sh2, s2, h2) in zip(ragged.rows(i0, i1), st.source.rows(i0, i1)):
            np.testing.assert_array_equal(c1, c2)
            np.testing.assert_array_equal(sh1, sh2)
            np.testing.assert_allclose(s1, s2, rtol=1e-14, atol=0)
            np.testing.assert_allclose(h1, h2, rtol=1e-14, atol=0)


def test_known_pencils_hold_their_eigenpairs():
    """The refinement tests' pencils: H C = S C diag(w), C^T S C = I, S symmetric
    with the stated conditioning, eigenvalues ascending at least half their spacing
    apart; seeded (the same seed gives the same pencils)."""
    H, S, C, w = T.known_pencils(2, 33, seed=7)
    H2, _, _, _ = T.known_pencils(2, 33, seed=7)
    assert np.array_equal(H, H2)
    for p in range(2):
        assert np.max(np.abs(H[p] @ C[p] - S[p] @ C[p] * w[p])) <= 1e-13
        assert np.max(np.abs(C[p].T @ S[p] @ C[p] - np.eye(33))) <= 1e-13
        assert np.array_equal(S[p], S[p].T) and np.array_equal(H[p], H[p].T)
        ev = np.linalg.eigvalsh(S[p])
        assert abs(ev[-1] / ev[0] - 100.0) <= 1e-8
        assert np.min(np.diff(w[p])) >= 0.5 * 4.0 / 32
