"""Pins of the oracle's cluster assembly (Eq. (Hi)) against dense projections.

H^(i) = B^T H B and S^(i) = B^T S B, with B the basis map of the cluster: the
identity on the PAOs of a short-range member, V_j on an LNO member, members in
the cluster's order.  Both pins build B and the matrices densely, independently
of the block-by-block assembly:

* an open, fully connected system with LNOs (k < M, so the LNO blocks matter);
* a periodic cell more than three overlap radii wide, where every member pair
  has one stored image and the cluster's blocks are the folded dense blocks of
  the members' atoms at their displacements inside the cluster.
"""
import numpy as np

import oracle as O
import tbsystems as T


def _dense(s, vals):
    off = np.concatenate([[0], np.cumsum(s.norb)])
    D = np.zeros((off[-1], off[-1]))
    brow = s.block_rows()
    for b in range(s.nnzb):
        i, j = int(brow[b]), int(s.col[b])
        D[off[i]:off[i + 1], off[j]:off[j + 1]] += s.block(vals, b)
    return D, off


def _basis_map(s, cl, V, off):
    B = np.zeros((off[-1], cl.dim))
    for m, (j, core) in enumerate(zip(cl.atoms, cl.core)):
        j = int(j)
        rows = slice(off[j], off[j + 1])
        cols = slice(int(cl.offsets[m]), int(cl.offsets[m + 1]))
        B[rows, cols] = np.eye(int(s.norb[j])) if core else V[j]
    return B


def test_assemble_open_system_with_lnos(cfg1, cfg1_dc0):
    s = cfg1
    assert np.diff(s.row_ptr).min() == s.natoms  # every pair stored: the dense H is the BSR H
    lno = O.compute_lnos(s, cfg1_dc0[2], 2)
    V = {i: v[0] for i, v in lno.items()}
    H, off = _dense(s, s.H)
    S, _ = _dense(s, s.S)
    for i in (0, 21, 63):
        cl = O.cluster_members(s, i, 5.0, 8.0, 2)
        assert np.any(~cl.core) and np.any(cl.core)
        Hc, Sc = O.assemble(s, cl, V)
        B = _basis_map(s, cl, V, off)
        np.testing.assert_allclose(Hc, B.T @ H @ B, rtol=0, atol=1e-12)
        np.testing.assert_allclose(Sc, B.T @ S @ B, rtol=0, atol=1e-12)
        assert int(cl.atoms[-1]) == i and np.all(cl.core[cl.dist <= 5.0 + 1e-9])


def test_assemble_periodic_cell():
    pos, _ = T._sc_lattice(8, 8, 8, 2.4)
    pos = pos + np.random.default_rng(3).normal(0, 0.05, pos.shape)
    n = len(pos)
    s = T.assemble_system("periodic512", pos, np.eye(3) * 19.2, np.ones(3, bool), np.zeros(n, np.int32),
                          [np.array([1.5, 3.5])] * n, [np.array([-0.4, 0.3])] * n, float(n), 0.02, 3.0, 5.0, 1)
    brow = s.block_rows()
    d = np.linalg.norm(s.pos[s.col] + s.shift @ s.cell - s.pos[brow], axis=1)
    assert 3 * d.max() < 19.2
    H, off = _dense(s, s.H)  # image sums fold into one entry per pair
    S, _ = _dense(s, s.S)
    for i in (0, 7, 511):  # corner atoms: the cluster wraps across the cell
        cl = O.cluster_members(s, i, 5.0, 5.0, 0)
        assert np.any(cl.shifts != 0)
        assert len(set(int(a) for a in cl.atoms)) == len(cl.atoms)  # no atom twice
        Hc, Sc = O.assemble(s, cl, {})
        B = _basis_map(s, cl, {}, off)
        np.testing.assert_allclose(Hc, B.T @ H @ B, rtol=0, atol=1e-14)
        np.testing.assert_allclose(Sc, B.T @ S @ B, rtol=0, atol=1e-14)
