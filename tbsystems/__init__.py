"""Seeded synthetic tight-binding systems: the inputs of a DC-LNO step.

The paper's workloads are DFT solids described by pseudo-atomic orbitals (PAOs)
and GGA Hamiltonians (Sec. III).  Neither the PAO database nor a DFT code is
available here, so the systems below stand in for them: every atom carries
normalised s-type Gaussians, the overlap S is the analytic Gaussian overlap
and H follows the Wolfsberg-Helmholz rule.  The matrices are stored in the
paper's atom-pair block form S_{0i,Rj}, H_{0i,Rj} (the M_i x M_j blocks of
Sec. II.B, between atom i in the central cell and atom j in cell R), as a
block-sparse-row (BSR) structure keyed by (i, j, R).

This module holds no DC-LNO arithmetic.  It serves both the CUDA path and the
oracle: geometry, basis, the analytic S and H, and a seeded synthetic density
matrix used as the input of a single LNO step in tests.

Conventions
-----------
* Units: bohr and hartree.
* ``cell`` rows are the lattice vectors; ``pbc[d]`` says whether direction d
  is periodic.  A shift R is an integer triple; the image of atom j in cell R
  sits at ``pos[j] + R @ cell``.
* BSR: row i holds blocks ``b`` in ``row_ptr[i]:row_ptr[i+1]``, sorted by
  ``(col[b], shift[b][0], shift[b][1], shift[b][2])``.  Block b is the
  M_i x M_col row-major matrix starting at element ``blk_off[b]`` of ``S`` and
  ``H``.
* Entries of S below ``drop_tol`` (1e-10) are dropped (set to zero, and blocks
  that become all-zero are removed); H is zero wherever S is.
* Hamiltonian (extended-Hueckel form): two-centre elements (orbitals on
  different atoms, or on different images of one atom) follow Wolfsberg-Helmholz,
  H_ab = 1.75 S_ab (h_a + h_b)/2; one-centre elements use the same form with
  K = 1, H_ab = S_ab (h_a + h_b)/2, which gives H_aa = h_a (the on-site energy).
  Applying K = 1.75 to one-centre pairs of the strongly overlapping same-atom
  Gaussians would make H inconsistent with S in its near-null space and put
  spurious eigenvalues of order h / lambda_min(S) ~ 1e5 Ha into every cluster.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

DROP_TOL = 1e-10
WH_K = 1.75  # Wolfsberg-Helmholz constant


@dataclasses.dataclass
class System:
    name: str
    pos: np.ndarray          # (N, 3) float64, bohr
    cell: np.ndarray         # (3, 3) float64, rows = lattice vectors
    pbc: np.ndarray          # (3,) bool
    species: np.ndarray      # (N,) int32
    exps: list               # per atom: (M_i,) Gaussian exponents
    onsite: list             # per atom: (M_i,) on-site energies, hartree
    norb: np.ndarray         # (N,) int32, M_i
    row_ptr: np.ndarray      # (N+1,) int64
    col: np.ndarray          # (nnzb,) int32
    shift: np.ndarray        # (nnzb, 3) int8
    blk_off: np.ndarray      # (nnzb,) int64, element offset of each block
    S: np.ndarray            # (nval,) float64
    H: np.ndarray            # (nval,) float64
    n_electrons: float
    kT: float
    r_core: float
    r_lno: float
    k_lno: int
    source: object = None    # BsrRows of a system whose S, H are filled on demand (make_system_streamed)

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    def block(self, arr: np.ndarray, b: int) -> np.ndarray:
        """Block b of the flat value array ``arr`` as an M_i x M_j view."""
        i = int(np.searchsorted(self.row_ptr, b, side="right") - 1)
        mi, mj = int(self.norb[i]), int(self.norb[self.col[b]])
        o = int(self.blk_off[b])
        return arr[o:o + mi * mj].reshape(mi, mj)

    def block_rows(self) -> np.ndarray:
        """Row (atom i) of every block, (nnzb,) int64."""
        return np.repeat(np.arange(self.natoms), np.diff(self.row_ptr))


# --------------------------------------------------------------------------
# Basis and pair matrices
# --------------------------------------------------------------------------

def gaussian_overlap(a: np.ndarray, b: np.ndarray, r2: np.ndarray) -> np.ndarray:
    """Overlap of normalised s-Gaussians (2a/pi)^(3/4) exp(-a r^2).

    S_ab(R) = (2 sqrt(ab)/(a+b))^(3/2) exp(-ab R^2/(a+b)); shapes broadcast.
    """
    p = a + b
    return (2.0 * np.sqrt(a * b) / p) ** 1.5 * np.exp(-(a * b / p) * r2)


def overlap_cutoff(min_exp: float, tol: float = DROP_TOL) -> float:
    """Distance beyond which every overlap entry is below ``tol``.

    The slowest-decaying pair is the most diffuse exponent with itself,
    exp(-a R^2 / 2), whose prefactor is 1.
    """
    return math.sqrt(2.0 * math.log(1.0 / tol) / min_exp)


def _image_shifts(cell: np.ndarray, pbc: np.ndarray, rcut: float) -> np.ndarray:
    vol = abs(np.linalg.det(cell)) if np.all(pbc) else None
    nmax = []
    for d in range(3):
        if not pbc[d]:
            nmax.append(0)
            continue
        e, f = [x for x in range(3) if x != d]
        area = np.linalg.norm(np.cross(cell[e], cell[f]))
        height = abs(np.dot(cell[d], np.cross(cell[e], cell[f]))) / area
        nmax.append(int(math.ceil(rcut / height)))
    del vol
    rng = [np.arange(-n, n + 1) for n in nmax]
    g = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    return g.astype(np.int64)


class BsrRows:
    """Rows of the block-sparse S and H on demand: (i, j, R) pairs with a kept
    overlap entry, Wolfsberg-Helmholz H.  One KD-tree over the periodic images.

    When every atom carries the same exponents (all workloads here) the blocks of a
    row range are computed in one vectorised pass from per-exponent-pair tables
    (prefactor and decay of the Gaussian overlap), and the structure alone (which
    pairs are kept) needs only the block's largest entry, the most diffuse exponent
    with itself, except in a thin shell around the cutoff where the whole block is
    evaluated.  Other bases take a per-block loop."""

    def __init__(self, pos, cell, pbc, exps, onsite, drop_tol=DROP_TOL):
        from scipy.spatial import cKDTree

        self.pos, self.exps, self.onsite, self.drop_tol = pos, exps, onsite, drop_tol
        self.n = pos.shape[0]
        self.norb = np.array([len(e) for e in exps], dtype=np.int32)
        min_exp = min(float(np.min(e)) for e in exps)
        self.rcut = overlap_cutoff(min_exp, drop_tol)
        self.shifts = _image_shifts(cell, pbc, self.rcut)
        self.imgpos = (pos[None, :, :] + (self.shifts @ cell)[:, None, :]).reshape(-1, 3)
        self.tree = cKDTree(self.imgpos)
        e0 = np.asarray(exps[0], dtype=np.float64)
        self.tabled = all(len(e) == len(e0) and np.array_equal(e, e0) for e in exps)
        if self.tabled:
            a, b = e0[:, None], e0[None, :]
            p = a + b
            self.pref = (2.0 * np.sqrt(a * b) / p) ** 1.5  # gaussian_overlap's factors, per exponent pair
            self.decay = a * b / p
            k = int(np.argmin(e0))
            self.kmin = k  # the block's largest entry at every distance: pref 1, slowest decay
            self.onsite_tab = np.stack([np.asarray(h, dtype=np.float64) for h in onsite])

    def _candidates(self, i0, i1):
        """(row, col, shift, r2) of the images within the cutoff of rows i0 .. i1-1,
        sorted by (row, col, shift)."""
        lists = self.tree.query_ball_point(self.pos[i0:i1], self.rcut * (1 + 1e-12) + 1e-9)
        cnt = np.fromiter((len(x) for x in lists), dtype=np.int64, count=i1 - i0)
        idx = np.fromiter(itertools.chain.from_iterable(lists), dtype=np.int64, count=int(cnt.sum()))
        row = np.repeat(np.arange(i0, i1, dtype=np.int64), cnt)
        j = idx % self.n
        sh = self.shifts[idx // self.n]
        d = self.imgpos[idx] - self.pos[row]
        r2 = np.einsum("kd,kd->k", d, d)
        order = np.lexsort((sh[:, 2], sh[:, 1], sh[:, 0], j, row))
        return row[order], j[order], sh[order], r2[order]

    def _blocks(self, row, j, sh, r2):
        """S and H blocks (K, M, M) of tabled pairs, entries below drop_tol zeroed."""
        sblk = self.pref[None, :, :] * np.exp(-self.decay[None, :, :] * r2[:, None, None])
        sblk[sblk < self.drop_tol] = 0.0
        ea = self.onsite_tab[row][:, :, None]
        eb = self.onsite_tab[j][:, None, :]
        self_mask = (j == row) & np.all(sh == 0, axis=1)
        kfac = np.where(self_mask, 1.0, WH_K)[:, None, None]
        hblk = kfac * sblk * 0.5 * (ea + eb)
        return sblk, hblk

    def _kept(self, row, j, sh, r2):
        """Which candidate pairs keep a block: some entry >= drop_tol.  The diffuse
        entry decides away from the cutoff (>= 2 tol: kept; < tol / 2: every entry is
        below tol); in between the whole block is evaluated."""
        k = self.kmin
        smax = self.pref[k, k] * np.exp(-self.decay[k, k] * r2)
        keep = smax >= 2.0 * self.drop_tol
        edge = np.nonzero(~keep & (smax >= 0.5 * self.drop_tol))[0]
        if len(edge):
            sblk, _ = self._blocks(row[edge], j[edge], sh[edge], r2[edge])
            keep[edge] = np.any(sblk != 0.0, axis=(1, 2))
        return keep

    def rows(self, i0, i1):
        """[(col, shift, S, H)] of rows i0 .. i1-1, blocks sorted by (col, shift)."""
        if self.tabled:
            row, j, sh, r2 = self._candidates(i0, i1)
            sblk, hblk = self._blocks(row, j, sh, r2)
            keep = np.any(sblk != 0.0, axis=(1, 2))
            row, j, sh, sblk, hblk = row[keep], j[keep], sh[keep], sblk[keep], hblk[keep]
            bounds = np.searchsorted(row, np.arange(i0, i1 + 1))
            return [(j[b0:b1].astype(np.int32), sh[b0:b1].astype(np.int8), sblk[b0:b1].reshape(-1),
                     hblk[b0:b1].reshape(-1)) for b0, b1 in zip(bounds[:-1], bounds[1:])]
        n, pos, exps, onsite, drop_tol = self.n, self.pos, self.exps, self.onsite, self.drop_tol
        out = []
        lists = self.tree.query_ball_point(pos[i0:i1], self.rcut * (1 + 1e-12) + 1e-9)
        for ii, lst in enumerate(lists):  # ragged basis: per-block loop
            i = i0 + ii
            idx = np.asarray(sorted(lst), dtype=np.int64)
            j = idx % n
            sh = self.shifts[idx // n]
            d = self.imgpos[idx] - pos[i]
            r2 = np.einsum("kd,kd->k", d, d)
            blocks = []
            for k in range(len(idx)):
                jj = int(j[k])
                sb = gaussian_overlap(exps[i][:, None], exps[jj][None, :], r2[k])
                sb[sb < drop_tol] = 0.0
                if not np.any(sb != 0.0):
                    continue
                kf = 1.0 if (jj == i and not np.any(sh[k])) else WH_K
                hb = kf * sb * 0.5 * (onsite[i][:, None] + onsite[jj][None, :])
                blocks.append((jj, tuple(int(x) for x in sh[k]), sb, hb))
            blocks.sort(key=lambda t: (t[0],) + t[1])
            out.append((np.array([t[0] for t in blocks], dtype=np.int32),
                        np.array([t[1] for t in blocks], dtype=np.int8).reshape(-1, 3),
                        np.concatenate([t[2].reshape(-1) for t in blocks]),
                        np.concatenate([t[3].reshape(-1) for t in blocks])))
        return out

    def _structure_chunk(self, i0, i1):
        if not self.tabled:
            rows = self.rows(i0, i1)
            return [len(r[0]) for r in rows], [r[0] for r in rows], [r[1] for r in rows]
        row, j, sh, r2 = self._candidates(i0, i1)
        keep = self._kept(row, j, sh, r2)
        row, j, sh = row[keep], j[keep], sh[keep]
        ns = np.bincount(row - i0, minlength=i1 - i0)
        return list(ns), [j.astype(np.int32)], [sh.astype(np.int8)]

    def structure(self, chunk=256, workers=None):
        """row_ptr, col, shift, blk_off of all rows (the values are not kept); row
        ranges in parallel threads."""
        spans = [(i0, min(self.n, i0 + chunk)) for i0 in range(0, self.n, chunk)]
        with _pool(workers) as ex:
            parts = list(ex.map(lambda s: self._structure_chunk(*s), spans))
        ns = [x for p in parts for x in p[0]]
        cols = [c for p in parts for c in p[1]]
        shs = [s for p in parts for s in p[2]]
        return _layout(self.norb, ns, cols, shs)


def _nworkers(workers=None):
    import os

    return workers or min(32, os.cpu_count() or 1)


def _pool(workers=None):
    import concurrent.futures

    return concurrent.futures.ThreadPoolExecutor(max_workers=_nworkers(workers))


def _layout(norb, ns, cols, shs):
    n = len(ns)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(ns)
    col = np.concatenate(cols)
    shift = np.concatenate(shs).reshape(-1, 3)
    brow = np.repeat(np.arange(n), ns)
    sizes = norb[brow].astype(np.int64) * norb[col].astype(np.int64)
    blk_off = np.zeros(len(col), dtype=np.int64)
    blk_off[1:] = np.cumsum(sizes)[:-1]
    return row_ptr, col, shift, blk_off


def build_bsr(pos, cell, pbc, exps, onsite, drop_tol=DROP_TOL):
    """Block-sparse S and H over all (i, j, R) pairs with a kept overlap entry."""
    b = BsrRows(pos, cell, pbc, exps, onsite, drop_tol)
    rows = []
    for i0 in range(0, b.n, 256):
        rows += b.rows(i0, min(b.n, i0 + 256))
    row_ptr, col, shift, blk_off = _layout(b.norb, [len(r[0]) for r in rows], [r[0] for r in rows],
                                           [r[1] for r in rows])
    S = np.concatenate([r[2] for r in rows])
    H = np.concatenate([r[3] for r in rows])
    return b.norb, row_ptr, col, shift, blk_off, S, H


# --------------------------------------------------------------------------
# Geometries of the five workloads
# --------------------------------------------------------------------------

def _sc_lattice(nx, ny, nz, a):
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    return g.reshape(-1, 3).astype(np.float64) * a, g.reshape(-1, 3)


def make_system(cfg: int, seed: int | None = None, n_atoms: int | None = None, **over) -> System:
    """One of the five workloads (see workload_spec)."""
    return assemble_system(**workload_spec(cfg, seed, n_atoms, **over))


def make_system_streamed(cfg: int, seed: int | None = None, n_atoms: int | None = None, **over) -> System:
    """A workload's geometry and BSR structure with S and H not computed: both are
    full-length zero arrays (the operating system backs untouched pages lazily),
    ``source`` produces the blocks of any row range (BsrRows.rows) and fill_rows
    writes chosen rows.  For systems whose matrices do not fit host memory."""
    sp = workload_spec(cfg, seed, n_atoms, **over)
    pos = np.ascontiguousarray(sp["pos"], dtype=np.float64)
    exps = [np.asarray(e, dtype=np.float64) for e in sp["exps"]]
    onsite = [np.asarray(h, dtype=np.float64) for h in sp["onsite"]]
    src = BsrRows(pos, np.asarray(sp["cell"], dtype=np.float64), np.asarray(sp["pbc"], dtype=bool), exps, onsite)
    row_ptr, col, shift, blk_off = src.structure()
    last = len(col) - 1
    nval = int(blk_off[last] + src.norb[np.searchsorted(row_ptr, last, side="right") - 1] * src.norb[col[last]])
    return System(name=sp["name"], pos=pos, cell=np.asarray(sp["cell"], dtype=np.float64),
                  pbc=np.asarray(sp["pbc"], dtype=bool), species=np.asarray(sp["species"], np.int32), exps=exps,
                  onsite=onsite, norb=src.norb, row_ptr=row_ptr, col=col, shift=shift, blk_off=blk_off,
                  S=np.zeros(nval), H=np.zeros(nval), n_electrons=float(sp["n_electrons"]), kT=float(sp["kT"]),
                  r_core=float(sp["r_core"]), r_lno=float(sp["r_lno"]), k_lno=int(sp["k_lno"]), source=src)


def row_values(system: System, i0: int, i1: int):
    """(offset, S, H) of the blocks of rows i0 .. i1-1 of a streamed system."""
    src = system.source
    if src.tabled:
        row, j, sh, r2 = src._candidates(i0, i1)
        sblk, hblk = src._blocks(row, j, sh, r2)
        keep = np.any(sblk != 0.0, axis=(1, 2))
        sv, hv = sblk[keep].reshape(-1), hblk[keep].reshape(-1)
    else:
        rows = src.rows(i0, i1)
        sv, hv = np.concatenate([r[2] for r in rows]), np.concatenate([r[3] for r in rows])
    o0 = int(system.blk_off[system.row_ptr[i0]])
    o1 = int(system.blk_off[system.row_ptr[i1]]) if i1 < system.natoms else len(system.S)
    if len(sv) != o1 - o0:
        raise RuntimeError(f"rows {i0}..{i1}: {len(sv)} values against {o1 - o0} in the structure")
    return o0, sv, hv


def row_chunks(system: System, chunk: int = 128, workers=None, density_seed=None):
    """(i0, i1, offset, S, H[, rho]) of consecutive row ranges of a streamed system,
    in order, computed by a pool of threads a few ranges ahead of the consumer; with
    density_seed the synthetic_density blocks of the same rows come along."""
    import collections

    def job(i0):
        i1 = min(system.natoms, i0 + chunk)
        o0, sv, hv = row_values(system, i0, i1)
        if density_seed is None:
            return i0, i1, o0, sv, hv
        rv = np.empty(len(sv))
        synthetic_density_rows(system, i0, i1, rv, seed=density_seed, base=o0)
        return i0, i1, o0, sv, hv, rv

    with _pool(workers) as ex:
        depth = 2 * _nworkers(workers)
        starts = iter(range(0, system.natoms, chunk))
        pending = collections.deque(ex.submit(job, i0) for i0 in itertools.islice(starts, depth))
        while pending:
            res = pending.popleft().result()
            nxt = next(starts, None)
            if nxt is not None:
                pending.append(ex.submit(job, nxt))
            yield res


def fill_rows(system: System, atoms) -> None:
    """Compute the S and H blocks of the given rows of a streamed system in place."""
    for i in sorted(set(int(a) for a in atoms)):
        o0, sv, hv = row_values(system, i, i + 1)
        system.S[o0:o0 + len(sv)] = sv
        system.H[o0:o0 + len(hv)] = hv


def workload_spec(cfg: int, seed: int | None = None, n_atoms: int | None = None, **over) -> dict:
    """Geometry, basis and parameters of one of the five workloads; keyword
    overrides replace r_core, r_lno, k_lno.
    n_atoms (workload 5 only) packs fewer atoms at the same density (a smaller cube);
    n_cells (workload 2 only) sets the sites per edge of the periodic rock-salt cube.

    1  64-atom simple-cubic 4x4x4, a=2.5, open, 4 s-Gaussians, 2 e/atom.
    2  1,728-atom rock-salt arrangement on SC 12^3, a=3.0, periodic, jitter 0.05,
       9 s-Gaussians, 4.5 e/atom (the gapped FP64 workload).
    3  the same system as 2 (it differs only in the arithmetic precision).
    4  bcc slab 20x20x10 conventional cells, a=5.4, periodic in x and y,
       2% seeded vacancies, 9 s-Gaussians, 1 e/atom (metallic, uneven).
    5  32,000-atom random sequential packing in a periodic cube, two species.
    """
    if cfg == 1:
        pos, _ = _sc_lattice(4, 4, 4, 2.5)
        n = len(pos)
        e = np.array([0.2, 0.5, 1.2, 3.0])
        h = np.array([-0.5, -0.3, 0.1, 0.4])
        sys = dict(name="cfg1_sc64", pos=pos, cell=np.eye(3) * 10.0,
                   pbc=np.zeros(3, bool), species=np.zeros(n, np.int32),
                   exps=[e.copy() for _ in range(n)], onsite=[h.copy() for _ in range(n)],
                   n_electrons=2.0 * n, kT=0.01, r_core=5.0, r_lno=8.0, k_lno=2)
    elif cfg in (2, 3):
        rng = np.random.default_rng(1001 if seed is None else seed)
        nc = int(over.pop("n_cells", 12))  # sites per edge (12 in the recipe; even keeps the rock-salt order)
        pos, ijk = _sc_lattice(nc, nc, nc, 3.0)
        pos = pos + rng.normal(0.0, 0.05, size=pos.shape)
        n = len(pos)
        species = (ijk.sum(1) % 2).astype(np.int32)  # 0 = A (even x+y+z), 1 = B
        e = np.geomspace(0.1, 5.0, 9)
        base = np.linspace(-0.6, 0.5, 9)
        onsite = [base + (-0.3 if s == 0 else 0.3) for s in species]
        sys = dict(name=f"cfg2_rocksalt{n}", pos=pos, cell=np.eye(3) * (3.0 * nc),
                   pbc=np.ones(3, bool), species=species,
                   exps=[e.copy() for _ in range(n)], onsite=onsite,
                   n_electrons=4.5 * n, kT=0.01, r_core=6.0, r_lno=10.0, k_lno=3)
    elif cfg == 4:
        rng = np.random.default_rng(1004 if seed is None else seed)
        a = 5.4
        g, _ = _sc_lattice(20, 20, 10, a)
        pos = np.concatenate([g, g + 0.5 * a]).astype(np.float64)
        order = np.lexsort((pos[:, 2], pos[:, 1], pos[:, 0]))
        pos = pos[order]
        vac = rng.choice(len(pos), size=int(round(0.02 * len(pos))), replace=False)
        pos = np.delete(pos, np.sort(vac), axis=0)
        n = len(pos)
        e = np.geomspace(0.1, 5.0, 9)
        h = np.linspace(-0.4, 0.6, 9)
        cell = np.diag([20 * a, 20 * a, 10 * a + 60.0])
        sys = dict(name="cfg4_bccslab", pos=pos, cell=cell,
                   pbc=np.array([True, True, False]), species=np.zeros(n, np.int32),
                   exps=[e.copy() for _ in range(n)], onsite=[h.copy() for _ in range(n)],
                   n_electrons=1.0 * n, kT=0.005, r_core=6.0, r_lno=11.0, k_lno=3)
    elif cfg == 5:
        rng = np.random.default_rng(1005 if seed is None else seed)
        n = 32000 if n_atoms is None else int(n_atoms)
        L = (n / 0.012) ** (1.0 / 3.0)
        pos = _rsa(n, L, 3.8, rng)
        species = np.zeros(n, np.int32)
        species[rng.permutation(n)[: n // 2]] = 1
        e = np.geomspace(0.08, 6.0, 13)
        base = np.linspace(-0.6, 0.5, 13)
        onsite = [base + (-0.15 if s == 0 else 0.15) for s in species]
        sys = dict(name=f"cfg5_rsa{n}", pos=pos, cell=np.eye(3) * L,
                   pbc=np.ones(3, bool), species=species,
                   exps=[e.copy() for _ in range(n)], onsite=onsite,
                   n_electrons=5.0 * n, kT=0.01, r_core=6.0, r_lno=10.0, k_lno=4)
    else:
        raise ValueError(f"unknown workload {cfg}")
    sys.update(over)
    return sys


def assemble_system(name, pos, cell, pbc, species, exps, onsite, n_electrons, kT,
                    r_core, r_lno, k_lno) -> System:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    pbc = np.asarray(pbc, dtype=bool)
    exps = [np.asarray(e, dtype=np.float64) for e in exps]
    onsite = [np.asarray(h, dtype=np.float64) for h in onsite]
    norb, row_ptr, col, shift, blk_off, S, H = build_bsr(pos, cell, pbc, exps, onsite)
    return System(name=name, pos=pos, cell=cell, pbc=pbc,
                  species=np.asarray(species, np.int32), exps=exps, onsite=onsite,
                  norb=norb, row_ptr=row_ptr, col=col, shift=shift, blk_off=blk_off,
                  S=S, H=H, n_electrons=float(n_electrons), kT=float(kT),
                  r_core=float(r_core), r_lno=float(r_lno), k_lno=int(k_lno))


def _rsa(n, L, dmin, rng, batch=65536):
    """Random sequential addition in a periodic cube with a minimum distance.

    Candidates are drawn uniformly in batches and considered in draw order; a
    candidate is kept when no point kept before it lies within dmin under the
    minimum-image convention and its cell of a grid of width >= dmin / sqrt(3) holds
    no kept point (one point per cell, so every conflict lies within
    ceil(dmin / width) cells).  Within a batch, the candidates free of the points of
    earlier batches are resolved in draw order over their conflict graph (pairs
    closer than dmin or sharing a cell).
    """
    from scipy.spatial import cKDTree

    g = max(1, int(L / (dmin / np.sqrt(3.0))))
    cw = L / g
    reach = int(np.ceil(dmin / cw))
    occ = -np.ones((g, g, g), dtype=np.int64)
    pts = np.empty((n, 3))
    off = np.array([(a, b, c) for a in range(-reach, reach + 1) for b in range(-reach, reach + 1)
                    for c in range(-reach, reach + 1)], dtype=np.int64)
    k = 0
    tries = 0
    while k < n:
        if tries > 20000 * n:
            raise RuntimeError("random sequential addition jammed")
        cand = rng.uniform(0.0, L, size=(batch, 3))
        tries += batch
        cell = np.minimum((cand // cw).astype(np.int64), g - 1)
        ok = occ[cell[:, 0], cell[:, 1], cell[:, 2]] < 0
        if k:
            # nearest earlier point by a KD-tree; the exact minimum-image test near dmin
            near = cKDTree(np.mod(pts[:k], L), boxsize=L).query(np.mod(cand, L), k=1,
                                                                   distance_upper_bound=dmin * (1 + 1e-6))[0]
            ok &= near >= dmin * (1 - 1e-6)
            edge = np.nonzero(ok & (near < dmin * (1 + 1e-6)))[0]
            if len(edge):
                nb = (cell[edge][:, None, :] + off[None, :, :]) % g
                who = occ[nb[..., 0], nb[..., 1], nb[..., 2]]
                d = pts[np.maximum(who, 0)] - cand[edge][:, None, :]
                d -= L * np.round(d / L)
                ok[edge] = ~((who >= 0) & (np.einsum("bkd,bkd->bk", d, d) < dmin * dmin)).any(axis=1)
        free = np.nonzero(ok)[0]
        if len(free) == 0:
            continue
        # conflicts among the free candidates: same cell, or closer than dmin
        fp = cand[free]
        pairs = cKDTree(np.mod(fp, L), boxsize=L).query_pairs(max(dmin, cw * np.sqrt(3.0)) * (1 + 1e-9),
                                                              output_type="ndarray")
        if len(pairs):
            pairs.sort(axis=1)  # (earlier, later) in draw order
            a, b = pairs[:, 0], pairs[:, 1]
            dd = fp[a] - fp[b]
            dd -= L * np.round(dd / L)
            hit = np.all(cell[free[a]] == cell[free[b]], axis=1) | (np.einsum("kd,kd->k", dd, dd) < dmin * dmin)
            a, b = a[hit], b[hit]
            order = np.argsort(b, kind="stable")
            a, b = a[order], b[order]
            starts = np.searchsorted(b, np.arange(len(free) + 1))
        else:
            a = np.zeros(0, dtype=np.int64)
            starts = np.zeros(len(free) + 1, dtype=np.int64)
        kept = np.zeros(len(free), dtype=bool)
        al = a.tolist()
        st = starts.tolist()
        for f in range(len(free)):
            if any(kept[x] for x in al[st[f]:st[f + 1]]):
                continue
            kept[f] = True
            c = cell[free[f]]
            pts[k] = cand[free[f]]
            occ[c[0], c[1], c[2]] = k
            k += 1
            if k == n:
                break
    return pts


def small_lattice(nx, ny, nz, a=2.5, jitter=0.0, seed=7, exps=(0.2, 0.5, 1.2, 3.0),
                  onsite=(-0.5, -0.3, 0.1, 0.4), e_per_atom=2.0, kT=0.01,
                  r_core=5.0, r_lno=8.0, k_lno=2, periodic=False, name=None) -> System:
    """A small open (or periodic) simple-cubic lattice for tests."""
    pos, _ = _sc_lattice(nx, ny, nz, a)
    if jitter:
        pos = pos + np.random.default_rng(seed).normal(0.0, jitter, size=pos.shape)
    n = len(pos)
    if periodic:
        cell, pbc = np.diag([nx * a, ny * a, nz * a]), np.ones(3, bool)
    else:
        cell, pbc = np.eye(3) * (max(nx, ny, nz) * a + 10.0), np.zeros(3, bool)
    return assemble_system(name or f"sc{nx}x{ny}x{nz}", pos, cell, pbc, np.zeros(n, np.int32),
                           [np.array(exps, float)] * n, [np.array(onsite, float)] * n,
                           e_per_atom * n, kT, r_core, r_lno, k_lno)


def synthetic_density(system: System, seed: int = 11, width: float = 3.0) -> np.ndarray:
    """A seeded, symmetric density-like matrix in the BSR pattern of S.

    It stands in for the density matrix of the previous SCF step when a test
    runs one LNO step on a system too large for the oracle to converge.  The
    on-site block is diag(p) with populations p_a = 0.9 exp(-0.6 a) times a
    seeded per-atom factor in [0.9, 1.1]; an off-site block is
    0.05 exp(-d^2/width^2) sqrt(s_i s_j) w_a w_b with w_a = exp(-0.4 a).
    Symmetry rho_{0i,Rj} = rho_{0j,-Ri}^T holds by construction.  Only the
    pattern and the geometry are read from ``system``.
    """
    rho = np.zeros_like(system.S)
    synthetic_density_rows(system, 0, system.natoms, rho, seed, width)
    return rho


def synthetic_density_rows(system: System, i0: int, i1: int, out: np.ndarray, seed: int = 11,
                           width: float = 3.0, base: int = 0) -> None:
    """The blocks of rows i0 .. i1-1 of synthetic_density, written to out[blk_off - base]."""
    rng = np.random.default_rng(seed)
    n = system.natoms
    scale = rng.uniform(0.9, 1.1, size=n)
    b0, b1 = int(system.row_ptr[i0]), int(system.row_ptr[i1])
    brow = np.repeat(np.arange(i0, i1), np.diff(system.row_ptr[i0:i1 + 1]))
    col = system.col[b0:b1].astype(np.int64)
    shift = system.shift[b0:b1]
    d = system.pos[col] + shift.astype(np.float64) @ system.cell - system.pos[brow]
    r2 = np.einsum("kd,kd->k", d, d)
    onsite = (brow == col) & ~np.any(shift != 0, axis=1)
    amp = 0.05 * np.exp(-r2 / (width * width)) * np.sqrt(scale[brow] * scale[col])
    mi_all = system.norb[brow].astype(np.int64)
    mj_all = system.norb[col].astype(np.int64)
    offs = system.blk_off[b0:b1] - base
    for mi in np.unique(mi_all):
        for mj in np.unique(mj_all):
            sel = np.nonzero((mi_all == mi) & (mj_all == mj))[0]
            if len(sel) == 0:
                continue
            wi = np.exp(-0.4 * np.arange(mi))
            wj = np.exp(-0.4 * np.arange(mj))
            blocks = amp[sel, None, None] * np.outer(wi, wj)[None, :, :]
            ons = onsite[sel]
            if np.any(ons):
                p = 0.9 * np.exp(-0.6 * np.arange(mi))
                blocks[ons] = np.diag(p)[None, :, :] * scale[brow[sel[ons]], None, None]
            idx = offs[sel][:, None] + np.arange(mi * mj)[None, :]
            out[idx] = blocks.reshape(len(sel), -1)


def known_pencils(count: int, n: int, seed: int = 5, cond_s: float = 100.0):
    """`count` symmetric pencils (H, S) of dimension n whose eigenpairs are known by
    construction: S = U diag(s) U^T with s geometric over [0.5, 0.5 cond_s], C = U
    diag(s^-1/2) V (so C^T S C = I), H = S C diag(w) C^T S (so H C = S C diag(w)),
    eigenvalues w ascending over [-2, 2] (spacing 4/(n-1), each jittered by under a
    quarter of it, so neighbours are at least half the spacing apart).
    U, V are orthogonal factors of seeded Gaussian matrices.  Returns H, S, C as
    [count, n, n] and w as [count, n], all float64."""
    rng = np.random.default_rng(seed)
    H = np.empty((count, n, n))
    S = np.empty((count, n, n))
    C = np.empty((count, n, n))
    w = np.empty((count, n))
    s = np.geomspace(0.5, 0.5 * cond_s, n)
    step = 4.0 / max(n - 1, 1)
    for p in range(count):
        U = np.linalg.qr(rng.standard_normal((n, n)))[0]
        V = np.linalg.qr(rng.standard_normal((n, n)))[0]
        Sp = (U * s) @ U.T
        Cp = (U / np.sqrt(s)) @ V
        wp = np.linspace(-2.0, 2.0, n) + 0.25 * step * rng.uniform(-1.0, 1.0, n) if n > 1 else np.zeros(1)
        SC = Sp @ Cp
        Hp = (SC * wp) @ SC.T
        H[p] = 0.5 * (Hp + Hp.T)
        S[p] = 0.5 * (Sp + Sp.T)
        C[p] = Cp
        w[p] = wp
    return H, S, C, w
