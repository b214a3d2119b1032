"""Seeded synthetic tight-binding matrix pairs (A, B) shaped like the paper's workloads.

The paper measures on ELSES matrices (Section 4.1, Table "Matrix data"): real symmetric A and
symmetric positive definite B that share one sparsity pattern and come from a transferable
tight-binding model with atom-centred, non-orthogonal orbitals (Appendix A, Eq. A.2). Those files are
not available here, so this module builds stand-ins with the same structure: a periodic carbon
diamond lattice, four sp3 orbitals (s, px, py, pz) per atom, 4x4 Slater-Koster hopping blocks
between atoms closer than a cutoff, and an overlap matrix B = I + S on the same pattern.

This module holds input construction only: no step of the eigenvalue method lives here, so the
oracle and the GPU path can both draw their inputs from it without sharing method arithmetic.

Random streams: every random draw comes from ``numpy.random.default_rng([seed, stream])`` with a
fixed stream number per purpose (positions, onsite energies, vacancies), so changing one knob does
not reshuffle the others.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

DIAMOND_A = 3.567  # lattice constant (Angstrom); the paper gives none, this one puts the
# first (1.545 A) and second (2.522 A) neighbour shells inside a 2.9 A cutoff.

# Slater-Koster two-centre amplitudes (eV) multiplied by exp(-r / 1 A).
V_SSS, V_SPS, V_PPS, V_PPP = -5.0, 5.0, 6.0, -3.0
ONSITE_S, ONSITE_P = -5.0, 1.0

_STREAM_POS, _STREAM_ONSITE, _STREAM_VAC, _STREAM_PHASE = 1, 2, 3, 4

# Fractional positions of the 8 atoms of the conventional diamond cell.
_BASIS = np.array([
    [0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


@dataclass
class Pencil:
    """A symmetric (or, with complex values, Hermitian) pencil (A, B) in CSR form (both triangles
    stored, sorted columns)."""
    n: int
    rowptr: np.ndarray      # int64, n+1
    colind: np.ndarray      # int32, nnz
    a: np.ndarray           # float64 (complex128 for a Hermitian pencil), nnz
    b: np.ndarray           # same dtype as a, nnz
    coords: np.ndarray | None = None   # float64 (n, 3): position of the atom owning each row
    box: np.ndarray | None = None      # float64 (3,): periodic box lengths
    k: int = 0                          # target index (1-based)
    meta: dict = field(default_factory=dict)

    def A(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.a, self.colind, self.rowptr), shape=(self.n, self.n))

    def B(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.b, self.colind, self.rowptr), shape=(self.n, self.n))

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def diamond_sites(nx: int, ny: int, nz: int, a: float = DIAMOND_A):
    """Atom positions of an nx x ny x nz block of conventional diamond cells, and the box."""
    cells = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    cells = cells.reshape(-1, 3).astype(np.float64)
    pos = (cells[:, None, :] + _BASIS[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx, ny, nz], dtype=np.float64) * a
    return pos, box


def _min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    return d - box * np.round(d / box)


def neighbour_pairs(pos: np.ndarray, box: np.ndarray, cutoff: float):
    """All pairs i < j with periodic minimum-image distance < cutoff (cell-list search).

    Returns (i, j, dvec) with dvec = r_j - r_i (minimum image)."""
    natom = pos.shape[0]
    nbin = np.floor(box / cutoff).astype(np.int64)
    if natom <= 3000 or np.any(nbin < 3):
        ii, jj = np.triu_indices(natom, 1)
        d = _min_image(pos[jj] - pos[ii], box)
        r = np.sqrt((d * d).sum(1))
        keep = r < cutoff
        return ii[keep].astype(np.int64), jj[keep].astype(np.int64), d[keep]
    b3 = np.floor(pos / (box / nbin)).astype(np.int64) % nbin
    bid = (b3[:, 0] * nbin[1] + b3[:, 1]) * nbin[2] + b3[:, 2]
    order = np.argsort(bid, kind="stable")
    nb_tot = int(nbin.prod())
    counts = np.bincount(bid, minlength=nb_tot)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    maxc = int(counts.max())
    out_i, out_j, out_d = [], [], []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for oz in (-1, 0, 1):
                nb3 = (b3 + np.array([ox, oy, oz])) % nbin
                nbid = (nb3[:, 0] * nbin[1] + nb3[:, 1]) * nbin[2] + nb3[:, 2]
                st, ct = starts[nbid], counts[nbid]
                for s in range(maxc):
                    sel = np.nonzero(s < ct)[0]
                    j = order[st[sel] + s]
                    i = sel
                    m = i < j
                    i, j = i[m], j[m]
                    d = _min_image(pos[j] - pos[i], box)
                    r = np.sqrt((d * d).sum(1))
                    keep = r < cutoff
                    out_i.append(i[keep]); out_j.append(j[keep]); out_d.append(d[keep])
    i = np.concatenate(out_i); j = np.concatenate(out_j); d = np.concatenate(out_d)
    # a pair can be met through two bin offsets only when a box side has < 3 bins (excluded above)
    return i.astype(np.int64), j.astype(np.int64), d


def sk_blocks(dvec: np.ndarray) -> np.ndarray:
    """4x4 Slater-Koster sp3 hopping blocks for displacement vectors dvec (r_j - r_i).

    Orbital order (s, px, py, pz); textbook two-centre forms with direction cosines, every
    amplitude scaled by exp(-r)."""
    r = np.sqrt((dvec * dvec).sum(1))
    c = dvec / r[:, None]
    f = np.exp(-r)
    npair = dvec.shape[0]
    h = np.empty((npair, 4, 4))
    h[:, 0, 0] = V_SSS * f
    h[:, 0, 1:] = c * (V_SPS * f)[:, None]
    h[:, 1:, 0] = -c * (V_SPS * f)[:, None]
    pp = c[:, :, None] * c[:, None, :] * (V_PPS - V_PPP)
    pp += np.eye(3)[None] * V_PPP
    h[:, 1:, 1:] = pp * f[:, None, None]
    return h


def _assemble(natom, ii, jj, hblk, sblk, onsite, sdiag):
    """CSR (both triangles) from atom-pair blocks (i < j) and per-orbital diagonals; the mirrored
    block (j, i) holds the complex conjugate of block (i, j) transposed (plain transpose when real)."""
    n = 4 * natom
    oa = np.arange(4)
    # off-diagonal blocks (i, j) and mirrored (j, i)
    rows = (4 * ii[:, None, None] + oa[None, :, None]) + 0 * oa[None, None, :]
    cols = (4 * jj[:, None, None] + oa[None, None, :]) + 0 * oa[None, :, None]
    r_all = np.concatenate([rows.ravel(), cols.ravel(), np.arange(n)])
    c_all = np.concatenate([cols.ravel(), rows.ravel(), np.arange(n)])
    a_all = np.concatenate([hblk.ravel(), np.conj(hblk).ravel(), onsite])
    b_all = np.concatenate([sblk.ravel(), np.conj(sblk).ravel(), sdiag])
    # the same pattern for A and B: sort by (row, col) once
    key = r_all * n + c_all
    o = np.argsort(key, kind="stable")
    r_all, c_all, a_all, b_all = r_all[o], c_all[o], a_all[o], b_all[o]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r_all + 1, 1)
    rowptr = np.cumsum(rowptr)
    return n, rowptr, c_all.astype(np.int32), a_all, b_all


def make_pair(nx: int, ny: int, nz: int, *, seed: int = 0, jitter: float = 0.05,
              vacancies: int = 0, cutoff: float = 2.9, overlap: float = 0.1,
              onsite_noise: float = 0.1, max_offdiag_rowsum: float = 0.9, phases=None) -> Pencil:
    """Tight-binding pencil on an nx x ny x nz block of periodic conventional diamond cells.

    * positions: lattice sites, `vacancies` sites removed uniformly at random, then each
      coordinate jittered by N(0, jitter) and wrapped into the box;
    * A: onsite s = -5 eV, p = +1 eV, each plus N(0, onsite_noise); hopping blocks from
      `sk_blocks` for every atom pair closer than `cutoff` (minimum image);
    * B = I + S, S = -overlap * (hopping blocks), scaled down if needed so that every
      off-diagonal row sum of |B| is <= max_offdiag_rowsum (strict diagonal dominance, so B is SPD).
      The scale actually applied is in meta["overlap_scale"].
    * phases (a Hermitian pencil, complex128 values): "peierls" multiplies the hopping and overlap
      blocks of each atom pair (i < j) by e^{i theta_ij}, theta_ij ~ U(-pi, pi) drawn per pair
      (block (j, i) gets e^{-i theta_ij}); an array of per-atom phases phi gives the pure gauge
      theta_ij = phi_i - phi_j, whose spectrum equals that of the real pencil.  The magnitudes and
      the pattern are those of the real pencil of the same seed.
    k = n/2 (the highest occupied state of a half-filled sp3 band, Appendix B).
    """
    pos, box = diamond_sites(nx, ny, nz)
    rng_vac = np.random.default_rng([seed, _STREAM_VAC])
    if vacancies:
        keep = np.sort(rng_vac.choice(pos.shape[0], pos.shape[0] - vacancies, replace=False))
        pos = pos[keep]
    natom = pos.shape[0]
    rng_pos = np.random.default_rng([seed, _STREAM_POS])
    if jitter:
        pos = np.mod(pos + rng_pos.normal(0.0, jitter, pos.shape), box)
    ii, jj, d = neighbour_pairs(pos, box, cutoff)
    h = sk_blocks(d)
    rng_on = np.random.default_rng([seed, _STREAM_ONSITE])
    onsite = np.tile(np.array([ONSITE_S, ONSITE_P, ONSITE_P, ONSITE_P]), natom)
    if onsite_noise:
        onsite = onsite + rng_on.normal(0.0, onsite_noise, onsite.shape)
    s = -overlap * h
    # strict diagonal dominance of B = I + S
    rowsum = np.zeros(4 * natom)
    np.add.at(rowsum, (4 * ii[:, None] + np.arange(4)[None, :]).ravel(), np.abs(s).sum(2).ravel())
    np.add.at(rowsum, (4 * jj[:, None] + np.arange(4)[None, :]).ravel(), np.abs(s).sum(1).ravel())
    rho = float(rowsum.max()) if rowsum.size else 0.0
    scale = 1.0 if rho < max_offdiag_rowsum else max_offdiag_rowsum / rho
    s = s * scale
    if phases is not None:
        if isinstance(phases, str):
            if phases != "peierls":
                raise ValueError("phases: 'peierls' or an array of per-atom phases")
            theta = np.random.default_rng([seed, _STREAM_PHASE]).uniform(-np.pi, np.pi, ii.size)
        else:
            phi = np.asarray(phases, dtype=np.float64)
            if phi.shape != (natom,):
                raise ValueError("per-atom phases must have one value per atom")
            theta = phi[ii] - phi[jj]
        ph = np.exp(1j * theta)[:, None, None]
        h = h * ph
        s = s * ph
    n, rowptr, colind, a, b = _assemble(natom, ii, jj, h, s, onsite, np.ones(4 * natom))
    coords = np.repeat(pos, 4, axis=0)
    return Pencil(n=n, rowptr=rowptr, colind=colind, a=a, b=b, coords=coords, box=box, k=n // 2,
                  meta=dict(kind="diamond", cells=(nx, ny, nz), seed=seed, jitter=jitter,
                            vacancies=vacancies, cutoff=cutoff, overlap_scale=scale,
                            phases=None if phases is None else (phases if isinstance(phases, str) else "gauge"),
                            natom=natom, npairs=int(ii.size)))


def perfect_diamond_pencil(nx: int, ny: int, nz: int, *, beta: float = 1.0, gamma: float = 0.02,
                           cutoff: float = 2.9) -> Pencil:
    """Unjittered periodic diamond lattice, noise-free onsite energies, and B = beta*I + gamma*A.

    A and B commute and share eigenvectors, so the pencil's eigenvalues are mu/(beta + gamma*mu)
    for the eigenvalues mu of A; those follow from 32x32 Bloch matrices (see oracle.closed_forms)
    at any size. B is SPD when beta + gamma*mu > 0 for every mu."""
    p = make_pair(nx, ny, nz, seed=0, jitter=0.0, onsite_noise=0.0, cutoff=cutoff)
    A = p.A().tocsr()
    B = (beta * sp.identity(p.n, format="csr") + gamma * A).tocsr()
    B.sort_indices(); A.sort_indices()
    # B's pattern equals A's (A has a full diagonal), keep A's index arrays
    bvals = _values_on_pattern(B, p.rowptr, p.colind)
    return Pencil(n=p.n, rowptr=p.rowptr, colind=p.colind, a=p.a.copy(), b=bvals, coords=p.coords,
                  box=p.box, k=p.n // 2,
                  meta=dict(kind="perfect_diamond", cells=(nx, ny, nz), beta=beta, gamma=gamma,
                            cutoff=cutoff))


def sband_cubic_pencil(l1: int, l2: int, l3: int, *, eps: float = 0.0, t: float = -1.0,
                       beta: float = 1.0, gamma: float = 0.05) -> Pencil:
    """Periodic simple-cubic s-band: A = eps*I + t*(adjacency), B = beta*I + gamma*A.

    n = l1*l2*l3 (each l >= 3). A's eigenvalues are eps + 2t*sum_d cos(2*pi*m_d/l_d); the
    pencil's are mu/(beta + gamma*mu)."""
    n = l1 * l2 * l3
    idx = np.arange(n).reshape(l1, l2, l3)
    rows, cols = [np.arange(n)], [np.arange(n)]
    vals = [np.full(n, eps)]
    for axis in range(3):
        nb = np.roll(idx, -1, axis=axis).ravel()
        rows += [idx.ravel(), nb]
        cols += [nb, idx.ravel()]
        vals += [np.full(n, t), np.full(n, t)]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sum_duplicates(); A.sort_indices()
    B = (beta * sp.identity(n, format="csr") + gamma * A).tocsr()
    B.sort_indices()
    rowptr = A.indptr.astype(np.int64)
    colind = A.indices.astype(np.int32)
    bvals = _values_on_pattern(B, rowptr, colind)
    g = np.stack(np.meshgrid(np.arange(l1), np.arange(l2), np.arange(l3), indexing="ij"), -1)
    coords = g.reshape(-1, 3).astype(np.float64)
    return Pencil(n=n, rowptr=rowptr, colind=colind, a=A.data.astype(np.float64), b=bvals,
                  coords=coords, box=np.array([l1, l2, l3], dtype=np.float64), k=n // 2,
                  meta=dict(kind="sband", dims=(l1, l2, l3), eps=eps, t=t, beta=beta, gamma=gamma))


def diagonal_pencil(a_diag: np.ndarray, b_diag: np.ndarray) -> Pencil:
    """Diagonal pencil: eigenvalues a_ii / b_ii."""
    n = a_diag.size
    return Pencil(n=n, rowptr=np.arange(n + 1, dtype=np.int64), colind=np.arange(n, dtype=np.int32),
                  a=np.asarray(a_diag, np.float64).copy(), b=np.asarray(b_diag, np.float64).copy(),
                  k=max(1, n // 2), meta=dict(kind="diagonal"))


def _values_on_pattern(M: sp.csr_matrix, rowptr: np.ndarray, colind: np.ndarray) -> np.ndarray:
    """Values of M at the (row, col) positions of the given CSR pattern (0 where M has none)."""
    n = rowptr.size - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return np.asarray(M[rows, colind]).ravel().astype(np.float64)


# Named workloads (the configurations the paper's experiments are shaped like).
def workload(name: str, seed: int = 0) -> Pencil:
    """Named synthetic workloads.

    * ``small``:    4x4x4 cells, 512 atoms, n = 2,048, jitter 0.05 A.
    * ``scale``:    32x32x18 cells (147,456 sites) with 16,384 random vacancies (11.1 %),
                    131,072 atoms, n = 524,288, jitter 0.05 A.
    * ``mid``:      12x12x12 cells with 10 % vacancies (n = 49,768) for mid-size checks.
    * ``million``:  32x32x32 cells, 262,144 atoms, n = 1,048,576.
    * ``mid_peierls``: the ``mid`` pencil with a Peierls phase e^{i theta}, theta ~ U(-pi, pi), on
                    every atom pair (complex Hermitian, n = 49,768).
    * ``scale_peierls``: the ``scale`` pencil with Peierls phases (complex Hermitian, n = 524,288,
                    the differentiation workload).
    * ``batch``:    32x16x16 cells, 65,536 atoms, n = 262,144 (the multisection workload).
    * ``precision``: 25x25x75 cells (the most nearly cubic periodic block with exactly 375,000
                    atoms), amorphous-like jitter 0.3 A, n = 1,500,000, k = 0.3 n (the
                    mixed-precision workload).
    """
    if name == "small":
        return make_pair(4, 4, 4, seed=seed)
    if name == "scale":
        return make_pair(32, 32, 18, seed=seed, vacancies=16384)
    if name == "mid":
        return make_pair(12, 12, 12, seed=seed, vacancies=1382)
    if name == "mid_peierls":
        return make_pair(12, 12, 12, seed=seed, vacancies=1382, phases="peierls")
    if name == "million":
        return make_pair(32, 32, 32, seed=seed)
    if name == "scale_peierls":
        return make_pair(32, 32, 18, seed=seed, vacancies=16384, phases="peierls")
    if name == "batch":
        return make_pair(32, 16, 16, seed=seed)
    if name == "precision":
        p = make_pair(25, 25, 75, seed=seed, jitter=0.3)
        p.k = (3 * p.n) // 10
        return p
    if name.startswith("cells:"):
        nx, ny, nz = (int(v) for v in name[6:].split("x"))
        return make_pair(nx, ny, nz, seed=seed)
    raise ValueError(f"unknown workload {name!r}")
