"""Oracle core (test infrastructure only): inertia, dense generalized eigenpairs, closed forms.

Routes (each pinned in tests/test_oracle_core.py against something other than itself):

* ``dense_bk``            (c1) Bunch-Kaufman LDL^T of a dense symmetric matrix (C, orc.c).
                          Pins: Jacobi's sign-change rule on leading minors computed by brute-force
                          permutation expansion (n <= 6); diagonal matrices; 2x2-pivot-forcing
                          matrices with known spectra; reconstruction P M P^T = L D L^T; the
                          closed-form lattice spectra below; counts from numpy's eigvalsh.
* ``sparse_inertia``      (c3) plain multifrontal LDL^T with its own nested dissection (C, orc.c).
                          Pins: equality with (c1) on many pencils (Sylvester's law, Section 2.1);
                          closed-form lattice spectra at sizes (c1) cannot reach.
* ``gen_eig``             (c2) B = L L^T, C = L^{-1} A L^{-T}, C = Y diag(lam) Y^T, X = L^{-T} Y:
                          the Cholesky reduction the paper's dense comparison uses (LAPACK dsygvd,
                          Section 4.2).  Library routines (Cholesky, triangular solve, symmetric
                          eigensolver) serve as steps.  Pins: closed-form spectra; residual and
                          B-orthonormality of the returned vectors.
* ``eig_grad``            derivatives of lambda_k with respect to the entries of A and B from the
                          (c2) eigenvector (Hellmann-Feynman).  Pins: central finite differences of
                          lambda_k under symmetric perturbations of single entries.
* ``sband_eigs`` / ``diamond_bloch_eigs`` / diagonal: closed-form pencil spectra.
                          Pins: the s-band formula against a brute-force dense eigensolve at tiny
                          sizes; the Bloch spectrum likewise.

Conventions (Section 2.1): nu(sigma) = #{i : lambda_i < sigma}; k is 1-based.
"""
from __future__ import annotations

import ctypes
import itertools
import math

import numpy as np
import scipy.linalg as sla

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.orc_dense_bk.argtypes = [ctypes.c_int64, P, P, P, P, P, P]
        lib.orc_dense_bk.restype = None
        lib.orc_sparse_inertia.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int64, ctypes.c_double, P]
        lib.orc_sparse_inertia.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------------------------------
# (c1) dense Bunch-Kaufman
# ------------------------------------------------------------------------------------------
class DenseBK:
    """Result of (c1): P M P^T = L D L^T with D block diagonal (1x1 / 2x2)."""

    def __init__(self, L, d, e, piv, perm, inertia):
        self.L, self.d, self.e, self.piv, self.perm = L, d, e, piv, perm
        self.neg, self.zero, self.pos, self.n2x2 = inertia

    def D(self) -> np.ndarray:
        n = self.d.size
        D = np.diag(self.d.copy())
        for k in range(n):
            if self.piv[k] == 2:
                D[k + 1, k] = D[k, k + 1] = self.e[k]
        return D


def dense_bk(M: np.ndarray) -> DenseBK:
    """(c1) Bunch-Kaufman factorization of the dense symmetric M (lower triangle read).

    Follows the partial-pivoting strategy of Bunch and Kaufman (1977), which the paper cites for the
    stability permutation P of Algorithm 1: alpha = (1 + sqrt 17)/8, a 1x1 pivot when the diagonal
    is large enough relative to the column, else a 1x1 pivot at the column's argmax r or a 2x2 pivot
    on (k, r)."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    W = np.asfortranarray(np.tril(M))
    perm = np.zeros(n, dtype=np.int32)
    d = np.zeros(n); e = np.zeros(n); piv = np.zeros(n, dtype=np.int8)
    out = np.zeros(4, dtype=np.int64)
    _lib().orc_dense_bk(n, _ptr(W), _ptr(perm), _ptr(d), _ptr(e), _ptr(piv), _ptr(out))
    L = np.tril(W, -1) + np.eye(n)
    for k in range(n):                      # the 2x2 blocks' off-diagonal is D's, not L's
        if piv[k] == 2:
            L[k + 1, k] = 0.0
    return DenseBK(L, d, e, piv, perm, tuple(int(v) for v in out))


def dense_inertia(M: np.ndarray) -> tuple[int, int, int]:
    """(neg, zero, pos) of the dense symmetric M by (c1)."""
    r = dense_bk(M)
    return r.neg, r.zero, r.pos


def dense_nu(A: np.ndarray, B: np.ndarray, sigma: float) -> int:
    """nu_sigma(A, B) = nu_0(D, I) for P (A - sigma B) P^T = L D L^T (Algorithm 1, via (c1))."""
    return dense_inertia(np.asarray(A) - sigma * np.asarray(B))[0]


# ------------------------------------------------------------------------------------------
# (c3) plain sparse multifrontal LDL^T
# ------------------------------------------------------------------------------------------
def sparse_inertia(rowptr, colind, a, b, ca: float, cb: float, *, leaf: int = 64,
                   u: float = 0.01) -> dict:
    """(c3) inertia of ca*A + cb*B (CSR with both triangles, A and B on one pattern).

    Plain multifrontal LDL^T with the oracle's own nested-dissection ordering (Algorithm 1', the
    fill-reducing Q) and threshold-restricted pivoting inside each front, failed pivots passed to
    the parent.  Returns dict(neg, zero, pos, delayed, n2x2, nfronts, max_front)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rowptr.size - 1
    out = np.zeros(7, dtype=np.int64)
    rc = _lib().orc_sparse_inertia(n, _ptr(rowptr), _ptr(colind), _ptr(a), _ptr(b), float(ca),
                                   float(cb), int(leaf), float(u), _ptr(out))
    if rc != 0:
        raise MemoryError("orc_sparse_inertia: allocation failed")
    keys = ["neg", "zero", "pos", "delayed", "n2x2", "nfronts", "max_front"]
    return {k: int(v) for k, v in zip(keys, out)}


def sparse_nu(pencil, sigma: float, **kw) -> int:
    """nu_sigma(A, B) for a gen.Pencil by (c3)."""
    return sparse_inertia(pencil.rowptr, pencil.colind, pencil.a, pencil.b, 1.0, -sigma, **kw)["neg"]


# ------------------------------------------------------------------------------------------
# (c2) dense generalized eigenpairs
# ------------------------------------------------------------------------------------------
def gen_eig(A: np.ndarray, B: np.ndarray):
    """(c2) all eigenpairs of A x = lambda B x, B-orthonormal X, ascending lambda.

    Cholesky reduction as in the dense comparison solver of Section 4.2: B = L L^H,
    C = L^{-1} A L^{-H}, C = Y diag(lam) Y^H, X = L^{-H} Y.  Real symmetric or complex Hermitian
    (A, B); raises LinAlgError if B is not positive definite."""
    dt = np.complex128 if (np.iscomplexobj(A) or np.iscomplexobj(B)) else np.float64
    A = np.asarray(A, dtype=dt); B = np.asarray(B, dtype=dt)
    L = np.linalg.cholesky(B)
    T = sla.solve_triangular(L, A, lower=True)                 # L^{-1} A
    C = sla.solve_triangular(L, T.conj().T, lower=True)        # L^{-1} A^H L^{-H} = L^{-1} A L^{-H}
    C = 0.5 * (C + C.conj().T)
    lam, Y = np.linalg.eigh(C)
    X = sla.solve_triangular(L.conj().T, Y, lower=False)
    return lam, X


def eig_grad(A: np.ndarray, B: np.ndarray, k: int):
    """Derivatives of lambda_k of A x = lambda B x (Hellmann-Feynman): with x the (c2) eigenvector,
    B-normalized, every stored entry an independent variable, G^A_ij = x_i conj(x_j) and
    G^B_ij = -lambda x_i conj(x_j), so that d lambda = sum_ij Re(conj(G_ij) dM_ij) (for real pencils
    G^A_ij = x_i x_j).  Returns (lambda_k, GA, GB) as dense matrices."""
    lam, X = gen_eig(A, B)
    x = X[:, k - 1]
    G = np.outer(x, x.conj())
    return float(lam[k - 1]), G, -float(lam[k - 1]) * G


def hermitian_nu(A: np.ndarray, B: np.ndarray, sigma: float) -> int:
    """nu_sigma(A, B) of a Hermitian pencil with B positive definite: the number of negative
    eigenvalues of A - sigma B (Sylvester's law of inertia, Section 2.1), from the library
    Hermitian eigenvalue routine."""
    return int(np.count_nonzero(np.linalg.eigvalsh(np.asarray(A) - sigma * np.asarray(B)) < 0.0))


def count_below(eigs: np.ndarray, sigma: float) -> int:
    """nu(sigma) from a list of eigenvalues (the definition, Section 2.1)."""
    return int(np.count_nonzero(np.asarray(eigs) < sigma))


# ------------------------------------------------------------------------------------------
# closed forms
# ------------------------------------------------------------------------------------------
def sband_eigs(l1: int, l2: int, l3: int, eps: float, t: float, beta: float, gamma: float):
    """Pencil eigenvalues of the periodic simple-cubic s-band pencil (gen.sband_cubic_pencil).

    A = eps I + t * adjacency has eigenvalues mu = eps + 2t sum_d cos(2 pi m_d / l_d) (plane waves);
    B = beta I + gamma A shares the eigenvectors, so lambda = mu / (beta + gamma mu)."""
    c1 = np.cos(2 * np.pi * np.arange(l1) / l1)
    c2 = np.cos(2 * np.pi * np.arange(l2) / l2)
    c3 = np.cos(2 * np.pi * np.arange(l3) / l3)
    mu = eps + 2 * t * (c1[:, None, None] + c2[None, :, None] + c3[None, None, :])
    mu = mu.ravel()
    return np.sort(mu / (beta + gamma * mu))


def diamond_bloch_eigs(nx: int, ny: int, nz: int, beta: float, gamma: float, cutoff: float = 2.9):
    """Pencil eigenvalues of gen.perfect_diamond_pencil by Bloch's theorem.

    The periodic supercell of nx*ny*nz conventional cells (each >= 2) is invariant under cell
    translations R, so A's eigenvalues are those of the 32x32 Bloch matrices
    H(q) = sum_R H(0, R) exp(i q.R) over q = 2 pi (m1/nx, m2/ny, m3/nz)/a; B = beta I + gamma A gives
    lambda = mu / (beta + gamma mu).  The hopping blocks come from the same Slater-Koster definition
    the generator uses (input construction, not method arithmetic)."""
    from gen.tightbinding import DIAMOND_A, _BASIS, sk_blocks, ONSITE_S, ONSITE_P
    a = DIAMOND_A
    basis = _BASIS * a
    blocks = []   # (alpha, beta, R, 4x4)
    for R in itertools.product((-1, 0, 1), repeat=3):
        Rv = np.array(R, dtype=np.float64) * a
        for al in range(8):
            for be in range(8):
                d = basis[be] + Rv - basis[al]
                r = math.sqrt(float(d @ d))
                if 0 < r < cutoff:
                    blocks.append((al, be, np.array(R), sk_blocks(d[None, :])[0]))
    m1, m2, m3 = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    q = np.stack([m1.ravel() / nx, m2.ravel() / ny, m3.ravel() / nz], 1) * 2 * np.pi
    nq = q.shape[0]
    H = np.zeros((nq, 32, 32), dtype=np.complex128)
    onsite = np.array([ONSITE_S, ONSITE_P, ONSITE_P, ONSITE_P])
    for al in range(8):
        H[:, 4 * al:4 * al + 4, 4 * al:4 * al + 4] += np.diag(onsite)[None]
    for al, be, R, h in blocks:
        ph = np.exp(1j * (q @ R.astype(np.float64)))
        H[:, 4 * al:4 * al + 4, 4 * be:4 * be + 4] += ph[:, None, None] * h[None]
    mu = np.linalg.eigvalsh(H).ravel()
    return np.sort(mu / (beta + gamma * mu))


def certified_shifts(eigs: np.ndarray, count: int, delta: float, seed: int,
                     lo: float | None = None, hi: float | None = None) -> np.ndarray:
    """`count` shifts drawn uniformly in [lo, hi] (default: the spectrum) and kept only if no
    eigenvalue lies within `delta` of them (so nu is unambiguous there)."""
    eigs = np.sort(np.asarray(eigs))
    lo = eigs[0] if lo is None else lo
    hi = eigs[-1] if hi is None else hi
    rng = np.random.default_rng([seed, 77])
    out = []
    while len(out) < count:
        s = rng.uniform(lo, hi)
        i = np.searchsorted(eigs, s)
        near = min(abs(eigs[max(i - 1, 0)] - s), abs(eigs[min(i, eigs.size - 1)] - s))
        if near > delta:
            out.append(s)
    return np.array(out)


# ------------------------------------------------------------------------------------------
# brute force (pins)
# ------------------------------------------------------------------------------------------
def leibniz_det(M: np.ndarray) -> float:
    """Determinant by the permutation expansion (brute force, n <= 7)."""
    n = M.shape[0]
    if n == 0:
        return 1.0
    tot = 0.0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        prod = 1.0
        for i in range(n):
            prod *= M[i, p[i]]
        tot += -prod if inv % 2 else prod
    return tot


def jacobi_negative_count(M: np.ndarray):
    """Negative eigenvalue count of symmetric M by Jacobi's rule: the number of sign changes in
    1, D_1, ..., D_n (leading principal minors), valid when every minor is nonzero.
    Returns None if a minor vanishes."""
    n = M.shape[0]
    minors = [1.0] + [leibniz_det(M[:k, :k]) for k in range(1, n + 1)]
    if any(m == 0.0 for m in minors):
        return None
    return sum(1 for i in range(n) if minors[i] * minors[i + 1] < 0)
