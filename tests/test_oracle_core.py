"""Pins for the oracle's inertia and eigenvalue routes (no GPU).

Each check ties an oracle route to something other than itself: brute force, closed forms,
a different library routine, or an invariant that a plausible slip (dropped term, wrong sign,
transposed operand, wrong 2x2 sign rule) would break."""
import numpy as np
import pytest

from gen import diagonal_pencil, make_pair, perfect_diamond_pencil, sband_cubic_pencil
from oracle import core


def _sym(rng, n, diag_zero=False):
    M = rng.normal(size=(n, n))
    M = M + M.T
    if diag_zero:
        np.fill_diagonal(M, 0.0)
    return M


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_dense_bk_matches_jacobi_bruteforce(n):
    """(c1) negative count == sign changes of leading minors from permutation expansion."""
    rng = np.random.default_rng(100 + n)
    checked = 0
    for trial in range(40):
        M = _sym(rng, n, diag_zero=(trial % 3 == 0))
        ref = core.jacobi_negative_count(M)
        if ref is None:
            continue
        neg, zero, pos = core.dense_inertia(M)
        assert (neg, zero, pos) == (ref, 0, n - ref)
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("n,diag_zero", [(7, False), (60, False), (60, True), (250, True)])
def test_dense_bk_reconstruction(n, diag_zero):
    """P M P^T == L D L^T, L unit lower, D 1x1/2x2 (a dropped update term breaks this)."""
    rng = np.random.default_rng(n)
    M = _sym(rng, n, diag_zero)
    r = core.dense_bk(M)
    P = np.eye(n)[r.perm]
    assert np.allclose(np.diag(r.L), 1.0)
    assert np.all(np.triu(r.L, 1) == 0)
    err = np.abs(P @ M @ P.T - r.L @ r.D() @ r.L.T).max()
    assert err <= 1e-12 * np.abs(M).max() * n
    if diag_zero:
        assert r.n2x2 > 0          # the 2x2 branch really ran


def test_dense_bk_exact_special_cases():
    # [[0, 1], [1, 0]]: eigenvalues +-1, forces a 2x2 pivot with det < 0
    r = core.dense_bk(np.array([[0.0, 1.0], [1.0, 0.0]]))
    assert (r.neg, r.zero, r.pos, r.n2x2) == (1, 0, 1, 1)
    # rank one: [[1, 1], [1, 1]] -> one exact zero pivot
    assert core.dense_inertia(np.ones((2, 2))) == (0, 1, 1)
    # all-zero matrix
    assert core.dense_inertia(np.zeros((4, 4))) == (0, 4, 0)
    # diag(1, 0, -1)
    assert core.dense_inertia(np.diag([1.0, 0.0, -1.0])) == (1, 1, 1)
    # negative definite 2x2 blocks: [[-1, 3], [3, -1]] has eigenvalues 2, -4
    M = np.kron(np.eye(3), np.array([[-1.0, 3.0], [3.0, -1.0]]))
    assert core.dense_inertia(M) == (3, 0, 3)
    # [[-4, 1], [1, -4]] -> both negative
    M = np.kron(np.eye(2), np.array([[-4.0, 1.0], [1.0, -4.0]]))
    assert core.dense_inertia(M) == (4, 0, 0)


def test_dense_bk_vs_eigvalsh_and_invariants():
    rng = np.random.default_rng(7)
    n = 300
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.concatenate([rng.uniform(-5, -1e-3, 120), rng.uniform(1e-3, 5, 180)])
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    assert core.dense_inertia(M) == (120, 0, 180)
    # -M swaps the counts; a symmetric permutation leaves them unchanged (Sylvester)
    assert core.dense_inertia(-M) == (180, 0, 120)
    p = rng.permutation(n)
    assert core.dense_inertia(M[np.ix_(p, p)]) == (120, 0, 180)
    # against an independent library eigensolver on a random indefinite matrix
    M2 = _sym(rng, 200)
    assert core.dense_inertia(M2)[0] == int((np.linalg.eigvalsh(M2) < 0).sum())


def test_diagonal_pencil_closed_form():
    rng = np.random.default_rng(3)
    a = rng.normal(size=97); b = rng.uniform(0.5, 2.0, 97)
    p = diagonal_pencil(a, b)
    for sigma in [-1.0, -0.1, 0.0, 0.3, 2.0]:
        ref = int(np.count_nonzero(a / b < sigma))
        assert core.dense_nu(np.diag(a), np.diag(b), sigma) == ref
        assert core.sparse_nu(p, sigma) == ref


def test_sband_closed_form_vs_dense_eig():
    """The s-band formula and (c2) are independent routes to the same spectrum."""
    p = sband_cubic_pencil(5, 4, 3, eps=0.3, t=-1.0, beta=1.0, gamma=0.05)
    lam, X = core.gen_eig(p.A().toarray(), p.B().toarray())
    cf = core.sband_eigs(5, 4, 3, 0.3, -1.0, 1.0, 0.05)
    assert np.abs(lam - cf).max() < 1e-13


def test_bloch_closed_form_vs_dense_eig():
    p = perfect_diamond_pencil(2, 2, 3, beta=1.0, gamma=0.02)
    lam, _ = core.gen_eig(p.A().toarray(), p.B().toarray())
    cf = core.diamond_bloch_eigs(2, 2, 3, 1.0, 0.02)
    assert np.abs(lam - cf).max() < 1e-12


def test_gen_eig_residual_and_b_orthonormality():
    p = make_pair(2, 2, 2, seed=4)
    A, B = p.A().toarray(), p.B().toarray()
    lam, X = core.gen_eig(A, B)
    assert np.all(np.diff(lam) >= 0)
    R = A @ X - (B @ X) * lam
    assert np.abs(R).max() < 1e-12 * np.abs(A).sum(1).max()
    assert np.abs(X.T @ B @ X - np.eye(p.n)).max() < 1e-12


def test_sparse_matches_dense_on_workload():
    """(c3) == (c1) == count of (c2) eigenvalues (Sylvester's law, Section 2.1)."""
    p = make_pair(3, 3, 3, seed=11)          # n = 864
    A, B = p.A().toarray(), p.B().toarray()
    lam, _ = core.gen_eig(A, B)
    nrm = np.abs(A).sum(1).max()
    for s in core.certified_shifts(lam, 6, 1e-8 * nrm, seed=1):
        ref = core.count_below(lam, s)
        assert core.dense_nu(A, B, s) == ref
        assert core.sparse_nu(p, s) == ref


def test_sparse_forced_delays_and_2x2():
    """Zero diagonal in A - sigma B: every 1x1 pivot fails the threshold first, so the sparse route
    must use 2x2 pivots and pass columns to parent fronts; it must still agree with (c1)."""
    p = make_pair(2, 2, 3, seed=5)           # n = 384
    sigma = 0.25
    a = p.a.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    dmask = rows == p.colind
    a[dmask] = sigma * p.b[dmask]            # (A - sigma B)_ii = 0 exactly
    M = (p.A().toarray() * 0)
    import scipy.sparse as sp
    Am = sp.csr_matrix((a, p.colind, p.rowptr), shape=(p.n, p.n)).toarray()
    M = Am - sigma * p.B().toarray()
    assert np.all(np.diag(M) == 0)
    ref = core.dense_inertia(M)
    r = core.sparse_inertia(p.rowptr, p.colind, a, p.b, 1.0, -sigma, leaf=16)
    assert (r["neg"], r["zero"], r["pos"]) == ref
    assert r["n2x2"] > 0
    assert r["delayed"] > 0


@pytest.mark.parametrize("dims", [(24, 24, 24)])
def test_sparse_sband_closed_form(dims):
    p = sband_cubic_pencil(*dims, eps=0.0, t=-1.0, beta=1.0, gamma=0.05)
    cf = core.sband_eigs(*dims, 0.0, -1.0, 1.0, 0.05)
    for s in core.certified_shifts(cf, 3, 1e-6, seed=2):
        assert core.sparse_nu(p, s) == core.count_below(cf, s)


def test_sparse_bloch_closed_form():
    p = perfect_diamond_pencil(4, 4, 4)
    cf = core.diamond_bloch_eigs(4, 4, 4, 1.0, 0.02)
    for s in core.certified_shifts(cf, 3, 1e-6, seed=3):
        assert core.sparse_nu(p, s) == core.count_below(cf, s)


def test_generator_structure():
    p = make_pair(4, 4, 4, seed=0)
    A, B = p.A(), p.B()
    assert p.n == 2048 and p.k == 1024
    assert abs(A - A.T).max() == 0 and abs(B - B.T).max() == 0
    # same pattern, strictly diagonally dominant B
    Bd = B.toarray()
    off = np.abs(Bd).sum(1) - np.abs(np.diag(Bd))
    assert np.all(off < np.diag(Bd))
    assert 60 < p.nnz / p.n < 80
    # deterministic from the seed
    q = make_pair(4, 4, 4, seed=0)
    assert np.array_equal(p.a, q.a) and np.array_equal(p.colind, q.colind)
