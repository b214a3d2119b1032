"""GPU parity: inertia, solves and sparse products of the CUDA path against the oracle.

Inertia is compared bit-exactly (an integer) at shifts certified to lie at least 1e-8*||A||
from every eigenvalue (closed forms or the oracle's dense eigenvalues give the certificate).
Solves are compared element by element with the oracle's dense solve within a tolerance derived
from the conditioning: |x - x_ref| <= 1e-9 * ||x_ref||_inf (backward-stable LDL^T with growth
bounded by the threshold u = 0.01 and condition numbers ~1e3 of these shifted pencils)."""
import numpy as np
import pytest
import scipy.sparse as sp

from gen import diagonal_pencil, make_pair, perfect_diamond_pencil, sband_cubic_pencil, workload
from oracle import core, three_stage as ts
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kep():
    return require_gpu()


@pytest.fixture(scope="module")
def small():
    p = workload("small")                    # n = 2048
    A, B = p.A().toarray(), p.B().toarray()
    lam, X = core.gen_eig(A, B)
    return p, A, B, lam


def test_inertia_small_workload_vs_dense(kep, small):
    p, A, B, lam = small
    nrm = np.abs(A).sum(1).max()
    P = kep.Problem.from_pencil(p)
    shifts = core.certified_shifts(lam, 16, 1e-8 * nrm, seed=11, lo=lam[0] - 1, hi=lam[-1] + 1)
    for i, s in enumerate(shifts):
        r = P.factor(s)
        assert r.status == 0
        ref = core.count_below(lam, s)
        assert (r.neg, r.zero, r.pos) == (ref, 0, p.n - ref), s
        if i < 3:                            # the oracle's own LDL^T route agrees too
            assert core.dense_nu(A, B, s) == ref
    # outside the spectrum
    assert P.factor(lam[0] - 1.0).neg == 0
    assert P.factor(lam[-1] + 1.0).neg == p.n


def test_inertia_graph_ordering(kep, small):
    """The coordinate-free ordering gives the same exact counts (Sylvester: any P, Q)."""
    p, A, B, lam = small
    nrm = np.abs(A).sum(1).max()
    P = kep.Problem.from_pencil(p, graph_order=True)
    for s in core.certified_shifts(lam, 4, 1e-8 * nrm, seed=12):
        assert P.factor(s).neg == core.count_below(lam, s)


def test_lower_pattern_input(kep, small):
    p, A, B, lam = small
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    keep = p.colind <= rows
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=p.n))])
    P = kep.Problem(p.n, rp, p.colind[keep], p.a[keep], p.b[keep], p.coords, lower=True)
    s = 0.5 * (lam[p.k - 1] + lam[p.k])
    assert P.factor(s).neg == p.k


def test_tiny_and_diagonal(kep):
    for n in [1, 2, 7, 33]:
        rng = np.random.default_rng(n)
        a = rng.normal(size=n); b = rng.uniform(0.5, 2.0, n)
        P = kep.Problem.from_pencil(diagonal_pencil(a, b))
        for s in [-0.3, 0.1, 0.7]:
            r = P.factor(s)
            assert r.neg == int((a / b < s).sum())


def test_exact_zero_pivot_reports_singular(kep):
    a = np.array([1.0, 2.0, -1.0]); b = np.ones(3)
    P = kep.Problem.from_pencil(diagonal_pencil(a, b))
    r = P.factor(2.0)                        # sigma equals an eigenvalue
    assert r.status == kep.KEP_ERR_SINGULAR and (r.neg, r.zero, r.pos) == (2, 1, 0)
    with pytest.raises(kep.KepError):
        P.solve(np.ones(3))


def test_B_is_positive_definite(kep, small):
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    r = P.factor_pencil(0.0, 1.0)
    assert (r.neg, r.zero, r.pos) == (0, 0, p.n)


def test_forced_delays_zero_diagonal(kep):
    """Zero diagonal in A - sigma B: pivots fail the threshold, get delayed; counts stay exact."""
    p = make_pair(2, 2, 3, seed=5)
    sigma = 0.25
    a = p.a.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    d = rows == p.colind
    a[d] = sigma * p.b[d]
    M = sp.csr_matrix((a, p.colind, p.rowptr), shape=(p.n, p.n)).toarray() - sigma * p.B().toarray()
    ref = core.dense_inertia(M)
    P = kep.Problem(p.n, p.rowptr, p.colind, a, p.b, p.coords)
    r = P.factor(sigma)
    assert (r.neg, r.zero, r.pos) == ref
    assert r.delayed > 0


@pytest.mark.parametrize("dims", [(32, 32, 32), (17, 23, 29)])
def test_inertia_sband_closed_form(kep, dims):
    p = sband_cubic_pencil(*dims, eps=0.0, t=-1.0, beta=1.0, gamma=0.05)
    cf = core.sband_eigs(*dims, 0.0, -1.0, 1.0, 0.05)
    P = kep.Problem.from_pencil(p)
    for s in core.certified_shifts(cf, 5, 1e-6, seed=2):
        assert P.factor(s).neg == core.count_below(cf, s)


def test_inertia_diamond_bloch_closed_form(kep):
    p = perfect_diamond_pencil(8, 8, 8)      # n = 16384
    cf = core.diamond_bloch_eigs(8, 8, 8, 1.0, 0.02)
    P = kep.Problem.from_pencil(p)
    for s in core.certified_shifts(cf, 5, 1e-6, seed=2):
        assert P.factor(s).neg == core.count_below(cf, s)


def test_inertia_vs_sparse_oracle_mid(kep):
    """A jittered workload the dense route cannot reach: the oracle's sparse LDL^T (c3) certifies
    the shift (equal counts at sigma -+ delta) and gives the count."""
    p = make_pair(5, 5, 5, seed=7, vacancies=100)     # n = 3600
    P = kep.Problem.from_pencil(p)
    nrm = np.abs(p.A()).sum(1).max()
    delta = 1e-8 * nrm
    rng = np.random.default_rng(3)
    done = 0
    while done < 3:
        s = rng.uniform(-8, 4)
        lo, hi = core.sparse_nu(p, s - delta), core.sparse_nu(p, s + delta)
        if lo != hi:
            continue
        assert P.factor(s).neg == lo
        done += 1


def test_solve_vs_dense(kep, small):
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    s = 0.5 * (lam[p.k - 1] + lam[p.k]) + 1e-3
    P.factor(s)
    rng = np.random.default_rng(0)
    b = rng.normal(size=p.n)
    x = P.solve(b)
    M = A - s * B
    xr = ts.DenseOps(A, B).shifted_solver(s)(b)
    assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
    assert np.linalg.norm(M @ x - b) <= 1e-13 * np.linalg.norm(M, np.inf) * np.linalg.norm(x)
    # several right-hand sides at once, and a B solve
    R = rng.normal(size=(3, p.n))
    X = P.solve(R)
    for i in range(3):
        assert np.linalg.norm(M @ X[i] - R[i]) <= 1e-13 * np.linalg.norm(M, np.inf) * np.linalg.norm(X[i])
    P.factor_pencil(0.0, 1.0)
    xb = P.solve(b)
    assert np.linalg.norm(B @ xb - b) <= 1e-13 * np.linalg.norm(b)


def test_solve_device_tensors(kep, small):
    import torch
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    s = lam[10] + 1e-3
    P.factor(s)
    b = torch.randn(p.n, dtype=torch.float64, device="cuda")
    x = P.solve(b)
    M = A - s * B
    xn = x.cpu().numpy()
    assert np.linalg.norm(M @ xn - b.cpu().numpy()) <= 1e-13 * np.linalg.norm(M, np.inf) * np.linalg.norm(xn)


def test_spmv(kep, small):
    import torch
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    x = np.random.default_rng(1).normal(size=p.n)
    ax, bx = P.spmv(x)
    As, Bs = p.A(), p.B()
    assert np.abs(ax - As @ x).max() <= 1e-14 * np.abs(As).sum(1).max() * np.abs(x).max()
    assert np.abs(bx - Bs @ x).max() <= 1e-14 * np.abs(Bs).sum(1).max() * np.abs(x).max()
    xd = torch.from_numpy(x).cuda()
    ad, bd = P.spmv(xd)
    assert np.array_equal(ad.cpu().numpy(), ax) and np.array_equal(bd.cpu().numpy(), bx)


def test_timing_counters(kep, small):
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    P.timing(reset=True)
    P.set_timing(True)
    P.factor(0.3)
    t = P.timing(reset=True)
    assert t["update"][0] > 0 and t["update"][1] > 0
    assert t["total_launches"] == sum(v[0] for k, v in t.items() if k not in ("total_launches", "flops"))
    assert t["flops"]["update"] > 0


def test_solve_multiblock_fronts_vs_sparse_lu(kep):
    """Fronts of order >= 512 take the dataflow solve (many CTAs per front, 64-row blocks, flags);
    compare with the oracle's sparse LU."""
    p = make_pair(8, 8, 8, seed=3)            # n = 16384, largest front > 2048
    P = kep.Problem.from_pencil(p)
    assert P.info.max_front >= 2048
    s = 0.37
    r = P.factor(s)
    assert r.status == 0
    ops = ts.SparseOps(p)
    rng = np.random.default_rng(4)
    b = rng.normal(size=p.n)
    x = P.solve(b)
    xr = ops.shifted_solver(s)(b)
    assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
    M = (p.A() - s * p.B()).tocsr()
    assert np.linalg.norm(M @ x - b) <= 1e-13 * abs(M).sum(1).max() * np.linalg.norm(x)


def test_solve_two_by_two_pivots_and_delays_dataflow(kep):
    """A zero diagonal in A - sigma B forces 2x2 pivots and delayed columns inside fronts large
    enough for the dataflow solve (block boundaries moved around 2x2 pairs); the solve must match
    the oracle's dense solve, for several right-hand sides in a row."""
    import scipy.sparse as sp
    p = make_pair(4, 4, 4, seed=6)            # n = 2048
    sigma = 0.3
    a = p.a.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    d = rows == p.colind
    a[d] = sigma * p.b[d]
    A = sp.csr_matrix((a, p.colind, p.rowptr), shape=(p.n, p.n)).toarray()
    B = p.B().toarray()
    M = A - sigma * B
    P = kep.Problem(p.n, p.rowptr, p.colind, a, p.b, p.coords)
    assert P.info.max_front >= 512
    r = P.factor(sigma)
    assert (r.neg, r.zero, r.pos) == core.dense_inertia(M)
    rng = np.random.default_rng(11)
    for _ in range(3):
        b = rng.normal(size=p.n)
        x = P.solve(b)
        xr = np.linalg.solve(M, b)
        assert np.abs(x - xr).max() <= 1e-8 * np.abs(xr).max()
        assert np.linalg.norm(M @ x - b) <= 1e-12 * np.linalg.norm(M, np.inf) * np.linalg.norm(x)


def test_schur_tile_32_parity(kep, small):
    """The 32 x 32 FP64 Schur tiles (the autotuner's other tile shape) give the same exact counts
    as the dense spectrum and solves of the same accuracy, with every front below the tensor-core
    threshold."""
    p, A, B, lam = small
    nrm = np.abs(A).sum(1).max()
    with kep.Problem.from_pencil(p) as P:
        P.set_schur_mode(False)
        P.set_schur_tile(32)
        assert P.schur_config()["tile"] == 32
        for s in core.certified_shifts(lam, 8, 1e-8 * nrm, seed=23):
            r = P.factor(s)
            ref = core.count_below(lam, s)
            assert (r.neg, r.zero, r.pos) == (ref, 0, p.n - ref), s
        b = np.random.default_rng(12).normal(size=p.n)
        x = P.solve(b)
        M = A - s * B
        assert np.linalg.norm(M @ x - b) <= 1e-13 * np.linalg.norm(M, np.inf) * np.linalg.norm(x)
        with pytest.raises(kep.KepError):
            P.set_schur_tile(48)
