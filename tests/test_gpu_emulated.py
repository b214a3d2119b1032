"""Parity of the tensor-core (FP64-accurate splitting) Schur update against the oracle.

With the threshold lowered to a few hundred rows, nearly every front's deferred update runs on
the tensor cores; inertia must still match the closed forms / oracle exactly at certified shifts,
and solves must meet the same tolerances as the FP64 path."""
import numpy as np
import pytest
import scipy.sparse as sp

from gen import make_pair, perfect_diamond_pencil, sband_cubic_pencil, workload
from oracle import core, three_stage as ts
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kep():
    return require_gpu()


@pytest.fixture(scope="module")
def small():
    p = workload("small")
    A, B = p.A().toarray(), p.B().toarray()
    lam, _ = core.gen_eig(A, B)
    return p, A, B, lam


def test_emulated_inertia_small(kep, small):
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    P.set_schur_mode(True, min_front=256)
    nrm = np.abs(A).sum(1).max()
    for s in core.certified_shifts(lam, 12, 1e-8 * nrm, seed=21, lo=lam[0] - 1, hi=lam[-1] + 1):
        r = P.factor(s)
        ref = core.count_below(lam, s)
        assert (r.neg, r.zero, r.pos) == (ref, 0, p.n - ref), s


def test_emulated_solve_matches_dense(kep, small):
    p, A, B, lam = small
    P = kep.Problem.from_pencil(p)
    P.set_schur_mode(True, min_front=256)
    s = 0.5 * (lam[p.k - 1] + lam[p.k]) + 1e-3
    P.factor(s)
    b = np.random.default_rng(0).normal(size=p.n)
    x = P.solve(b)
    xr = ts.DenseOps(A, B).shifted_solver(s)(b)
    M = A - s * B
    assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
    assert np.linalg.norm(M @ x - b) <= 1e-13 * np.linalg.norm(M, np.inf) * np.linalg.norm(x)


@pytest.mark.parametrize("dims", [(32, 32, 32), (17, 23, 29)])
def test_emulated_sband_closed_form(kep, dims):
    p = sband_cubic_pencil(*dims, eps=0.0, t=-1.0, beta=1.0, gamma=0.05)
    cf = core.sband_eigs(*dims, 0.0, -1.0, 1.0, 0.05)
    P = kep.Problem.from_pencil(p)
    P.set_schur_mode(True, min_front=512)
    for s in core.certified_shifts(cf, 5, 1e-6, seed=4):
        assert P.factor(s).neg == core.count_below(cf, s)


def test_emulated_diamond_closed_form_and_residual(kep):
    p = perfect_diamond_pencil(8, 8, 8)
    cf = core.diamond_bloch_eigs(8, 8, 8, 1.0, 0.02)
    P = kep.Problem.from_pencil(p)
    P.set_schur_mode(True, min_front=512)
    shifts = core.certified_shifts(cf, 5, 1e-6, seed=5)
    for s in shifts:
        assert P.factor(s).neg == core.count_below(cf, s)
    s = shifts[-1]
    b = np.random.default_rng(1).normal(size=p.n)
    x = P.solve(b)
    M = (p.A() - s * p.B()).tocsr()
    assert np.linalg.norm(M @ x - b) <= 1e-13 * abs(M).sum(1).max() * np.linalg.norm(x)


def test_emulated_forced_delays(kep):
    p = make_pair(2, 2, 3, seed=5)
    sigma = 0.25
    a = p.a.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    d = rows == p.colind
    a[d] = sigma * p.b[d]
    M = sp.csr_matrix((a, p.colind, p.rowptr), shape=(p.n, p.n)).toarray() - sigma * p.B().toarray()
    ref = core.dense_inertia(M)
    P = kep.Problem(p.n, p.rowptr, p.colind, a, p.b, p.coords)
    P.set_schur_mode(True, min_front=64)
    r = P.factor(sigma)
    assert (r.neg, r.zero, r.pos) == ref


def test_emulated_matches_fp64_factor(kep):
    """The two arithmetics give solves that agree to FP64 accuracy on a mid-size pencil."""
    p = make_pair(8, 8, 8, seed=3)
    P = kep.Problem.from_pencil(p)
    s = 0.37
    b = np.random.default_rng(2).normal(size=p.n)
    P.set_schur_mode(False)
    r64 = P.factor(s)
    x64 = P.solve(b)
    P.set_schur_mode(True, min_front=512)
    re = P.factor(s)
    xe = P.solve(b)
    assert (r64.neg, r64.zero, r64.pos) == (re.neg, re.zero, re.pos)
    assert np.abs(xe - x64).max() <= 1e-10 * np.abs(x64).max()


def test_emulated_near_eigenvalue_shifts(kep, small):
    """Shifts 2e-8 ||A|| from an eigenvalue (the Schur complements cancel down to the size of the
    nearest eigenvalue's gap): the tensor-core update must still give the exact count, on the
    oracle's dense spectrum (n = 2,048, fronts from order 256 on the tensor cores) and on the
    closed-form diamond spectrum (n = 16,384)."""
    p, A, B, lam = small
    nrm = np.abs(A).sum(1).max()
    P = kep.Problem.from_pencil(p)
    P.set_schur_mode(True, min_front=256)
    idx = np.random.default_rng(8).choice(np.arange(1, p.n - 1), 16, replace=False)
    tried = 0
    for i in idx:
        for sgn in (1.0, -1.0):
            s = lam[i] + sgn * 2e-8 * nrm
            if np.abs(lam - s).min() < 1e-8 * nrm:
                continue
            r = P.factor(s)
            ref = core.count_below(lam, s)
            assert (r.neg, r.zero, r.pos) == (ref, 0, p.n - ref), (i, sgn)
            tried += 1
    assert tried >= 16
    q = perfect_diamond_pencil(8, 8, 8)
    cf = core.diamond_bloch_eigs(8, 8, 8, 1.0, 0.02)
    nq = float(abs(q.A()).sum(1).max())
    lv = np.unique(np.round(cf / (1e-10 * nq))) * 1e-10 * nq
    gaps = np.diff(lv)
    ok = np.where((gaps[:-1] > 1e-7 * nq) & (gaps[1:] > 1e-7 * nq))[0] + 1
    Q = kep.Problem.from_pencil(q)
    Q.set_schur_mode(True, min_front=256)
    assert Q.info.max_front >= 256
    for i in np.random.default_rng(9).choice(ok, 6, replace=False):
        for sgn in (1.0, -1.0):
            s = lv[i] + sgn * 2e-8 * nq
            assert np.abs(cf - s).min() > 1e-8 * nq
            assert Q.factor(s).neg == core.count_below(cf, s), (i, sgn)
