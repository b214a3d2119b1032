"""GPU parity of Algorithm 4 (kep_kth_eigenpair) against the oracle.

The random start vectors of Algorithms 2 and 3 are inputs: both sides get the same ones.
lambda_k must agree with the oracle's dense generalized eigensolver within 1e-10 * ||A||_inf
(the tolerance the method's validation targets), the eigenvector within 1e-8 after B-normalization
and sign alignment, the relative residual must be below tau_res, and the intervals of Algorithms 2
and 1' must carry the same exact inertia counts as the oracle's run."""
import numpy as np
import pytest

from gen import make_pair, workload
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
    lam, X = core.gen_eig(A, B)
    return p, A, B, lam, X


def _check_pair(p, A, B, lam, X, k, lam_gpu, x_gpu, rep):
    nrm = np.abs(A).sum(1).max()
    assert abs(lam_gpu - lam[k - 1]) <= 1e-10 * nrm
    assert abs(x_gpu @ B @ x_gpu - 1.0) < 1e-10
    xd = X[:, k - 1]
    x = x_gpu * np.sign(x_gpu @ B @ xd)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    r = np.linalg.norm(A @ x_gpu - lam_gpu * (B @ x_gpu)) / np.linalg.norm(x_gpu)
    assert r < 1e-10 and rep["rel_res"] < 1e-10
    assert rep["nu_lo"] < k <= rep["nu_hi"] and rep["nu_hi"] - rep["nu_lo"] <= 20
    assert rep["init_nu_lo"] < k <= rep["init_nu_hi"]
    assert rep["nu_lo"] == core.count_below(lam, rep["sigma_lo"])
    assert rep["nu_hi"] == core.count_below(lam, rep["sigma_hi"])


def test_kth_eigenpair_matches_oracle(kep, small):
    p, A, B, lam, X = small
    k = p.k
    rng = np.random.default_rng(5)
    v1, vt1 = rng.normal(size=p.n), rng.normal(size=p.n)
    P = kep.Problem.from_pencil(p)
    lam_g, x_g, rep = P.kth_eigenpair(k, start_vectors=np.concatenate([v1, vt1]))
    _check_pair(p, A, B, lam, X, k, lam_g, x_g, rep)
    # the oracle's Algorithm 4 from the same start vectors: same intervals and counts
    r = ts.three_stage(ts.DenseOps(A, B), k, v1, vt1)
    assert (rep["init_nu_lo"], rep["init_nu_hi"]) == (r.initial.nu_lower, r.initial.nu_upper)
    assert abs(rep["init_lo"] - r.initial.lower) <= 1e-9 * abs(r.initial.lower)
    assert abs(rep["init_hi"] - r.initial.upper) <= 1e-9 * abs(r.initial.upper)
    assert (rep["nu_lo"], rep["nu_hi"]) == (r.narrowed.nu_lower, r.narrowed.nu_upper)
    assert rep["n_lanczos"] == len(r.initial.history)
    assert rep["n_bisect"] == len(r.narrowed.history)
    nrm = np.abs(A).sum(1).max()
    assert abs(lam_g - r.lam) <= 1e-10 * nrm
    assert abs(rep["n_si_iter"] - r.kth.iterations) <= 3


@pytest.mark.parametrize("frac", [0.05, 0.3, 0.8])
def test_kth_eigenpair_other_indices(kep, small, frac):
    p, A, B, lam, X = small
    k = max(2, int(frac * p.n))
    P = kep.Problem.from_pencil(p)
    lam_g, x_g, rep = P.kth_eigenpair(k, seed=k)
    _check_pair(p, A, B, lam, X, k, lam_g, x_g, rep)


def test_kth_eigenpair_vacancy_pencil(kep):
    p = make_pair(3, 3, 3, seed=2, vacancies=20)      # irregular spectrum
    A, B = p.A().toarray(), p.B().toarray()
    lam, X = core.gen_eig(A, B)
    P = kep.Problem.from_pencil(p)
    lam_g, x_g, rep = P.kth_eigenpair(p.k)
    _check_pair(p, A, B, lam, X, p.k, lam_g, x_g, rep)


def test_not_spd_B_rejected(kep):
    p = make_pair(2, 2, 2, seed=1)
    P = kep.Problem(p.n, p.rowptr, p.colind, p.a, p.a, p.coords)   # "B" = A is indefinite
    with pytest.raises(kep.KepError) as e:
        P.kth_eigenpair(p.k)
    assert e.value.code == kep.KEP_ERR_NOT_SPD


def test_kth_eigenpair_shared_b_slot(kep, small):
    """Algorithm 4 with B's factor in the slot of the shifted factorizations (the layout of the
    largest problems): B is factored once, the later B-solves run conjugate gradients.  Same
    interval, counts and lambda_k as with B's own slot, and no further factorization of B."""
    p, A, B, lam, X = small
    k = p.k
    rng = np.random.default_rng(17)
    sv = rng.normal(size=2 * p.n)
    with kep.Problem.from_pencil(p) as P:
        lo, xo, ro = P.kth_eigenpair(k, start_vectors=sv, b_factor="own")
        ls, xs, rs = P.kth_eigenpair(k, start_vectors=sv, b_factor="shared")
    _check_pair(p, A, B, lam, X, k, ls, xs, rs)
    assert abs(ls - lo) <= 1e-12 * np.abs(A).sum(1).max()
    assert (rs["init_nu_lo"], rs["init_nu_hi"], rs["nu_lo"], rs["nu_hi"]) == \
        (ro["init_nu_lo"], ro["init_nu_hi"], ro["nu_lo"], ro["nu_hi"])
    assert rs["n_factor"] == ro["n_factor"]          # B factored once in both layouts


@pytest.mark.parametrize("frac", [0.3, 0.5])
def test_kth_eigenpair_interp_split_matches_oracle(kep, small, frac):
    """Algorithm 1' with the interpolating shift rule (split="interp"): the same Algorithm 2
    interval, the same sequence of counts and the same narrowed interval as the oracle's run from
    the same start vectors, and lambda_k within the method's tolerance."""
    p, A, B, lam, X = small
    k = max(2, int(frac * p.n))
    rng = np.random.default_rng(9)
    v1, vt1 = rng.normal(size=p.n), rng.normal(size=p.n)
    P = kep.Problem.from_pencil(p)
    lam_g, x_g, rep = P.kth_eigenpair(k, start_vectors=np.concatenate([v1, vt1]), split="interp")
    _check_pair(p, A, B, lam, X, k, lam_g, x_g, rep)
    r = ts.three_stage(ts.DenseOps(A, B), k, v1, vt1, split="interp")
    assert (rep["init_nu_lo"], rep["init_nu_hi"]) == (r.initial.nu_lower, r.initial.nu_upper)
    assert (rep["nu_lo"], rep["nu_hi"]) == (r.narrowed.nu_lower, r.narrowed.nu_upper)
    assert rep["n_bisect"] == len(r.narrowed.history)
    w = r.initial.upper - r.initial.lower
    assert abs(rep["sigma_lo"] - r.narrowed.lower) <= 1e-9 * w
    assert abs(rep["sigma_hi"] - r.narrowed.upper) <= 1e-9 * w
    nrm = np.abs(A).sum(1).max()
    assert abs(lam_g - r.lam) <= 1e-10 * nrm
    # the paper's bisection from the same interval takes at least as many factorizations here
    rb = ts.multisect_mmax(ts.DenseOps(A, B), k, r.initial, 20, 1)
    assert rep["n_bisect"] <= len(rb.history)
    with pytest.raises(kep.KepError):
        P.kth_eigenpair(k, split="interp", nshift=4)     # the rule takes one shift per step


def test_kth_eigenpair_restart_after_inexact_solves(kep, small):
    """Algorithm 3 on solves that carry rounding well above FP64's (every factor of the run taken in
    reduced precision, solves unrefined): the Lanczos relation and the relative differences
    converge on the perturbed operator while the explicit residuals stop far above tau_res.  The
    driver then runs Algorithm 3 once more with every shifted solve refined in FP64 and returns
    lambda_k and x_k to the method's tolerances."""
    p, A, B, lam, X = small
    k = p.k
    P = kep.Problem.from_pencil(p)
    P.set_schur_mode(True, fp32=True)
    lam_g, x_g, rep = P.kth_eigenpair(k, seed=3)
    assert rep["restarted"] == 1
    _check_pair(p, A, B, lam, X, k, lam_g, x_g, rep)
    # the FP64-accurate run does not need it
    P.set_schur_mode(True)
    lam_f, _, rep_f = P.kth_eigenpair(k, seed=3)
    assert rep_f["restarted"] == 0
    assert abs(lam_g - lam_f) <= 1e-10 * np.abs(A).sum(1).max()
