"""Pins (no GPU) for the oracle pieces behind the next rows: the Gershgorin initial interval of the
variant in Section 4.2, multisection in Algorithm 1', and the Hellmann-Feynman derivatives of
lambda_k.

Pins come from outside the routines: the spectrum from the dense generalized eigensolver must lie
in the intervals, and for a diagonal pencil with B = I the Gershgorin interval is exactly
[min a, max a]; multisection with one point is bisection; the derivatives match central finite
differences of lambda_k (a different route: eigensolves of perturbed pencils)."""
import numpy as np
import pytest

from gen import make_pair
from oracle import core, three_stage as ts


@pytest.fixture(scope="module")
def small():
    p = make_pair(3, 3, 2, seed=21)          # n = 576
    A, B = p.A().toarray(), p.B().toarray()
    lam, X = core.gen_eig(A, B)
    return p, A, B, lam, X


def test_gershgorin_interval_holds_spectrum(small):
    p, A, B, lam, _ = small
    iv = ts.gershgorin_interval(A, B)
    assert iv.lower < lam[0] and lam[-1] < iv.upper
    assert core.count_below(lam, iv.lower) == 0 and core.count_below(lam, iv.upper) == p.n
    # same on the sparse operators
    iv2 = ts.gershgorin_interval(p.A(), p.B())
    assert abs(iv2.lower - iv.lower) <= 1e-12 * abs(iv.lower) and abs(iv2.upper - iv.upper) <= 1e-12 * abs(iv.upper)
    # the paper's construction (column discs of B^{-1} A) holds it too
    lo, hi = ts.gershgorin_columns_interval(A, B)
    assert lo <= lam[0] + 1e-9 and lam[-1] <= hi + 1e-9


def test_gershgorin_diagonal_closed_form():
    rng = np.random.default_rng(3)
    a = rng.normal(size=40) * 3.0
    iv = ts.gershgorin_interval(np.diag(a), np.eye(40), pad=0.0)
    assert iv.lower == a.min() and iv.upper == a.max()
    # B = c I scales the spectrum by 1/c
    iv2 = ts.gershgorin_interval(np.diag(a), 4.0 * np.eye(40), pad=0.0)
    assert np.isclose(iv2.lower, a.min() / 4.0) and np.isclose(iv2.upper, a.max() / 4.0)


def test_multisection_contract_and_bisection(small):
    p, A, B, lam, _ = small
    k = p.k
    iv0 = ts.gershgorin_interval(A, B)
    ops1 = ts.DenseOps(A, B)
    r1 = ts.multisect_mmax(ops1, k, iv0, 20, 1)
    r0 = ts.bisect_mmax(ts.DenseOps(A, B), k, iv0, 20)
    assert (r1.lower, r1.upper, r1.nu_lower, r1.nu_upper) == (r0.lower, r0.upper, r0.nu_lower, r0.nu_upper)
    for s in (3, 8):
        r = ts.multisect_mmax(ts.DenseOps(A, B), k, iv0, 20, s)
        assert r.nu_lower < k <= r.nu_upper and r.nu_upper - r.nu_lower <= 20
        assert r.lower <= lam[k - 1] < r.upper
        assert core.count_below(lam, r.lower) == r.nu_lower and core.count_below(lam, r.upper) == r.nu_upper
        # fewer steps than bisection: each step divides the width by s + 1
        steps = len({round(h[0], 15) for h in r.history})
        assert steps <= s * len(r0.history)


def test_three_stage_gershgorin_multisection(small):
    p, A, B, lam, _ = small
    rng = np.random.default_rng(5)
    r = ts.three_stage(ts.DenseOps(A, B), p.k, rng.normal(size=p.n), rng.normal(size=p.n),
                       init="gershgorin", nshift=8)
    nrm = np.abs(A).sum(1).max()
    assert abs(r.lam - lam[p.k - 1]) <= 1e-10 * nrm
    assert r.initial.nu_lower == 0 and r.initial.nu_upper == p.n


def test_eig_grad_matches_finite_differences():
    rng = np.random.default_rng(11)
    n, k, h = 40, 17, 1e-6
    M = rng.normal(size=(n, n))
    A = 0.5 * (M + M.T)
    R = rng.normal(size=(n, n)) * 0.05
    B = np.eye(n) * 2.0 + 0.5 * (R + R.T)
    lam, GA, GB = core.eig_grad(A, B, k)
    assert np.isclose(lam, core.gen_eig(A, B)[0][k - 1])
    scale = np.abs(GA).max()
    for (i, j) in [(0, 0), (3, 7), (12, 30), (39, 39), (5, 21)]:
        S = np.zeros((n, n)); S[i, j] += 1.0; S[j, i] += 1.0 if i != j else 0.0
        fa = (core.gen_eig(A + h * S, B)[0][k - 1] - core.gen_eig(A - h * S, B)[0][k - 1]) / (2 * h)
        fb = (core.gen_eig(A, B + h * S)[0][k - 1] - core.gen_eig(A, B - h * S)[0][k - 1]) / (2 * h)
        ga = GA[i, j] + (GA[j, i] if i != j else 0.0)
        gb = GB[i, j] + (GB[j, i] if i != j else 0.0)
        assert abs(fa - ga) <= 1e-6 * scale, (i, j, fa, ga)
        assert abs(fb - gb) <= 1e-6 * scale * max(1.0, abs(lam)), (i, j, fb, gb)


class _CountOps:
    """nu(sigma) = #{eigenvalues < sigma} of a sorted array (a count function with no matrix)."""

    def __init__(self, lam):
        self.lam = np.sort(np.asarray(lam, dtype=np.float64))
        self.calls = 0

    def nu(self, s):
        self.calls += 1
        return int(np.searchsorted(self.lam, s, side="left"))


@pytest.mark.parametrize("k", [1234, 5000, 8765])
def test_interp_linear_count_closed_form(k):
    # eigenvalues 1..N: nu is linear between the ends, so linear interpolation lands exactly on the
    # target counts k - 5 and k + 4 (h = m_max / 4 = 5): two steps, from either side
    N = 10000
    ops = _CountOps(np.arange(1, N + 1))
    iv = ts.Interval(0.5, N + 0.5, 0, N)
    r = ts.interp_mmax(ops, k, iv, 20)
    assert len(r.history) == 2
    assert (r.nu_lower, r.nu_upper) == (k - 5, k + 4)
    assert abs(r.lower - (k - 4.5)) < 1e-9 and abs(r.upper - (k + 4.5)) < 1e-9


def test_interp_contract_on_pencil(small):
    p, A, B, lam, _ = small
    k = p.k
    for iv0 in (ts.gershgorin_interval(A, B), ts.lanczos_interval(ts.DenseOps(A, B), k,
                                                                  np.random.default_rng(7).normal(size=p.n))):
        r = ts.interp_mmax(ts.DenseOps(A, B), k, iv0, 20)
        assert r.nu_lower < k <= r.nu_upper and r.nu_upper - r.nu_lower <= 20
        assert r.lower <= lam[k - 1] < r.upper
        assert core.count_below(lam, r.lower) == r.nu_lower and core.count_below(lam, r.upper) == r.nu_upper
        rb = ts.bisect_mmax(ts.DenseOps(A, B), k, iv0, 20)
        assert len(r.history) <= len(rb.history)


@pytest.mark.parametrize("kind", ["cluster", "cauchy", "gap"])
def test_interp_safeguard_bound(kind):
    # spectra that defeat interpolation: a dense cluster beside a sparse part, heavy tails, and a
    # wide gap right above k; the safeguard's midpoint steps keep the count at most about four
    # times bisection's, and the contract holds
    N = 200000
    rng = np.random.default_rng(11)
    if kind == "cluster":
        lam = np.concatenate([np.linspace(0, 1, N // 2), 1 + 1e-7 * np.arange(N - N // 2)])
    elif kind == "cauchy":
        lam = rng.standard_cauchy(N)
    else:
        lam = np.concatenate([rng.uniform(0, 1, N // 2), rng.uniform(50, 51, N - N // 2)])
    lam = np.sort(lam)
    for k in (N // 10, N // 2, N // 2 + 1, 9 * N // 10):
        iv = ts.Interval(lam[0] - 1.0, lam[-1] + 1.0, 0, N)
        ops = _CountOps(lam)
        r = ts.interp_mmax(ops, k, iv, 20)
        rb = ts.bisect_mmax(_CountOps(lam), k, iv, 20)
        assert r.nu_lower < k <= r.nu_upper and r.nu_upper - r.nu_lower <= 20
        assert r.lower <= lam[k - 1] < r.upper
        assert len(r.history) <= 4 * len(rb.history) + 4


def test_three_stage_interp_matches_dense(small):
    p, A, B, lam, _ = small
    rng = np.random.default_rng(5)
    r = ts.three_stage(ts.DenseOps(A, B), p.k, rng.normal(size=p.n), rng.normal(size=p.n), split="interp")
    nrm = np.abs(A).sum(1).max()
    assert abs(r.lam - lam[p.k - 1]) <= 1e-10 * nrm
    assert r.narrowed.nu_upper - r.narrowed.nu_lower <= 20
