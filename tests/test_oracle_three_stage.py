"""Pins for the oracle's Algorithms 1, 1', 2, 3 and 4 and Propositions 1-3 (no GPU).

The contracts come from the paper's statements: Algorithm 2 returns an interval with
nu_l < k <= nu_u; Algorithm 1' stops with nu_u - nu_l <= m_max; Algorithm 3 returns a pair with
relative residual < tau_res; Propositions 1-3 are identities / bounds checked here explicitly
against quantities the oracle computes by a different route (dense solves)."""
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


def test_three_stage_matches_dense(small):
    p, A, B, lam, X = small
    ops = ts.DenseOps(A, B)
    rng = np.random.default_rng(1)
    k = p.k
    r = ts.three_stage(ops, k, rng.normal(size=p.n), rng.normal(size=p.n))
    nrm = np.abs(A).sum(1).max()
    # Algorithm 2 contract and interval contents
    assert r.initial.nu_lower < k <= r.initial.nu_upper
    assert r.initial.nu_lower == core.count_below(lam, r.initial.lower)
    assert r.initial.nu_upper == core.count_below(lam, r.initial.upper)
    assert len(r.initial.history) >= 2
    # Algorithm 1' contract
    assert r.narrowed.nu_upper - r.narrowed.nu_lower <= 20
    assert r.narrowed.lower <= lam[k - 1] < r.narrowed.upper
    # Algorithm 3 / 4
    assert abs(r.lam - lam[k - 1]) <= 1e-10 * nrm
    assert r.kth.rel_res < 1e-10
    assert abs(r.x @ B @ r.x - 1) < 1e-12
    xd = X[:, k - 1]
    x = r.x * np.sign(r.x @ B @ xd)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    assert r.kth.lams.size == r.kth.m
    # every interval eigenvalue recovered
    inside = lam[(lam >= r.narrowed.lower) & (lam < r.narrowed.upper)]
    assert np.abs(np.sort(r.kth.lams) - inside).max() <= 1e-10 * nrm


def test_straight_bisection(small):
    p, A, B, lam, X = small
    ops = ts.DenseOps(A, B)
    lo, hi = lam[0] - 1, lam[-1] + 1
    lam_hat, it = ts.bisect_straight(ops, p.k, lo, hi, rel_tol=1e-12)
    assert abs(lam_hat - lam[p.k - 1]) <= 1e-12 * max(abs(lo), abs(hi))
    assert it >= 30


def _si_quantities(A, B, sigma, j, seed=0):
    ops = ts.DenseOps(A, B)
    st = ts.SIState(ops, ops.shifted_solver(sigma), np.random.default_rng(seed).normal(size=A.shape[0]))
    for _ in range(j):
        st.step()
    theta, Y = np.linalg.eigh(st.T())
    Vt = np.stack(st.Vt[:-1], 1)
    vnext = st.Vt[-1]
    return st, theta, Y, Vt, vnext


def test_decomposition_eq_2_5(small):
    """(A - sigma B)^{-1} V~ = B^{-1} V~ T~ + B^{-1} v~_{j+1} beta~ e_j^T and B^{-1}-orthonormality."""
    p, A, B, lam, X = small
    sigma = 0.5 * (lam[p.k - 1] + lam[p.k])
    st, theta, Y, Vt, vnext = _si_quantities(A, B, sigma, 12)
    M = A - sigma * B
    lhs = np.linalg.solve(M, Vt)
    e = np.zeros(12); e[-1] = 1
    rhs = np.linalg.solve(B, Vt @ st.T() + np.outer(vnext * st.beta[-1], e))
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(lhs).max()
    Binv = np.linalg.inv(B)
    V1 = np.column_stack([Vt, vnext])
    assert np.abs(V1.T @ Binv @ V1 - np.eye(13)).max() < 1e-10


def test_proposition_1_2_3_and_residual_identity(small):
    p, A, B, lam, X = small
    sigma = 0.5 * (lam[p.k - 1] + lam[p.k])
    j = 15
    st, theta, Y, Vt, vnext = _si_quantities(A, B, sigma, j, seed=3)
    M = A - sigma * B
    bj = st.beta[-1]
    X1 = np.linalg.solve(B, Vt @ Y)          # x_{i,1} (Eq. 2.8)
    X2 = np.linalg.solve(M, Vt @ Y)          # x_{i,2} (Eq. 2.9), by explicit solves
    # Proposition 1 (its proof's identity): x_{i,2} = theta_i x_{i,1} + B^{-1} v~_{j+1} beta~ y_{j,i}
    rec = X1 * theta + np.outer(np.linalg.solve(B, vnext), bj * Y[-1, :])
    assert np.abs(rec - X2).max() < 1e-9 * np.abs(X2).max()
    # residual identity r_{i,2} = -v~_{j+1} (beta~ e_j^T y~_i / theta~_i)
    lam_i = sigma + 1.0 / theta
    R = A @ X2 - (B @ X2) * lam_i
    Rid = -np.outer(vnext, bj * Y[-1, :] / theta)
    assert np.abs(R - Rid).max() < 1e-9 * np.abs(R).max()
    # Proposition 2: B-cosine between x_{l,2} and x_{m,2}
    rho = np.abs(bj * Y[-1, :] / theta)
    g = rho / np.sqrt(1 + rho ** 2)
    G = X2.T @ B @ X2
    nb = np.sqrt(np.diag(G))
    checked = 0
    for l_ in range(j):
        for m_ in range(l_ + 1, j):
            pred = g[l_] * g[m_]
            cos = abs(G[l_, m_]) / (nb[l_] * nb[m_])
            # rounding floor of the explicit cosine is ~1e-13; compare where the closed form is above
            if pred > 1e-8:
                assert abs(cos - pred) <= 1e-6 * pred
                checked += 1
            else:
                assert cos < 1e-8
    assert checked >= 5
    # Proposition 3: eta_i = ||r_{i,2}||_{B^{-1}} / ||x_{i,2}||_B, and the bound holds
    eta = (1 / np.abs(theta)) * rho / np.sqrt(1 + rho ** 2)
    Binv = np.linalg.inv(B)
    eta_explicit = np.sqrt(np.einsum("ij,ij->j", R, Binv @ R)) / nb
    # explicit residuals of converged pairs sit at the rounding floor (~1e-14 * ||A||)
    assert np.allclose(eta, eta_explicit, rtol=1e-6, atol=1e-12)
    assert np.sum(eta > 1e-6) >= 5
    for i in range(j):
        assert np.min(np.abs(lam - lam_i[i])) <= eta[i] * (1 + 1e-8) + 1e-13
