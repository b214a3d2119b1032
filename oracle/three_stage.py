"""Oracle three-stage k-th eigenpair method (test infrastructure only).

Algorithms of the paper, step by step and in its notation, on plain operators:
  * ``lanczos_interval``  Algorithm 2 (Section 3.1): an interval containing lambda_k from the
                          extreme Ritz values of the generalized Lanczos decomposition (Eq. 2.2).
  * ``bisect_mmax``       Algorithm 1' (Section 3.3): bisection until nu_u - nu_l <= m_max.
  * ``bisect_straight``   Algorithm 1 (Section 2.1) with the footnote's relative-width stop of
                          Section 4.3.2.
  * ``si_lanczos_kth``    Algorithm 3 (Section 3.2): shift-and-invert Lanczos (Eq. 2.5) with the
                          modified Ritz vectors x_{i,2} (Eq. 2.9), the error bound of Proposition 3
                          (Eq. 3.1), inclusion (3.3), disjointness (3.4), residual and relative
                          difference (Eq. 3.5) tests.
  * ``three_stage``       Algorithm 4 (Section 3.4), optionally with the Gershgorin initial
                          interval of the variant of Section 4.2 and multisection in Algorithm 1'.
  * ``gershgorin_interval``          an interval holding the whole spectrum from Gershgorin bounds
                          of A and B and the Rayleigh quotient (the reading the GPU path uses);
    ``gershgorin_columns_interval``  the paper's construction: Gershgorin discs of the columns of
                          B^{-1} A (Section 4.2, dense, small n).
  * ``multisect_mmax``    Algorithm 1' with s points per step (s + 1 equal parts; s = 1 is
                          bisection).
  * ``interp_mmax``       Algorithm 1' with the shift chosen by a bracketed, derivative-free
                          root-finder on the count function nu(sigma) instead of the midpoint: the
                          variant Section 2.1 describes and Section 5 proposes (any derivative-free
                          method that keeps the root bracketed locates lambda_k).  The rule itself
                          is this project's; its output contract is Algorithm 1''s.

Operators come from ``DenseOps`` (dense numpy, small n) or ``SparseOps`` (scipy sparse LU for
solves, (c3) for inertia).  Library solves serve as steps; the method's arithmetic is here.

Readings where the paper is silent:
  * random start vectors are N(0, 1) entries; callers may pass them in (the GPU path takes the same);
  * "with reorthogonalization" = full classical Gram-Schmidt applied twice, in the inner product the
    decomposition is orthonormal in (B for Eq. 2.2, B^{-1} for Eq. 2.5);
  * the relative difference (Eq. 3.5) compares the i-th pair of iteration j with the i-th pair of
    iteration j-1 in the distance-to-sigma order of Eq. 3.2, after scaling x^{(j)} to the 2-norm of
    x^{(j-1)} and choosing the sign that makes their inner product non-negative.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import core


class DenseOps:
    """Dense operators for small n: A, B as arrays, nu by (c1), solves by LU."""

    def __init__(self, A: np.ndarray, B: np.ndarray):
        self.A = np.asarray(A, dtype=np.float64)
        self.B = np.asarray(B, dtype=np.float64)
        self.n = self.A.shape[0]
        self.nfactor = 0
        self._Bcho = None

    def nu(self, sigma: float) -> int:
        self.nfactor += 1
        return core.dense_nu(self.A, self.B, sigma)

    def matA(self, x): return self.A @ x
    def matB(self, x): return self.B @ x
    def solveB(self, x):
        if self._Bcho is None:
            self._Bcho = sla.cho_factor(self.B, lower=True)
        return sla.cho_solve(self._Bcho, x)

    def shifted_solver(self, sigma: float):
        lu = sla.lu_factor(self.A - sigma * self.B)
        return lambda x: sla.lu_solve(lu, x)


class SparseOps:
    """Sparse operators: nu by (c3), solves by sparse LU (a library primitive)."""

    def __init__(self, pencil):
        self.p = pencil
        self.A = pencil.A().tocsc()
        self.B = pencil.B().tocsc()
        self.n = pencil.n
        self._Blu = None
        self.nfactor = 0

    def nu(self, sigma: float) -> int:
        self.nfactor += 1
        return core.sparse_nu(self.p, sigma)

    def matA(self, x): return self.A @ x
    def matB(self, x): return self.B @ x

    def solveB(self, x):
        if self._Blu is None:
            self._Blu = spla.splu(self.B)
        return self._Blu.solve(x)

    def shifted_solver(self, sigma: float):
        lu = spla.splu((self.A - sigma * self.B).tocsc())
        return lu.solve


@dataclass
class Interval:
    lower: float
    upper: float
    nu_lower: int
    nu_upper: int
    history: list = field(default_factory=list)   # (sigma, nu) per factorization


def lanczos_interval(ops, k: int, v1: np.ndarray, max_iter: int = 200) -> Interval:
    """Algorithm 2: interval [sigma_l, sigma_u) containing lambda_k from extreme Ritz values.

    j-step generalized Lanczos decomposition A V_j = B V_j T_j + B v_{j+1} beta_j e_j^T (Eq. 2.2),
    V_j B-orthonormal; sigma^(j) = theta_1^(j) if k <= nu^(j-1) else theta_j^(j); stop at j != 1
    once nu brackets k."""
    v = v1 / np.sqrt(v1 @ ops.matB(v1))            # v_1 := v_1 / ||v_1||_B
    V = [v]
    alpha, beta = [], []
    nu_prev, sig_prev = 0, None                    # nu^(0) := 0
    hist = []
    for j in range(1, max_iter + 1):
        # extend the decomposition by one step: w = B^{-1} A v_j - beta_{j-1} v_{j-1}
        vj = V[-1]
        w = ops.solveB(ops.matA(vj))
        if j > 1:
            w = w - beta[-1] * V[-2]
        a = float(vj @ ops.matA(vj))               # alpha_j = v_j^T A v_j
        alpha.append(a)
        w = w - a * vj
        Vm = np.stack(V, 1)
        for _ in range(2):                         # reorthogonalize in the B inner product
            w = w - Vm @ (Vm.T @ ops.matB(w))
        b = float(np.sqrt(w @ ops.matB(w)))
        beta.append(b)
        V.append(w / b)
        # Ritz values: eigenvalues of the j x j tridiagonal T_j (Eq. 2.3)
        T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
        theta = np.linalg.eigvalsh(T)
        sig = theta[0] if k <= nu_prev else theta[-1]
        nu = ops.nu(sig)
        hist.append((sig, nu))
        if j != 1 and (nu < k <= nu_prev or nu_prev < k <= nu):
            return Interval(min(sig_prev, sig), max(sig_prev, sig), min(nu_prev, nu),
                            max(nu_prev, nu), hist)
        nu_prev, sig_prev = nu, sig
    raise RuntimeError("Algorithm 2 did not bracket k")


def bisect_mmax(ops, k: int, iv: Interval, m_max: int = 20) -> Interval:
    """Algorithm 1': halve [sigma_l, sigma_u) until it holds at most m_max eigenvalues."""
    lo, hi, nl, nu_u = iv.lower, iv.upper, iv.nu_lower, iv.nu_upper
    hist = []
    while nu_u - nl > m_max:
        s = 0.5 * (lo + hi)
        nu = ops.nu(s)
        hist.append((s, nu))
        if k <= nu:
            hi, nu_u = s, nu
        else:
            lo, nl = s, nu
    return Interval(lo, hi, nl, nu_u, hist)


def multisect_mmax(ops, k: int, iv: Interval, m_max: int = 20, nshift: int = 1) -> Interval:
    """Algorithm 1' with nshift shifts per step: [sigma_l, sigma_u) is cut into nshift + 1 equal
    parts and the one with nu(left) < k <= nu(right) is kept, until nu_u - nu_l <= m_max.  With
    nshift = 1 the shift is the midpoint (bisection)."""
    lo, hi, nl, nu_u = iv.lower, iv.upper, iv.nu_lower, iv.nu_upper
    hist = []
    while nu_u - nl > m_max:
        plo, phi, pnl, pnu = lo, hi, nl, nu_u
        for q in range(1, nshift + 1):
            s = 0.5 * (lo + hi) if nshift == 1 else lo + (hi - lo) * q / (nshift + 1)
            nu = ops.nu(s)
            hist.append((s, nu))
            if k <= nu:
                phi, pnu = s, nu
                break
            plo, pnl = s, nu
        lo, hi, nl, nu_u = plo, phi, pnl, pnu
    return Interval(lo, hi, nl, nu_u, hist)


def gershgorin_interval(A, B, pad: float = 1e-12) -> Interval:
    """An interval holding every eigenvalue of A x = lambda B x.

    Each eigenvalue is a Rayleigh quotient x^T A x / x^T B x.  Gershgorin's theorem bounds the
    spectra of A and B: loA <= x^T A x / x^T x <= hiA, 0 < loB <= x^T B x / x^T x <= hiB (B's
    lower bound must be positive).  Hence lambda >= loA / (loB if loA < 0 else hiB) and
    lambda <= hiA / (loB if hiA > 0 else hiB).  The ends are widened by pad * max(|lo|, |hi|, 1)
    so that nu(lower) = 0 and nu(upper) = n."""
    def bounds(M):
        M = M.tocsr() if hasattr(M, "tocsr") else np.asarray(M)
        d = M.diagonal() if hasattr(M, "diagonal") else np.diag(M)
        r = np.asarray(abs(M).sum(axis=1)).ravel() - np.abs(d)
        return float(np.min(d - r)), float(np.max(d + r))
    loA, hiA = bounds(A)
    loB, hiB = bounds(B)
    if not loB > 0.0:
        raise ValueError("B's Gershgorin lower bound is not positive")
    lo = loA / (loB if loA < 0 else hiB)
    hi = hiA / (loB if hiA > 0 else hiB)
    w = pad * max(abs(lo), abs(hi), 1.0)
    n = A.shape[0]
    return Interval(lo - w, hi + w, 0, n, [])


def gershgorin_columns_interval(A: np.ndarray, B: np.ndarray) -> tuple[float, float]:
    """The construction of the Gershgorin variant of Section 4.2: the columns of C = B^{-1} A
    (linear solves), then the union of the column discs |z - c_jj| <= sum_{i != j} |c_ij|, whose
    real extent holds the spectrum of B^{-1} A."""
    C = np.linalg.solve(np.asarray(B, dtype=np.float64), np.asarray(A, dtype=np.float64))
    d = np.diag(C)
    r = np.abs(C).sum(axis=0) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def bisect_straight(ops, k: int, lo: float, hi: float, rel_tol: float = 1e-14,
                    max_iter: int = 200):
    """Algorithm 1 with the stop (sigma_u - sigma_l)/max(|sigma_l|, |sigma_u|) < rel_tol of the
    footnote in Section 4.3.2.  Returns (lambda_hat, iterations)."""
    it = 0
    while (hi - lo) / max(abs(lo), abs(hi)) >= rel_tol and it < max_iter:
        s = 0.5 * (lo + hi)
        if k <= ops.nu(s):
            hi = s
        else:
            lo = s
        it += 1
    return 0.5 * (lo + hi), it


class SIState:
    """The j-step SI Lanczos decomposition of Eq. 2.5, extended one step at a time.

    Vt: columns v~_1 .. v~_{j+1} (B^{-1}-orthonormal); W: (A - sigma B)^{-1} v~_i for i <= j;
    alpha/beta: the diagonal and off-diagonal of T~_j (beta[-1] = beta~_j)."""

    def __init__(self, ops, solve, vt1: np.ndarray):
        self.ops, self.solve = ops, solve
        binv = ops.solveB
        self.Vt = [vt1 / np.sqrt(vt1 @ binv(vt1))]  # v~_1 := v~_1 / ||v~_1||_{B^{-1}}
        self.W, self.alpha, self.beta = [], [], []

    def step(self):
        ops, binv, Vt = self.ops, self.ops.solveB, self.Vt
        vj = Vt[-1]
        wj = self.solve(vj)                        # (A - sigma B)^{-1} v~_j
        self.W.append(wj)
        a = float(vj @ wj)                         # alpha~_j = v~_j^T (A - sigma B)^{-1} v~_j
        r = ops.matB(wj) - a * vj                  # B (A - sigma B)^{-1} v~_j - alpha v~_j - beta v~_{j-1}
        if len(self.beta):
            r = r - self.beta[-1] * Vt[-2]
        Vm = np.stack(Vt, 1)
        for _ in range(2):                         # reorthogonalize in the B^{-1} inner product
            r = r - Vm @ (Vm.T @ binv(r))
        b = float(np.sqrt(r @ binv(r)))
        self.alpha.append(a); self.beta.append(b)
        Vt.append(r / b)

    def T(self) -> np.ndarray:
        a, b = self.alpha, self.beta
        return np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)


@dataclass
class KthResult:
    lam: float
    x: np.ndarray                 # B-normalized (x^T B x = 1)
    index_in_interval: int        # l
    m: int
    iterations: int
    eta: float
    rel_res: float                # ||(A - lam B) x||_2 / ||x||_2 (the paper's quantity)
    iters_bound: int = -1         # first j at which inclusion and disjointness held
    lams: np.ndarray | None = None


def si_lanczos_kth(ops, k: int, iv: Interval, vt1: np.ndarray, tau_res: float = 1e-10,
                   tau_diff: float = 1e-10, max_iter: int = 300) -> KthResult:
    """Algorithm 3: k-th eigenpair with index validation.

    SI Lanczos decomposition (A - sigma B)^{-1} V~_j = B^{-1} V~_j T~_j + B^{-1} v~_{j+1} beta~_j e_j^T
    (Eq. 2.5), V~_j B^{-1}-orthonormal.  Ritz values lambda_i = sigma + 1/theta~_i (Eq. 2.7), modified
    Ritz vectors x_{i,2} = (A - sigma B)^{-1} V~_j y~_i (Eq. 2.9), bounds eta_i (Eq. 3.1)."""
    l = k - iv.nu_lower
    m = iv.nu_upper - iv.nu_lower
    sigma = 0.5 * (iv.lower + iv.upper)
    solve = ops.shifted_solver(sigma)
    st = SIState(ops, solve, vt1)
    Vt, W, alpha, beta = st.Vt, st.W, st.alpha, st.beta
    prev_x = None
    iters_bound = -1
    for j in range(1, max_iter + 1):
        st.step()
        b = beta[-1]
        if j < m:
            continue
        T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
        theta, Y = np.linalg.eigh(T)               # Eq. 2.6, y~_i 2-normalized
        lam = sigma + 1.0 / theta                  # Eq. 2.7
        order = np.argsort(-np.abs(theta), kind="stable")   # Eq. 3.2
        theta, Y, lam = theta[order], Y[:, order], lam[order]
        Wm = np.stack(W, 1)
        X = Wm @ Y                                 # x_{i,2} = (A - sigma B)^{-1} V~_j y~_i (Eq. 2.9)
        rho = np.abs(b * Y[-1, :] / theta)         # |beta~_j e_j^T y~_i / theta~_i|
        eta = (1.0 / np.abs(theta)) * rho / np.sqrt(1.0 + rho * rho)    # Eq. 3.1
        lo_b, hi_b = lam[:m] - eta[:m], lam[:m] + eta[:m]
        inclusion = bool(np.all(lo_b >= iv.lower) and np.all(hi_b < iv.upper))   # (3.3)
        srt = np.argsort(lam[:m])
        disjoint = bool(np.all(hi_b[srt][:-1] < lo_b[srt][1:]))                   # (3.4)
        if inclusion and disjoint and iters_bound < 0:
            iters_bound = j
        ok = inclusion and disjoint
        res = np.zeros(m)
        for i in range(m):
            xi = X[:, i]
            res[i] = np.linalg.norm(ops.matA(xi) - lam[i] * ops.matB(xi)) / np.linalg.norm(xi)
        ok = ok and bool(np.all(res < tau_res))
        diff_ok = prev_x is not None
        if diff_ok:
            for i in range(m):
                xo = prev_x[:, i]
                xn = X[:, i] * (np.linalg.norm(xo) / np.linalg.norm(X[:, i]))
                if xn @ xo < 0:
                    xn = -xn
                if np.linalg.norm(xn - xo) / np.linalg.norm(xo) >= tau_diff:   # Eq. 3.5
                    diff_ok = False
                    break
        prev_x = X[:, :m].copy()
        if ok and diff_ok:
            srt = np.argsort(lam[:m])              # back to increasing order
            i = srt[l - 1]
            x = X[:, i]
            x = x / np.sqrt(x @ ops.matB(x))
            return KthResult(lam=float(lam[i]), x=x, index_in_interval=l, m=m, iterations=j,
                             eta=float(eta[i]), rel_res=float(res[i]), iters_bound=iters_bound,
                             lams=np.sort(lam[:m]))
    raise RuntimeError("Algorithm 3 did not validate the interval's eigenpairs")


class InterpBracket:
    """State of the interpolating shift rule for Algorithm 1' (see ``interp_mmax``).

    The bracket is [lower, upper) with nu(lower) = nu_lower < k <= nu_upper = nu(upper).  w_lower
    and w_upper are the counts the interpolation assigns to the two ends: the true counts, except
    that an end kept through two consecutive steps has its distance to k halved (the Illinois
    modification of regula falsi, which stops one far end from holding the interpolant back).
    widths holds the count widths nu_upper - nu_lower after each step (the first entry is the
    initial width); bisect_next marks the safeguard's midpoint step."""

    def __init__(self, k: int, lower: float, upper: float, nu_lower: int, nu_upper: int):
        if not (lower < upper and nu_lower < k <= nu_upper):
            raise ValueError("not a bracket of k")
        self.lower, self.upper = float(lower), float(upper)
        self.nu_lower, self.nu_upper = int(nu_lower), int(nu_upper)
        self.w_lower, self.w_upper = float(nu_lower), float(nu_upper)
        self.widths = [self.nu_upper - self.nu_lower]
        self.last = 0
        self.bisect_next = False

    def point(self, k: int, m_max: int) -> float:
        """The next shift.  The end farther from k in count is the one to move: the target count is
        k - h below k (to move the lower end) or k - 1 + h (to move the upper end), h = m_max // 4
        (at least 1), so that the moved end lands inside the final window.  Its shift is the linear
        interpolation of sigma between the ends at their weighted counts, kept at least 2^-20 of the
        bracket away from either end.  A safeguard step takes the midpoint instead."""
        lo, hi = self.lower, self.upper
        if self.bisect_next:
            return 0.5 * (lo + hi)
        h = max(1, m_max // 4)
        move_lower = (k - self.nu_lower) > (self.nu_upper - k)
        t = float(k - h) if move_lower else float(k - 1 + h)
        t = min(max(t, self.w_lower + 0.5), self.w_upper - 0.5)
        frac = (t - self.w_lower) / (self.w_upper - self.w_lower)
        s = lo + frac * (hi - lo)
        g = (hi - lo) / 1048576.0
        return min(max(s, lo + g), hi - g)

    def update(self, k: int, sigma: float, nu: int) -> None:
        """Replace the end on sigma's side by (sigma, nu(sigma)); the safeguard bisects once when
        the count width has not halved over the last three steps."""
        if not (self.lower < sigma < self.upper and self.nu_lower <= nu <= self.nu_upper):
            raise ValueError("shift outside the bracket or count not monotone")
        was_bisect = self.bisect_next
        if k <= nu:
            self.upper, self.nu_upper, self.w_upper = sigma, int(nu), float(nu)
            if self.last > 0 and not was_bisect:
                self.w_lower = k - 0.5 * (k - self.w_lower)
            self.last = 1
        else:
            self.lower, self.nu_lower, self.w_lower = sigma, int(nu), float(nu)
            if self.last < 0 and not was_bisect:
                self.w_upper = k + 0.5 * (self.w_upper - k)
            self.last = -1
        self.widths.append(self.nu_upper - self.nu_lower)
        w = self.widths
        self.bisect_next = (not was_bisect) and len(w) > 3 and 2 * w[-1] > w[-4]


def interp_mmax(ops, k: int, iv: Interval, m_max: int = 20) -> Interval:
    """Algorithm 1' with the interpolating shift rule (``InterpBracket``): until the interval holds
    at most m_max eigenvalues, factor at the rule's shift and keep the side that brackets k.  Like
    bisection it only needs nu at each shift, and the output interval satisfies the same contract
    nu_l < k <= nu_u, nu_u - nu_l <= m_max."""
    st = InterpBracket(k, iv.lower, iv.upper, iv.nu_lower, iv.nu_upper)
    hist = []
    while st.nu_upper - st.nu_lower > m_max:
        s = st.point(k, m_max)
        nu = ops.nu(s)
        hist.append((s, nu))
        st.update(k, s, nu)
    return Interval(st.lower, st.upper, st.nu_lower, st.nu_upper, hist)


@dataclass
class ThreeStageResult:
    lam: float
    x: np.ndarray
    initial: Interval
    narrowed: Interval
    kth: KthResult
    nfactor: int


def three_stage(ops, k: int, v1: np.ndarray, vt1: np.ndarray, m_max: int = 20,
                tau_res: float = 1e-10, tau_diff: float = 1e-10, init: str = "lanczos",
                nshift: int = 1, split: str = "bisect") -> ThreeStageResult:
    """Algorithm 4: Algorithm 2 (or the Gershgorin interval of the variant), then Algorithm 1'
    (bisection, multisection with nshift points, or the interpolating shift rule for
    split="interp"), then Algorithm 3."""
    iv0 = gershgorin_interval(ops.A, ops.B) if init == "gershgorin" else lanczos_interval(ops, k, v1)
    if split == "interp":
        iv1 = interp_mmax(ops, k, iv0, m_max)
    else:
        iv1 = multisect_mmax(ops, k, iv0, m_max, nshift)
    res = si_lanczos_kth(ops, k, iv1, vt1, tau_res, tau_diff)
    return ThreeStageResult(lam=res.lam, x=res.x, initial=iv0, narrowed=iv1, kth=res,
                            nfactor=ops.nfactor)
