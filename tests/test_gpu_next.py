"""GPU parity of the next rows: Hellmann-Feynman derivatives (kep_grad, the torch autograd wrapper),
new values on an analysed pattern (kep_set_values), the Gershgorin initial interval and
multisection in Algorithm 4, and kep_factor_multi.

References: the oracle's dense generalized eigensolver (c2) and its derivative formula (pinned by
finite differences in test_oracle_next.py), and the oracle's Gershgorin interval."""
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
def pen():
    p = make_pair(3, 3, 2, seed=21)          # n = 576
    A, B = p.A().toarray(), p.B().toarray()
    lam, X = core.gen_eig(A, B)
    return p, A, B, lam, X


def _entries(p):
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    return rows, p.colind


def test_grad_full_pattern(kep, pen):
    p, A, B, lam, X = pen
    k = p.k
    with kep.Problem.from_pencil(p) as P:
        lam_g, x, _ = P.kth_eigenpair(k)
        ga, gb = P.grad(lam_g, x, 1.0)
    _, GA, GB = core.eig_grad(A, B, k)
    r, c = _entries(p)
    scale = np.abs(GA).max()
    assert np.abs(ga - GA[r, c]).max() <= 1e-8 * scale
    assert np.abs(gb - GB[r, c]).max() <= 1e-8 * scale * max(1.0, abs(lam[k - 1]))
    # lambda_bar scales both
    with kep.Problem.from_pencil(p) as P:
        ga3, _ = P.grad(lam_g, 2.0 * x, 3.0)   # any scaling of x
    assert np.abs(ga3 - 3.0 * ga).max() <= 1e-12 * scale


def test_grad_lower_pattern_device(kep, pen):
    import torch
    p, A, B, lam, X = pen
    k = p.k + 3
    rows, cols = _entries(p)
    keep = cols <= rows
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=p.n))])
    with kep.Problem(p.n, rp, cols[keep], p.a[keep], p.b[keep], p.coords, lower=True) as P:
        lam_g, x, _ = P.kth_eigenpair(k)
        ga, gb = P.grad(lam_g, torch.from_numpy(x).cuda(), 1.0)
    _, GA, GB = core.eig_grad(A, B, k)
    r, c = rows[keep], cols[keep]
    want = GA[r, c] * np.where(r != c, 2.0, 1.0)
    scale = np.abs(GA).max()
    assert np.abs(ga.cpu().numpy() - want).max() <= 1e-8 * scale
    assert np.abs(gb.cpu().numpy() + lam[k - 1] * want).max() <= 1e-8 * scale * max(1.0, abs(lam[k - 1]))


def test_autograd_and_set_values(kep, pen):
    import torch
    p, A, B, lam, X = pen
    k = p.k
    a = torch.tensor(p.a, requires_grad=True)
    b = torch.tensor(p.b, requires_grad=True)
    with kep.Problem.from_pencil(p) as P:
        lam_t = kep.KthEigenvalue.apply(P, k, a, b)
        (2.0 * lam_t).backward()
        assert abs(float(lam_t.detach()) - lam[k - 1]) <= 1e-10 * np.abs(A).sum(1).max()
        _, GA, GB = core.eig_grad(A, B, k)
        r, c = _entries(p)
        scale = np.abs(GA).max()
        assert np.abs(a.grad.numpy() - 2.0 * GA[r, c]).max() <= 1e-8 * scale
        # new values on the same pattern: A -> 2 A doubles every eigenvalue (closed form)
        P.set_values(2.0 * p.a, p.b)
        lam2, _, _ = P.kth_eigenpair(k)
        assert abs(lam2 - 2.0 * lam[k - 1]) <= 2e-10 * np.abs(A).sum(1).max()
        sig = 2.0 * 0.5 * (lam[k - 1] + lam[k])
        assert P.factor(sig).neg == core.count_below(2.0 * lam, sig)


def test_gershgorin_multisection_driver(kep, pen):
    p, A, B, lam, X = pen
    k = p.k
    nrm = np.abs(A).sum(1).max()
    iv = ts.gershgorin_interval(A, B)
    with kep.Problem.from_pencil(p) as P:
        for nshift in (1, 8):
            lam_g, x, rep = P.kth_eigenpair(k, init="gershgorin", nshift=nshift)
            assert abs(lam_g - lam[k - 1]) <= 1e-10 * nrm
            assert rep["init_nu_lo"] == 0 and rep["init_nu_hi"] == p.n
            assert abs(rep["init_lo"] - iv.lower) <= 1e-12 * abs(iv.lower)
            assert abs(rep["init_hi"] - iv.upper) <= 1e-12 * abs(iv.upper)
            assert rep["nu_lo"] < k <= rep["nu_hi"] and rep["nu_hi"] - rep["nu_lo"] <= 20
            assert core.count_below(lam, rep["sigma_lo"]) == rep["nu_lo"]
            assert core.count_below(lam, rep["sigma_hi"]) == rep["nu_hi"]
            if nshift == 8:
                # the oracle's multisection from the same interval ends in the same place
                r = ts.multisect_mmax(ts.DenseOps(A, B), k, iv, 20, 8)
                assert (r.nu_lower, r.nu_upper) == (rep["nu_lo"], rep["nu_hi"])


def test_factor_multi(kep, pen):
    p, A, B, lam, X = pen
    sig = core.certified_shifts(lam, 6, 1e-8 * np.abs(A).sum(1).max(), seed=4)
    with kep.Problem.from_pencil(p) as P:
        res = P.factor_multi(sig)
        assert [r.neg for r in res] == [core.count_below(lam, s) for s in sig]
        assert all(r.neg + r.zero + r.pos == p.n for r in res)
        # the last factor stays for solve
        rhs = np.random.default_rng(2).normal(size=p.n)
        y = P.solve(rhs)
        M = A - sig[-1] * B
        assert np.linalg.norm(M @ y - rhs) <= 1e-11 * np.abs(M).sum(1).max() * np.linalg.norm(y)


def test_factor_multi_batched_closed_form_and_groups(kep):
    """kep_factor_multi factors up to 8 shifts in the same launches (each shift its own slot and
    contribution blocks; the tensor-core update batched over all shifts' fronts).  Counts equal the
    closed-form spectrum (n = 16,384 perfect diamond) for 8 shifts in one group, and for 11 shifts
    (groups of 6 and 5); the last shift's factor stays for the solve."""
    from gen import perfect_diamond_pencil
    q = perfect_diamond_pencil(8, 8, 8)
    cf = core.diamond_bloch_eigs(8, 8, 8, 1.0, 0.02)
    with kep.Problem.from_pencil(q) as P:
        P.set_schur_mode(True, min_front=512)
        for count in (8, 11):
            sig = core.certified_shifts(cf, count, 1e-6, seed=10 + count)
            res = P.factor_multi(sig)
            assert [r.neg for r in res] == [core.count_below(cf, s) for s in sig]
            assert all(r.neg + r.zero + r.pos == q.n for r in res)
        rhs = np.random.default_rng(3).normal(size=q.n)
        y = P.solve(rhs)
        M = (q.A() - sig[-1] * q.B()).tocsr()
        assert np.linalg.norm(M @ y - rhs) <= 1e-12 * abs(M).sum(1).max() * np.linalg.norm(y)
        # the same shifts one by one give the same counts (and the slot is reusable afterwards)
        seq = [P.factor(s).neg for s in sig]
        assert seq == [r.neg for r in res]


def test_factor_multi_delays_and_hermitian(kep):
    """Batched shifts with forced 2x2 pivots and delayed columns (zero diagonal of A - sigma B at
    the first shift) match the oracle's dense Bunch-Kaufman counts; a complex Hermitian pencil's
    batched counts match its dense spectrum."""
    import scipy.sparse as sp
    p = make_pair(4, 4, 4, seed=6)            # n = 2048
    sigma = 0.3
    a = p.a.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    d = rows == p.colind
    a[d] = sigma * p.b[d]
    A = sp.csr_matrix((a, p.colind, p.rowptr), shape=(p.n, p.n)).toarray()
    B = p.B().toarray()
    sig = [sigma, sigma + 0.2, sigma - 0.7, sigma + 1.1]
    with kep.Problem(p.n, p.rowptr, p.colind, a, p.b, p.coords) as P:
        P.set_schur_mode(True, min_front=256)
        res = P.factor_multi(sig)
        for s, r in zip(sig, res):
            assert (r.neg, r.zero, r.pos) == core.dense_inertia(A - s * B), s
    h = make_pair(3, 3, 2, seed=21, phases="peierls")          # n = 576 complex
    Ah, Bh = h.A().toarray(), h.B().toarray()
    lam, _ = core.gen_eig(Ah, Bh)
    hs = core.certified_shifts(lam, 5, 1e-8 * np.abs(Ah).sum(1).max(), seed=13)
    with kep.Problem.from_pencil(h) as H:
        res = H.factor_multi(hs)
        assert [r.neg for r in res] == [core.count_below(lam, s) for s in hs]


def test_fp32_factor_refined_solves(kep, pen):
    p, A, B, lam, X = pen
    sig = float(core.certified_shifts(lam, 1, 1e-6 * np.abs(A).sum(1).max(), seed=8)[0])
    M = A - sig * B
    rhs = np.random.default_rng(3).normal(size=p.n)
    x_ref = np.linalg.solve(M, rhs)
    nM = np.abs(M).sum(1).max()
    with kep.Problem.from_pencil(p) as P:
        P.set_schur_mode(False, fp32=True)
        P.factor(sig)
        x0 = P.solve(rhs)                       # the reduced-precision factor alone
        be0 = np.abs(rhs - M @ x0).max() / (nM * np.abs(x0).max() + np.abs(rhs).max())
        x, it, be = P.solve_refined(rhs, tol=1e-13)
        be_own = np.abs(rhs - M @ x).max() / (nM * np.abs(x).max() + np.abs(rhs).max())
    assert be0 > 1e-12                          # FP32 Schur arithmetic shows without refinement
    assert be <= 1e-13 and be_own <= 2e-13 and 1 <= it <= 10
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-10


def test_fp32_tensor_core_factor_refined_solves(kep):
    """The reduced-precision factor with fronts on the tensor cores (4-digit splitting, fronts of
    order >= 64 here): its plain solve shows the reduced precision, its refined solves reach a
    backward error of 1e-13 and the oracle's dense solution; the FP64-accurate factor afterwards is
    unaffected (its counts equal the dense spectrum's)."""
    p = workload("small")                     # n = 2,048
    A, B = p.A().toarray(), p.B().toarray()
    lam, _ = core.gen_eig(A, B)
    nrm = np.abs(A).sum(1).max()
    sig = float(core.certified_shifts(lam, 1, 1e-6 * nrm, seed=19)[0])
    M = A - sig * B
    nM = np.abs(M).sum(1).max()
    rng = np.random.default_rng(5)
    with kep.Problem.from_pencil(p) as P:
        P.set_schur_mode(False, min_front=64, fp32=True)
        P.factor(sig)
        for _ in range(2):
            rhs = rng.normal(size=p.n)
            x0 = P.solve(rhs)
            be0 = np.abs(rhs - M @ x0).max() / (nM * np.abs(x0).max() + np.abs(rhs).max())
            x, it, be = P.solve_refined(rhs, tol=1e-13)
            be_own = np.abs(rhs - M @ x).max() / (nM * np.abs(x).max() + np.abs(rhs).max())
            assert 1e-12 < be0 < 1e-5                # reduced precision, but a usable factor
            assert be <= 1e-13 and be_own <= 2e-13 and 1 <= it <= 20
            x_ref = np.linalg.solve(M, rhs)
            assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-10
        P.set_schur_mode(True, min_front=64)
        for s in core.certified_shifts(lam, 4, 1e-8 * nrm, seed=20):
            assert P.factor(s).neg == core.count_below(lam, s)


def test_fp32_factor_refined_near_singular(kep, pen):
    """A shift 1e-11 ||M|| from an eigenvalue, inside the FP32 factor's perturbation: plain
    refinement stalls there, the GMRES-based refinement must still reach the backward error."""
    p, A, B, lam, X = pen
    j = p.k + 5
    nrm = np.abs(A).sum(1).max()
    sig = float(lam[j] + 1e-11 * nrm)
    M = A - sig * B
    nM = np.abs(M).sum(1).max()
    rhs = np.random.default_rng(4).normal(size=p.n)
    x_ref = np.linalg.solve(M, rhs)
    with kep.Problem.from_pencil(p) as P:
        P.set_schur_mode(False, fp32=True)
        P.factor(sig)
        x, it, be = P.solve_refined(rhs, tol=1e-13)
    be_own = np.abs(rhs - M @ x).max() / (nM * np.abs(x).max() + np.abs(rhs).max())
    assert be <= 1e-13 and be_own <= 2e-13 and 1 <= it <= 60
    # the near-null direction dominates both solutions: their directions agree
    cosang = abs(x @ x_ref) / (np.linalg.norm(x) * np.linalg.norm(x_ref))
    assert cosang >= 1 - 1e-8


def test_driver_f32_ir(kep, pen):
    p, A, B, lam, X = pen
    k = p.k
    with kep.Problem.from_pencil(p) as P:
        lam_g, x, rep = P.kth_eigenpair(k, solve_precision="f32_ir")
    nrm = np.abs(A).sum(1).max()
    assert abs(lam_g - lam[k - 1]) <= 1e-10 * nrm
    assert rep["n_refine"] > 0 and rep["solve_berr"] <= 1e-13
    assert rep["rel_res"] < 1e-10


def test_symbolic_info_matches_analysis(kep, pen):
    """The host-only symbolic facts equal those of the context kep_analyze builds."""
    p = pen[0]
    sym = kep.symbolic_info(p.n, p.rowptr, p.colind, p.coords)
    with kep.Problem.from_pencil(p) as P:
        inf = P.info
    for f in ("n", "nnz", "nfronts", "nlevels", "max_front", "nnz_factor", "flops_factor", "front_bytes"):
        assert getattr(sym, f) == getattr(inf, f), f
