"""GPU parity of complex Hermitian pencils (kep_analyze_hermitian: the real symmetric embedding of
order 2n on the same kernels): inertia counts at certified shifts (FP64 and tensor-core Schur
updates), complex solves and products, Algorithm 4's lambda_k and x_k, the complex derivatives,
and refined solves with an FP32 factor.

References: the oracle's complex Hermitian dense eigenpairs (c2) and derivative formula (pinned in
test_oracle_hermitian.py), and numpy's dense complex solve."""
import numpy as np
import pytest

from gen import make_pair
from oracle import core
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kep():
    return require_gpu()


@pytest.fixture(scope="module")
def hpen():
    p = make_pair(3, 3, 2, seed=21, phases="peierls")          # n = 576 complex (embedding 1,152)
    A, B = p.A().toarray(), p.B().toarray()
    lam, X = core.gen_eig(A, B)
    return p, A, B, lam, X


def _lower(p):
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    keep = p.colind <= rows
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=p.n))])
    return rp, p.colind[keep], p.a[keep], p.b[keep], rows[keep]


@pytest.mark.parametrize("emulated", [False, True])
def test_inertia_at_certified_shifts(kep, hpen, emulated):
    p, A, B, lam, X = hpen
    nrm = np.abs(A).sum(1).max()
    shifts = core.certified_shifts(lam, 10, 1e-8 * nrm, seed=5)
    with kep.Problem.from_pencil(p) as P:
        assert P.hermitian and P.info.n == 2 * p.n
        P.set_schur_mode(emulated, 64)                        # tensor-core path on small fronts too
        for s in shifts:
            r = P.factor(s)
            assert r.status == kep.KEP_OK
            assert r.neg == core.count_below(lam, s) and r.neg + r.zero + r.pos == p.n
        # the extremes
        assert P.factor(lam[0] - 1.0).neg == 0
        assert P.factor(lam[-1] + 1.0).neg == p.n


def test_lower_pattern_solve_and_products(kep, hpen):
    p, A, B, lam, X = hpen
    nrm = np.abs(A).sum(1).max()
    sig = float(core.certified_shifts(lam, 1, 1e-6 * nrm, seed=6)[0])
    rng = np.random.default_rng(7)
    rhs = rng.normal(size=p.n) + 1j * rng.normal(size=p.n)
    M = A - sig * B
    x_ref = np.linalg.solve(M, rhs)
    rp, ci, a, b, _ = _lower(p)
    with kep.Problem(p.n, rp, ci, a, b, p.coords, lower=True) as P:
        r = P.factor(sig)
        assert r.neg == core.count_below(lam, sig)
        x = P.solve(rhs)
        assert x.dtype == np.complex128
        assert np.abs(x - x_ref).max() <= 1e-9 * np.abs(x_ref).max()
        ax, bx = P.spmv(x_ref)
        assert np.abs(ax - A @ x_ref).max() <= 1e-13 * nrm * np.abs(x_ref).max()
        assert np.abs(bx - B @ x_ref).max() <= 1e-13 * np.abs(B).sum(1).max() * np.abs(x_ref).max()
        # device tensors (complex128) and several right-hand sides
        import torch
        R = np.stack([rhs, rhs.conj(), 1j * rhs])
        Xd = P.solve(torch.from_numpy(R).cuda())
        Xr = np.linalg.solve(M, R.T).T
        assert np.abs(Xd.cpu().numpy() - Xr).max() <= 1e-9 * np.abs(Xr).max()


def test_kth_eigenpair_and_derivatives(kep, hpen):
    p, A, B, lam, X = hpen
    k = p.k
    nrm = np.abs(A).sum(1).max()
    with kep.Problem.from_pencil(p) as P:
        lam_g, x, rep = P.kth_eigenpair(k)
        assert abs(lam_g - lam[k - 1]) <= 1e-10 * nrm
        assert x.dtype == np.complex128
        assert abs(np.vdot(x, B @ x) - 1.0) <= 1e-10                     # x^H B x = 1
        r = A @ x - lam_g * (B @ x)
        assert np.linalg.norm(r) <= 1e-9 * nrm * np.linalg.norm(x)
        assert rep["nu_lo"] < k <= rep["nu_hi"] and rep["nu_hi"] - rep["nu_lo"] <= 20
        # the same eigenvector up to a phase (lambda_k is simple here)
        assert min(abs(lam[k - 2] - lam[k - 1]), abs(lam[k] - lam[k - 1])) > 1e-6 * nrm
        assert abs(abs(np.vdot(X[:, k - 1], B @ x)) - 1.0) <= 1e-8
        ga, gb = P.grad(lam_g, x, 1.0)
    _, GA, GB = core.eig_grad(A, B, k)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    scale = np.abs(GA).max()
    assert ga.dtype == np.complex128
    assert np.abs(ga - GA[rows, p.colind]).max() <= 1e-8 * scale
    assert np.abs(gb - GB[rows, p.colind]).max() <= 1e-8 * scale * max(1.0, abs(lam[k - 1]))
    # lower pattern: an off-diagonal stored entry gets twice G_ij
    rp, ci, a, b, rl = _lower(p)
    with kep.Problem(p.n, rp, ci, a, b, p.coords, lower=True) as P:
        gl, _ = P.grad(lam_g, 3.0 * x, 2.0)                               # any scaling of x
    mult = np.where(ci == rl, 1.0, 2.0)
    assert np.abs(gl - 2.0 * mult * GA[rl, ci]).max() <= 1e-8 * scale


def test_fp32_factor_refined_solve(kep, hpen):
    p, A, B, lam, X = hpen
    nrm = np.abs(A).sum(1).max()
    sig = float(core.certified_shifts(lam, 1, 1e-6 * nrm, seed=8)[0])
    M = A - sig * B
    rng = np.random.default_rng(9)
    rhs = rng.normal(size=p.n) + 1j * rng.normal(size=p.n)
    nM = np.abs(M).sum(1).max()
    with kep.Problem.from_pencil(p) as P:
        P.set_schur_mode(False, fp32=True)
        P.factor(sig)
        x, it, be = P.solve_refined(rhs, tol=1e-13)
    be_own = np.abs(rhs - M @ x).max() / (nM * np.abs(x).max() + np.abs(rhs).max())
    assert be <= 1e-13 and be_own <= 4e-13 and 1 <= it <= 30
    x_ref = np.linalg.solve(M, rhs)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-10


def test_autograd_and_new_values(kep, hpen):
    """KthEigenvalue on complex values: lambda_k and its gradient (d/dRe + i d/dIm of each stored
    entry) against the oracle; set_values with doubled A doubles lambda_k; conjugated values (the
    transposed pencil) keep it; an imaginary diagonal is rejected."""
    import torch
    p, A, B, lam, X = hpen
    k = p.k
    nrm = np.abs(A).sum(1).max()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    _, GA, GB = core.eig_grad(A, B, k)
    scale = np.abs(GA).max()
    with kep.Problem.from_pencil(p) as P:
        a = torch.tensor(p.a, requires_grad=True)
        b = torch.tensor(p.b, requires_grad=True)
        lk = kep.KthEigenvalue.apply(P, k, a, b)
        lk.backward()
        assert abs(lk.item() - lam[k - 1]) <= 1e-10 * nrm
        assert a.grad.dtype == torch.complex128
        assert np.abs(a.grad.numpy() - GA[rows, p.colind]).max() <= 1e-8 * scale
        assert np.abs(b.grad.numpy() - GB[rows, p.colind]).max() <= 1e-8 * scale * max(1.0, abs(lam[k - 1]))
        P.set_values(2.0 * p.a, p.b)
        assert abs(P.kth_eigenpair(k, want_vector=False)[0] - 2.0 * lam[k - 1]) <= 2e-10 * nrm
        P.set_values(np.conj(p.a), np.conj(p.b))
        assert abs(P.kth_eigenpair(k, want_vector=False)[0] - lam[k - 1]) <= 1e-10 * nrm
        bad = p.a.copy()
        bad[np.flatnonzero(rows == p.colind)[3]] += 0.5j
        with pytest.raises(kep.KepError) as e:
            P.set_values(bad, p.b)
        assert e.value.code == kep.KEP_ERR_INVALID


@pytest.mark.slow
def test_peierls_2048_gradient_dense_and_central_differences(kep):
    """The differentiation workload's dense check: a complex Hermitian Peierls pencil of order
    2,048.  The derivatives of lambda_k from the autograd wrapper equal the oracle's dense
    Hellmann-Feynman gradient element by element, and central differences (h = 1e-6) of lambda_k,
    each re-running Algorithm 4 end to end on perturbed values, match them at 100 stored entries
    (50 real and 50 imaginary Hermitian-tied perturbations, entries with |x_i x_j| in the top
    decile).  Each perturbed lambda_k is taken as the Rayleigh quotient of the returned x_k
    (second-order accurate in the vector)."""
    import torch
    p = make_pair(4, 4, 4, seed=31, phases="peierls")          # n = 2,048 complex
    A, B = p.A().toarray(), p.B().toarray()
    k = p.k
    nrm = np.abs(A).sum(1).max()
    lam_ref, GA, GB = core.eig_grad(A, B, k)
    lam_all, _ = core.gen_eig(A, B)
    assert min(lam_all[k] - lam_all[k - 1], lam_all[k - 1] - lam_all[k - 2]) > 1e-6 * nrm   # simple
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    scale = np.abs(GA).max()
    with kep.Problem.from_pencil(p) as P:
        a = torch.tensor(p.a, requires_grad=True)
        b = torch.tensor(p.b, requires_grad=True)
        lk = kep.KthEigenvalue.apply(P, k, a, b)
        lk.backward()
        assert abs(lk.item() - lam_ref) <= 1e-10 * nrm
        ga = a.grad.numpy()
        assert np.abs(ga - GA[rows, p.colind]).max() <= 1e-8 * scale
        assert np.abs(b.grad.numpy() - GB[rows, p.colind]).max() <= 1e-8 * scale * max(1.0, abs(lam_ref))
        # central differences through the full three-stage solve
        off = np.flatnonzero(rows < p.colind)                   # (i, j), i < j; (j, i) is tied to it
        mag = np.abs(GA[rows[off], p.colind[off]])
        top = off[mag >= np.quantile(mag, 0.9)]
        pick = np.random.default_rng(12).choice(top, 100, replace=False)
        pos = {(int(r), int(c)): e for e, (r, c) in enumerate(zip(rows, p.colind))}
        h = 1e-6
        worst = 0.0
        for q, e in enumerate(pick):
            i, j = int(rows[e]), int(p.colind[e])
            et = pos[(j, i)]
            dirn = 1.0 if q < 50 else 1j                        # real, then imaginary tied perturbation
            lam_pm = []
            for sgn in (1.0, -1.0):
                av = p.a.copy()
                av[e] += sgn * h * dirn
                av[et] += sgn * h * np.conj(dirn)
                P.set_values(av, p.b)
                _, x, _ = P.kth_eigenpair(k)
                Ap = A.copy()
                Ap[i, j] += sgn * h * dirn
                Ap[j, i] += sgn * h * np.conj(dirn)
                lam_pm.append(float(np.real(np.vdot(x, Ap @ x) / np.vdot(x, B @ x))))
            fd = (lam_pm[0] - lam_pm[1]) / (2 * h)
            g = ga[e]
            want = 2.0 * (g.real if q < 50 else g.imag)
            err = abs(fd - want)
            worst = max(worst, err)
            assert err <= 1e-5 * scale + 10 * 1e-15 * nrm / h, (q, i, j, fd, want)
        P.set_values(p.a, p.b)
