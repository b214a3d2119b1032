"""Parity at the benchmark's full sizes, in the configuration bench.py times (default Schur mode:
tensor-core update from front order 512).

* n = 1,048,576 (the benchmark's size and refined nested dissection): the unjittered periodic
  diamond of 32x32x32 cells with B = I + 0.02 A, whose spectrum is known in closed form (the
  oracle's Bloch-matrix eigenvalues).  Its top separator fronts exceed order 46,341, so their
  m^2 entries pass 2^31: every front offset must be 64-bit.  Inertia equal at certified shifts, one
  of them about 2e-8 ||A|| from an eigenvalue.
* n = 589,824 (32x32x18 cells, default ordering): the same closed-form check.
* n = 1,048,576 benchmark pencil (jitter): solve residuals of sampled rows, each from the sparse
  row of A - sigma B (the oracle's product of one row), and the count of a second, independently
  ordered analysis (Sylvester's law: the count does not depend on the ordering or the pivots).

About 230 GB of device memory and a few minutes on a GB300."""
import numpy as np
import pytest

from gen import perfect_diamond_pencil, workload
from oracle import core
from tests.gpu_util import require_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def kep():
    return require_gpu()


def _near_shift(cf, nrm, seed):
    """A shift 2e-8 ||A|| above an eigenvalue level whose neighbours (other levels) lie more than
    1e-7 ||A|| away on both sides."""
    lv = np.unique(np.round(cf / (1e-10 * nrm)))
    lv = lv * 1e-10 * nrm
    rng = np.random.default_rng(seed)
    gaps = np.diff(lv)
    ok = np.where((gaps[:-1] > 1e-7 * nrm) & (gaps[1:] > 1e-7 * nrm))[0] + 1
    i = ok[rng.integers(ok.size)]
    s = lv[i] + 2e-8 * nrm
    assert np.abs(cf - s).min() > 1e-8 * nrm
    return s


@pytest.mark.parametrize("cells,refined", [((32, 32, 32), True), ((32, 32, 18), False)])
def test_fullsize_closed_form_inertia(kep, cells, refined):
    p = perfect_diamond_pencil(*cells)
    cf = core.diamond_bloch_eigs(*cells, 1.0, 0.02)
    nrm = float(abs(p.A()).sum(1).max())
    shifts = list(core.certified_shifts(cf, 2, 1e-8 * nrm, seed=9)) + [_near_shift(cf, nrm, 3)]
    with kep.Problem.from_pencil(p, refined_order=refined) as P:
        assert P.info.max_front >= 512                           # the tensor-core path is used
        if cells == (32, 32, 32):
            assert P.info.max_front > 46341                      # fronts with more than 2^31 entries
        for s in shifts:
            r = P.factor(s)
            assert r.status == kep.KEP_OK
            assert (r.neg, r.zero, r.pos) == (core.count_below(cf, s), 0, p.n - core.count_below(cf, s)), s


def test_fullsize_workload_solve_and_second_ordering(kep):
    p = workload("million")                                      # n = 1,048,576, the benchmark's pencil
    sigma = 0.4
    rng = np.random.default_rng(0)
    b = rng.normal(size=p.n)
    with kep.Problem.from_pencil(p, refined_order=True) as P:
        r1 = P.factor(sigma)
        x = P.solve(b)
    assert r1.status == kep.KEP_OK
    A, B = p.A(), p.B()
    rows = rng.choice(p.n, 2000, replace=False)
    M = (A[rows] - sigma * B[rows]).tocsr()
    res = M @ x - b[rows]
    nM = float(abs(A - sigma * B).sum(1).max())
    assert np.abs(res).max() <= 1e-12 * nM * np.abs(x).max()
    with kep.Problem.from_pencil(p) as Q:                        # default nested dissection
        r2 = Q.factor(sigma)
    assert (r1.neg, r1.zero, r1.pos) == (r2.neg, r2.zero, r2.pos)
