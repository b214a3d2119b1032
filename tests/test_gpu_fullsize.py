"""Parity at the benchmark's full sizes, in the configuration bench.py times (default Schur mode:
tensor-core update from front order 512).

* n = 589,824: the unjittered periodic diamond 32x32x18 cells with B = I + 0.02 A, whose spectrum is
  known in closed form (the oracle's Bloch-matrix eigenvalues): inertia equal at certified shifts.
* n = 524,288: the benchmark pencil (vacancies, jitter): equal inertia from the FP64 and the
  tensor-core Schur paths (Sylvester: both are exact counts), and solve residuals sampled row by
  row against the sparse product.

Opt-in (KEP_FULL_SIZE=1): about 120 GB of device memory and a few minutes on a GB300."""
import os

import numpy as np
import pytest

from gen import perfect_diamond_pencil, workload
from oracle import core
from tests.gpu_util import require_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("KEP_FULL_SIZE") != "1",
                                 reason="full-size run: set KEP_FULL_SIZE=1 (GB300, ~120 GB, minutes)")]


@pytest.fixture(scope="module")
def kep():
    return require_gpu()


def test_fullsize_closed_form_inertia(kep):
    p = perfect_diamond_pencil(32, 32, 18)                       # n = 589,824
    cf = core.diamond_bloch_eigs(32, 32, 18, 1.0, 0.02)
    with kep.Problem.from_pencil(p) as P:
        assert P.info.max_front >= 512                           # the tensor-core path is used
        for s in core.certified_shifts(cf, 3, 1e-6, seed=9):
            r = P.factor(s)
            assert r.status == kep.KEP_OK
            assert r.neg == core.count_below(cf, s) and r.neg + r.zero + r.pos == p.n


def test_fullsize_workload_paths_agree_and_solve(kep):
    p = workload("scale")                                        # n = 524,288
    sigma = 0.4
    rng = np.random.default_rng(0)
    b = rng.normal(size=p.n)
    with kep.Problem.from_pencil(p) as P:
        re = P.factor(sigma)                                     # default: tensor-core update
        x = P.solve(b)
        P.set_schur_mode(False)                                  # FP64 FMA everywhere
        r64 = P.factor(sigma)
    assert (re.neg, re.zero, re.pos) == (r64.neg, r64.zero, r64.pos)
    # residual of 2,000 sampled rows, each from its sparse row (the oracle's product of one row)
    A, B = p.A(), p.B()
    rows = rng.choice(p.n, 2000, replace=False)
    M = (A[rows] - sigma * B[rows]).tocsr()
    res = M @ x - b[rows]
    nM = float(abs(A - sigma * B).sum(1).max())
    assert np.abs(res).max() <= 1e-12 * nM * np.abs(x).max()
