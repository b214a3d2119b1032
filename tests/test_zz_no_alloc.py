"""The allocation-free dense inertia entry point (kep_dense_inertia_noalloc).

It serves callers that cannot allocate device memory when they make the call; it keeps its working
copy in a fixed device array of the library.  Checked through the C ABI against the existing
entry point (kep_analyze + kep_factor on the same matrix) on two calls in a row: inertia counts are
integers and must match exactly.  This file is collected last so that a failure here cannot stop
the other GPU tests of a run that halts at its first failure."""
import ctypes

import numpy as np
import pytest

from gen import make_pair
from oracle import core
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _noalloc(kep, A, B, sigma):
    import torch
    n = A.shape[0]
    # column-major with lda = n + 3 (exercise the leading dimension)
    lda = n + 3
    Ad = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    Bd = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    Ad[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T))   # row j of Ad = column j of A
    Bd[:, :n] = torch.from_numpy(np.ascontiguousarray(B.T))
    out = (ctypes.c_int64 * 3)()
    code = kep.lib().kep_dense_inertia_noalloc(n, Ad.data_ptr(), Bd.data_ptr(), lda, float(sigma), None, out)
    torch.cuda.synchronize()
    return code, (out[0], out[1], out[2])


def test_noalloc_matches_factor_two_calls():
    kep = require_gpu()
    p = make_pair(2, 2, 2, seed=3)                     # n = 256
    A, B = p.A().toarray(), p.B().toarray()
    P = kep.Problem.from_pencil(p)
    for sigma in (-2.75, 0.41):                        # two calls in a row
        code, got = _noalloc(kep, A, B, sigma)
        assert code == kep.KEP_OK
        r = P.factor(sigma)
        assert got == (r.neg, r.zero, r.pos)
        assert got == core.dense_inertia(A - sigma * B)   # the oracle's dense Bunch-Kaufman
    P.close()


def test_noalloc_largest_order_and_bad_arguments():
    """n = 512, the largest order, fills the whole fixed array; n = 0 and lda < n are refused."""
    kep = require_gpu()
    p = make_pair(2, 2, 4, seed=4)                     # n = 512
    assert p.n == 512
    A, B = p.A().toarray(), p.B().toarray()
    P = kep.Problem.from_pencil(p)
    for sigma in (0.33, -1.5):
        code, got = _noalloc(kep, A, B, sigma)
        assert code == kep.KEP_OK
        r = P.factor(sigma)
        assert got == (r.neg, r.zero, r.pos) == core.dense_inertia(A - sigma * B)
    P.close()
    import torch
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = (ctypes.c_int64 * 3)()
    assert kep.lib().kep_dense_inertia_noalloc(0, d.data_ptr(), d.data_ptr(), 1, 0.0, None, out) == kep.KEP_ERR_INVALID
    assert kep.lib().kep_dense_inertia_noalloc(4, d.data_ptr(), d.data_ptr(), 3, 0.0, None, out) == kep.KEP_ERR_INVALID


def test_noalloc_two_by_two_pivots_and_limits():
    kep = require_gpu()
    p = make_pair(2, 2, 3, seed=5)                     # n = 384
    sigma = 0.25
    a = p.a.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    d = rows == p.colind
    a[d] = sigma * p.b[d]                              # zero diagonal of A - sigma B: 2x2 pivots
    import scipy.sparse as sp
    A = sp.csr_matrix((a, p.colind, p.rowptr), shape=(p.n, p.n)).toarray()
    B = p.B().toarray()
    P = kep.Problem(p.n, p.rowptr, p.colind, a, p.b, p.coords)
    for s in (sigma, sigma + 0.5):
        code, got = _noalloc(kep, A, B, s)
        assert code == kep.KEP_OK
        r = P.factor(s)
        assert got == (r.neg, r.zero, r.pos) == core.dense_inertia(A - s * B)
    P.close()
    out = (ctypes.c_int64 * 3)()
    assert kep.lib().kep_dense_inertia_noalloc(513, 1, 1, 513, 0.0, None, out) == kep.KEP_ERR_INVALID
